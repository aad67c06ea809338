/*
 * oracle_core.c -- plain, slow CPU oracle for the CASCI sigma build and RDMs.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares nothing with
 * the CUDA path: strings are found by filtering every bit mask, signs are
 * counted bit by bit, and every matrix element comes from the Slater-Condon
 * rules on spin-orbital determinants.
 *
 * Conventions (the paper's, Sec. III "Support for manipulating determinants"):
 *   - a determinant is one 64-bit word; alpha orbital p is bit p and beta
 *     orbital p is bit n+p, so spin orbital P has spatial part P mod n and
 *     spin P / n;
 *   - |I> = prod of creators in ascending bit order acting on the vacuum, with
 *     all alpha creators to the left of all beta creators (the canonical
 *     alpha-before-beta operator order of the SparseOperator class);
 *   - a_P|..> carries the phase (-1)^(number of occupied Q < P).
 * Hamiltonian (Eq. 1 with V = 0): one-body h_PQ, antisymmetrized two-body
 *   <PQ||RS> = <PQ|RS> - <PQ|SR>,  <PQ|RS> = (pr|qs) d(sP,sR) d(sQ,sS),
 * which is the chemist-notation (pq|rs) form of the spin-free operator.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------- bit-level fermion operators ---------- */

static int occ_below(uint64_t d, int P) {
  int c = 0;
  for (int Q = 0; Q < P; ++Q) c += (int)((d >> Q) & 1ULL);
  return c;
}

/* a_P |d>: returns the phase (+1/-1) and updates d, or 0 when P is empty. */
static int op_ann(uint64_t *d, int P) {
  if (!((*d >> P) & 1ULL)) return 0;
  int s = (occ_below(*d, P) & 1) ? -1 : 1;
  *d &= ~(1ULL << P);
  return s;
}

/* a^dagger_P |d>: returns the phase and updates d, or 0 when P is occupied. */
static int op_cre(uint64_t *d, int P) {
  if ((*d >> P) & 1ULL) return 0;
  int s = (occ_below(*d, P) & 1) ? -1 : 1;
  *d |= (1ULL << P);
  return s;
}

static int popc64(uint64_t x) {
  int c = 0;
  while (x) { c += (int)(x & 1ULL); x >>= 1; }
  return c;
}

/* ---------- spin-orbital integrals ---------- */

static double h_so(int n, const double *h, int P, int Q) {
  if (P / n != Q / n) return 0.0;
  return h[(P % n) * n + (Q % n)];
}

/* <PQ|RS> = (pr|qs) when spin(P)=spin(R) and spin(Q)=spin(S). */
static double v_so(int n, const double *eri, int P, int Q, int R, int S) {
  if (P / n != R / n || Q / n != S / n) return 0.0;
  int p = P % n, q = Q % n, r = R % n, s = S % n;
  return eri[(((size_t)p * n + r) * n + q) * n + s];
}

static double va_so(int n, const double *eri, int P, int Q, int R, int S) {
  return v_so(n, eri, P, Q, R, S) - v_so(n, eri, P, Q, S, R);
}

/* ---------- Slater-Condon rules ---------- */

/* <I|H|J> for determinants over 2n spin orbitals. */
double ora_hij(int n, const double *h, const double *eri, uint64_t I, uint64_t J) {
  uint64_t x = I ^ J;
  int nd = popc64(x);
  int nso = 2 * n;
  /* H of Eq. 1 conserves the number of alpha and of beta electrons: determinants
   * of different sectors do not couple (and the replacement analysis below
   * assumes equal counts). */
  const uint64_t amask = (n >= 64) ? ~0ULL : ((1ULL << n) - 1ULL);
  if (popc64(I & amask) != popc64(J & amask) || popc64(I & ~amask) != popc64(J & ~amask)) return 0.0;
  if (nd == 0) {
    double e = 0.0;
    for (int P = 0; P < nso; ++P) {
      if (!((I >> P) & 1ULL)) continue;
      e += h_so(n, h, P, P);
      for (int Q = 0; Q < nso; ++Q)
        if ((I >> Q) & 1ULL) e += 0.5 * va_so(n, eri, P, Q, P, Q);
    }
    return e;
  }
  if (nd == 2) {
    /* I = J - p + m */
    int m = -1, p = -1;
    for (int P = 0; P < nso; ++P) {
      if (((x >> P) & 1ULL) == 0) continue;
      if ((I >> P) & 1ULL) m = P; else p = P;
    }
    uint64_t t = J;
    int s = op_ann(&t, p);
    s *= op_cre(&t, m);
    double v = h_so(n, h, m, p);
    for (int K = 0; K < nso; ++K)
      if (((J >> K) & 1ULL) && K != p) v += va_so(n, eri, m, K, p, K);
    return s * v;
  }
  if (nd == 4) {
    /* I = J - {p,q} + {m,o}, m<o, p<q:  <I|H|J> = <mo||pq> <I|a+m a+o a_q a_p|J> */
    int m = -1, o = -1, p = -1, q = -1;
    for (int P = 0; P < nso; ++P) {
      if (((x >> P) & 1ULL) == 0) continue;
      if ((I >> P) & 1ULL) { if (m < 0) m = P; else o = P; }
      else { if (p < 0) p = P; else q = P; }
    }
    uint64_t t = J;
    int s = op_ann(&t, p);
    s *= op_ann(&t, q);
    s *= op_cre(&t, o);
    s *= op_cre(&t, m);
    return s * va_so(n, eri, m, o, p, q);
  }
  return 0.0;
}

/* Sigma over an arbitrary list of determinants (selected CI, Sec. II.A.2):
 * S[v][i] = sum_j <D_i|H|D_j> C[v][j], the sum over the j within two
 * replacements of i (every other element vanishes by the Slater-Condon rules).
 * n <= 32 (2n spin orbitals in one 64-bit word). */
void ora_sci_sigma(int n, long nd, const uint64_t *dets, const double *h, const double *eri, int nvec,
                   const double *C, double *S) {
#pragma omp parallel for schedule(dynamic, 8)
  for (long i = 0; i < nd; ++i) {
    for (int v = 0; v < nvec; ++v) S[(long)v * nd + i] = 0.0;
    for (long j = 0; j < nd; ++j) {
      if (popc64(dets[i] ^ dets[j]) > 4) continue;
      const double hij = ora_hij(n, h, eri, dets[i], dets[j]);
      for (int v = 0; v < nvec; ++v) S[(long)v * nd + i] += hij * C[(long)v * nd + j];
    }
  }
}

/* ---------- strings ---------- */

/* All n-bit masks with k bits set, ascending; returns the count. */
long ora_strings(int n, int k, uint32_t *out) {
  long c = 0;
  for (uint64_t m = 0; m < (1ULL << n); ++m)
    if (popc64(m) == k) {
      if (out) out[c] = (uint32_t)m;
      ++c;
    }
  return c;
}

/* Address of a string mask by linear search in the ascending list. */
static long addr_of(const uint32_t *str, long N, uint32_t m) {
  for (long i = 0; i < N; ++i)
    if (str[i] == m) return i;
  return -1;
}

/* Dense single-replacement table of one spin: for string I and orbitals p,q,
 * J[I][p][q] = address of a+_p a_q |I> and sgn its phase, or J = -1, sgn = 0. */
void ora_single_table(int n, int k, int *Jtab, signed char *sgn) {
  long N = ora_strings(n, k, NULL);
  uint32_t *str = (uint32_t *)malloc(sizeof(uint32_t) * (N > 0 ? N : 1));
  ora_strings(n, k, str);
  for (long I = 0; I < N; ++I)
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        uint64_t d = str[I];
        int s = op_ann(&d, q);
        if (s) s *= op_cre(&d, p);
        size_t o = ((size_t)I * n + p) * n + q;
        if (s == 0) { Jtab[o] = -1; sgn[o] = 0; }
        else { Jtab[o] = (int)addr_of(str, N, (uint32_t)d); sgn[o] = (signed char)s; }
      }
  free(str);
}

/* ---------- determinant space ---------- */

typedef struct {
  int n, na, nb;
  long Na, Nb;
  uint32_t *sa, *sb;
  /* strings within two replacements of each string (including itself), listed
   * by replacement degree: the string itself, then single, then double
   * replacements; near_*_end1[i] marks the end of the degree <= 1 part */
  long *near_a_ptr, *near_b_ptr;
  long *near_a, *near_b;
  long *near_a_end1, *near_b_end1;
} space_t;

static void build_near(const uint32_t *s, long N, long **ptr, long **idx, long **end1) {
  long *p = (long *)malloc(sizeof(long) * (N + 1));
  long *e1 = (long *)malloc(sizeof(long) * (N > 0 ? N : 1));
  p[0] = 0;
  for (long i = 0; i < N; ++i) {
    long c = 0;
    for (long j = 0; j < N; ++j)
      if (popc64((uint64_t)(s[i] ^ s[j])) <= 4) ++c;
    p[i + 1] = p[i] + c;
  }
  long *x = (long *)malloc(sizeof(long) * (p[N] > 0 ? p[N] : 1));
  for (long i = 0; i < N; ++i) {
    long c = p[i];
    for (int deg2 = 0; deg2 <= 4; deg2 += 2) {
      for (long j = 0; j < N; ++j)
        if (popc64((uint64_t)(s[i] ^ s[j])) == deg2) x[c++] = j;
      if (deg2 == 2) e1[i] = c;
    }
  }
  *ptr = p;
  *idx = x;
  *end1 = e1;
}

static void space_init(space_t *sp, int n, int na, int nb) {
  sp->n = n; sp->na = na; sp->nb = nb;
  sp->Na = ora_strings(n, na, NULL);
  sp->Nb = ora_strings(n, nb, NULL);
  sp->sa = (uint32_t *)malloc(sizeof(uint32_t) * sp->Na);
  sp->sb = (uint32_t *)malloc(sizeof(uint32_t) * sp->Nb);
  ora_strings(n, na, sp->sa);
  ora_strings(n, nb, sp->sb);
  build_near(sp->sa, sp->Na, &sp->near_a_ptr, &sp->near_a, &sp->near_a_end1);
  build_near(sp->sb, sp->Nb, &sp->near_b_ptr, &sp->near_b, &sp->near_b_end1);
}

static void space_free(space_t *sp) {
  free(sp->sa); free(sp->sb);
  free(sp->near_a_ptr); free(sp->near_b_ptr);
  free(sp->near_a); free(sp->near_b);
  free(sp->near_a_end1); free(sp->near_b_end1);
}

static uint64_t det_of(const space_t *sp, long ia, long ib) {
  return (uint64_t)sp->sa[ia] | ((uint64_t)sp->sb[ib] << sp->n);
}

/* Full Hamiltonian matrix [Ndet][Ndet], determinant index = ia*Nb + ib. */
void ora_hmat_dense(int n, int na, int nb, const double *h, const double *eri, double *H) {
  space_t sp;
  space_init(&sp, n, na, nb);
  long Nd = sp.Na * sp.Nb;
#pragma omp parallel for schedule(dynamic, 16)
  for (long i = 0; i < Nd; ++i) {
    uint64_t I = det_of(&sp, i / sp.Nb, i % sp.Nb);
    for (long j = 0; j < Nd; ++j) {
      uint64_t J = det_of(&sp, j / sp.Nb, j % sp.Nb);
      H[i * Nd + j] = ora_hij(n, h, eri, I, J);
    }
  }
  space_free(&sp);
}

/* Diagonal <I|H|I> for all determinants. */
void ora_hdiag(int n, int na, int nb, const double *h, const double *eri, double *d) {
  space_t sp;
  space_init(&sp, n, na, nb);
  long Nd = sp.Na * sp.Nb;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < Nd; ++i) {
    uint64_t I = det_of(&sp, i / sp.Nb, i % sp.Nb);
    d[i] = ora_hij(n, h, eri, I, I);
  }
  space_free(&sp);
}

/* Direct sigma: S[v][i] = sum_J <I|H|J> C[v][J] for the output rows listed in
 * rows[0..nrows) (all rows when rows == NULL).  Vectors are [nvec][Na*Nb]; with
 * a row list S holds nrows entries per vector, in list order. */
void ora_sigma(int n, int na, int nb, const double *h, const double *eri, int nvec,
               const double *C, double *S, long nrows, const long *rows) {
  space_t sp;
  space_init(&sp, n, na, nb);
  long Nd = sp.Na * sp.Nb;
  long nout = rows ? nrows : Nd;
#pragma omp parallel
  {
    double *acc = (double *)malloc(sizeof(double) * (nvec > 0 ? nvec : 1));
#pragma omp for schedule(dynamic, 64)
    for (long o = 0; o < nout; ++o) {
      long i = rows ? rows[o] : o;
      long ia = i / sp.Nb, ib = i % sp.Nb;
      uint64_t I = det_of(&sp, ia, ib);
      for (int v = 0; v < nvec; ++v) acc[v] = 0.0;
      for (long x = sp.near_a_ptr[ia]; x < sp.near_a_ptr[ia + 1]; ++x) {
        long ja = sp.near_a[x];
        int da = popc64((uint64_t)(sp.sa[ia] ^ sp.sa[ja])) / 2;
        /* a determinant at most two replacements away: beta part limited to 2 - da */
        long y_end = (da == 0) ? sp.near_b_ptr[ib + 1]
                   : (da == 1) ? sp.near_b_end1[ib] : sp.near_b_ptr[ib] + 1;
        for (long y = sp.near_b_ptr[ib]; y < y_end; ++y) {
          long jb = sp.near_b[y];
          int db = popc64((uint64_t)(sp.sb[ib] ^ sp.sb[jb])) / 2;
          if (da + db > 2) continue;
          double hij = ora_hij(n, h, eri, I, det_of(&sp, ja, jb));
          if (hij == 0.0) continue;
          long j = ja * sp.Nb + jb;
          for (int v = 0; v < nvec; ++v) acc[v] += hij * C[(size_t)v * Nd + j];
        }
      }
      for (int v = 0; v < nvec; ++v) S[(size_t)v * nout + o] = acc[v];
    }
    free(acc);
  }
  space_free(&sp);
}

/* ---------- reduced density matrices (Eqs. for gamma_1, gamma_2) ---------- */

/* Spin-free 1- and 2-RDM between bra and ket vectors:
 *   g1[p][q]       = sum_s    <bra| a+_{ps} a_{qs} |ket>
 *   g2[p][q][r][s] = sum_{st} <bra| a+_{ps} a+_{rt} a_{st} a_{qs} |ket>
 * (chemist order; = <E_pq E_rs> - d_qr <E_ps>).  Either output may be NULL.
 * Each element is found by applying the operator string to every ket
 * determinant and looking up the bra coefficient of the result. */
void ora_rdm12(int n, int na, int nb, const double *bra, const double *ket, double *g1, double *g2) {
  space_t sp;
  space_init(&sp, n, na, nb);
  long Nd = sp.Na * sp.Nb;
  /* address maps from mask to string index */
  long *ma = (long *)malloc(sizeof(long) << n), *mb = (long *)malloc(sizeof(long) << n);
  for (long m = 0; m < (1L << n); ++m) ma[m] = mb[m] = -1;
  for (long i = 0; i < sp.Na; ++i) ma[sp.sa[i]] = i;
  for (long i = 0; i < sp.Nb; ++i) mb[sp.sb[i]] = i;
  uint64_t lowmask = (n == 32) ? 0xffffffffULL : ((1ULL << n) - 1ULL);
  int n2 = n * n;
  if (g1) {
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        double acc = 0.0;
        for (int sg = 0; sg < 2; ++sg)
          for (long j = 0; j < Nd; ++j) {
            double c = ket[j];
            if (c == 0.0) continue;
            uint64_t d = det_of(&sp, j / sp.Nb, j % sp.Nb);
            int s = op_ann(&d, q + sg * n);
            if (!s) continue;
            s *= op_cre(&d, p + sg * n);
            if (!s) continue;
            long ia = ma[d & lowmask], ib = mb[(d >> n) & lowmask];
            acc += s * bra[ia * sp.Nb + ib] * c;
          }
        g1[p * n + q] = acc;
      }
  }
  if (g2) {
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q)
        for (int r = 0; r < n; ++r)
          for (int s_ = 0; s_ < n; ++s_) {
            double acc = 0.0;
            for (int sg = 0; sg < 2; ++sg)
              for (int tg = 0; tg < 2; ++tg)
                for (long j = 0; j < Nd; ++j) {
                  double c = ket[j];
                  if (c == 0.0) continue;
                  uint64_t d = det_of(&sp, j / sp.Nb, j % sp.Nb);
                  int s = op_ann(&d, q + sg * n);
                  if (!s) continue;
                  s *= op_ann(&d, s_ + tg * n);
                  if (!s) continue;
                  s *= op_cre(&d, r + tg * n);
                  if (!s) continue;
                  s *= op_cre(&d, p + sg * n);
                  if (!s) continue;
                  long ia = ma[d & lowmask], ib = mb[(d >> n) & lowmask];
                  acc += s * bra[ia * sp.Nb + ib] * c;
                }
            g2[(((size_t)p * n + q) * n + r) * n + s_] = acc;
          }
  }
  (void)n2;
  free(ma); free(mb);
  space_free(&sp);
}

/* Spin-free 3-RDM (Sec. II.A.1, the three-body gamma_3 of the string CI codes,
 * summed over spin):
 *   g3[p][q][r][s][t][u] = sum_{s1 s2 s3} <bra| a+_{p s1} a+_{r s2} a+_{t s3} a_{u s3} a_{s s2} a_{q s1} |ket>
 * (chemist-like order: creator p pairs with annihilator q, r with s, t with u).
 * Like ora_rdm12: every element by applying the operator string to each ket
 * determinant.  Cost n^6 * 8 * N_det: for small spaces only. */
void ora_rdm3(int n, int na, int nb, const double *bra, const double *ket, double *g3) {
  space_t sp;
  space_init(&sp, n, na, nb);
  long Nd = sp.Na * sp.Nb;
  long *ma = (long *)malloc(sizeof(long) << n), *mb = (long *)malloc(sizeof(long) << n);
  for (long m = 0; m < (1L << n); ++m) ma[m] = mb[m] = -1;
  for (long i = 0; i < sp.Na; ++i) ma[sp.sa[i]] = i;
  for (long i = 0; i < sp.Nb; ++i) mb[sp.sb[i]] = i;
  uint64_t lowmask = (1ULL << n) - 1ULL;
  long n3 = (long)n * n * n;
#pragma omp parallel for schedule(dynamic)
  for (long pqr = 0; pqr < n3; ++pqr) {
    int p = (int)(pqr / (n * n)), q = (int)((pqr / n) % n), r = (int)(pqr % n);
    for (int s_ = 0; s_ < n; ++s_)
      for (int t = 0; t < n; ++t)
        for (int u = 0; u < n; ++u) {
          double acc = 0.0;
          for (int s1 = 0; s1 < 2; ++s1)
            for (int s2 = 0; s2 < 2; ++s2)
              for (int s3 = 0; s3 < 2; ++s3)
                for (long j = 0; j < Nd; ++j) {
                  double c = ket[j];
                  if (c == 0.0) continue;
                  uint64_t d = det_of(&sp, j / sp.Nb, j % sp.Nb);
                  int s = op_ann(&d, q + s1 * n);
                  if (!s) continue;
                  s *= op_ann(&d, s_ + s2 * n);
                  if (!s) continue;
                  s *= op_ann(&d, u + s3 * n);
                  if (!s) continue;
                  s *= op_cre(&d, t + s3 * n);
                  if (!s) continue;
                  s *= op_cre(&d, r + s2 * n);
                  if (!s) continue;
                  s *= op_cre(&d, p + s1 * n);
                  if (!s) continue;
                  long ia = ma[d & lowmask], ib = mb[(d >> n) & lowmask];
                  acc += s * bra[ia * sp.Nb + ib] * c;
                }
          g3[((((((size_t)p * n + q) * n + r) * n + s_) * n + t) * n) + u] = acc;
        }
  }
  free(ma); free(mb);
  space_free(&sp);
}

/* Selected 2-RDM elements: idx[4*e..4*e+3] = (p,q,r,s); out[e] = g2[p][q][r][s]. */
void ora_rdm2_elements(int n, int na, int nb, const double *bra, const double *ket,
                       long nel, const int *idx, double *out) {
  space_t sp;
  space_init(&sp, n, na, nb);
  long Nd = sp.Na * sp.Nb;
  long *ma = (long *)malloc(sizeof(long) << n), *mb = (long *)malloc(sizeof(long) << n);
  for (long m = 0; m < (1L << n); ++m) ma[m] = mb[m] = -1;
  for (long i = 0; i < sp.Na; ++i) ma[sp.sa[i]] = i;
  for (long i = 0; i < sp.Nb; ++i) mb[sp.sb[i]] = i;
  uint64_t lowmask = (1ULL << n) - 1ULL;
#pragma omp parallel for schedule(dynamic)
  for (long e = 0; e < nel; ++e) {
    int p = idx[4 * e], q = idx[4 * e + 1], r = idx[4 * e + 2], s_ = idx[4 * e + 3];
    double acc = 0.0;
    for (int sg = 0; sg < 2; ++sg)
      for (int tg = 0; tg < 2; ++tg)
        for (long j = 0; j < Nd; ++j) {
          double c = ket[j];
          if (c == 0.0) continue;
          uint64_t d = det_of(&sp, j / sp.Nb, j % sp.Nb);
          int s = op_ann(&d, q + sg * n);
          if (!s) continue;
          s *= op_ann(&d, s_ + tg * n);
          if (!s) continue;
          s *= op_cre(&d, r + tg * n);
          if (!s) continue;
          s *= op_cre(&d, p + sg * n);
          if (!s) continue;
          long ia = ma[d & lowmask], ib = mb[(d >> n) & lowmask];
          acc += s * bra[ia * sp.Nb + ib] * c;
        }
    out[e] = acc;
  }
  free(ma); free(mb);
  space_free(&sp);
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

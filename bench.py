"""Benchmark of the CASCI hot path on CAS(14,14): 7 alpha + 7 beta electrons in
14 orbitals, 11,778,624 determinants, seeded synthetic integrals (28 factors,
seed 2), inputs resident in HBM (vectors of 94 MB, subspace > 2 GB: larger than
the 129 MB L2, so no flush is needed between steps).

One step = a Davidson-Liu solve of the lowest root from the standard guess to an
FP64-class residual of `--tol` (default 1e-5, energy error <= |r|^2/gap ~ 1e-10 Eh),
in the chosen sigma precision (default: split-BF16 tensor-core sigma on FP32 vectors,
then Jacobi-Davidson refinement with the double-FP32 sigma), followed by the
spin-free 1- and 2-RDMs of the root (tensor-core Gram in the reduced-precision modes).
``value`` = determinants x sigma vectors built in the timed steps / time (det/s).
The same run also times one FP64 solve of the same problem, which gives the
reference energy and the "mixed vs FP64 time-to-1e-8 Eh" comparison.

--impl reference times the CPU oracle (the plain Slater-Condon program under
oracle/) on a bounded random sample of output determinants of the same workload.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth_inputs as si  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")
# FP64 pipe: nominal GB300 FP64 rate (152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz); a DFMA
# probe measured 1.197 TF/s.  FP32 pipe: 152 x 128 FFMA/clk x 2 x 2.07 GHz.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 80.5
TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor ratio
# double-FP32 multiply-add: about 12 FP32 pipe operations for 2 FP64-equivalent flops
DF32_PEAK_TFLOPS = FP32_PEAK_TFLOPS / 6.0
OZ_PAIRS = 26  # digit pairs (i, j), 1 <= i, j <= 6, i + j <= 8, of the tensor-core RDM Gram

WORKLOADS = {"cas1414": si.CAS1414, "cas1212": si.CAS1212, "cas88": si.CAS88}
WORKLOAD_NAMES = {"cas1414": "CAS(14,14) 7a+7b in 14 orbitals, 11,778,624 determinants, seed 2, 28 factors",
                  "cas1212": "CAS(12,12) 6a+6b in 12 orbitals, 853,776 determinants, seed 1, 24 factors",
                  "cas88": "CAS(8,8) 4a+4b in 8 orbitals, 4,900 determinants, seed 0, 16 factors"}
METRIC = "CASCI H*C det/s and Davidson time-to-1e-8 Eh, CAS(14,14), mixed vs FP64, 1 GB300"


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return (p.get("hbm_gbs", 6800.0), p.get("bf16_tflops", 1900.0), p.get("bf16_tflops_sustained", 1700.0),
                "measured")
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def traffic_table():
    try:
        with open(TRAFFIC_FILE) as f:
            return json.load(f)
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        smax = [v for v in (num(r[2]) for r in rows) if v is not None]
        pw = [v for v in (num(r[3]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ oracle (CPU baseline / reference arm)
def oracle_sigma_rate(cfg, seconds=10.0, seed=21):
    """Oracle direct sigma on a bounded random sample of output determinants.
    Returns (det/s, rows, wall seconds, threads)."""
    import oracle
    n, na, nb = cfg["norb"], cfg["nalpha"], cfg["nbeta"]
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    Na, Nb = si.n_strings(n, na), si.n_strings(n, nb)
    C = si.random_vectors(1, Na, Nb, seed=7).reshape(1, -1)
    rng = np.random.default_rng(seed)
    t = []
    for m in (256, 4096):  # per-call set-up cost and per-row cost
        probe = rng.integers(0, Na * Nb, size=m)
        t0 = time.perf_counter()
        oracle.sigma(n, na, nb, h, eri, C, rows=probe)
        t.append(time.perf_counter() - t0)
    per_row = max((t[1] - t[0]) / 3840.0, 1e-7)
    nrows = int(max(4096, min(5_000_000, max(seconds - t[0], 0.5) / per_row)))
    rows = rng.integers(0, Na * Nb, size=nrows)
    t0 = time.perf_counter()
    oracle.sigma(n, na, nb, h, eri, C, rows=rows)
    dt = time.perf_counter() - t0
    return nrows / dt, nrows, dt, oracle.num_threads()


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    cfg = WORKLOADS[args.workload]
    for _ in range(args.warmup):
        oracle_sigma_rate(cfg, seconds=1.0)
    t_all, rows_tot, nthreads = 0.0, 0, 1
    for _ in range(args.steps):
        _, rows, dt, nthreads = oracle_sigma_rate(cfg, seconds=args.ref_seconds)
        t_all += dt
        rows_tot += rows
    value = rows_tot / t_all
    sample = (f"oracle direct sigma (Slater-Condon, FP64) on {rows_tot} random output determinants of "
              f"{args.workload}, {args.steps} steps")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "det/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_all / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.workload], "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": "det/s", "cores": nthreads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "det/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


# ------------------------------------------------------------------ roofline bookkeeping
def kernel_work(name, prob, n_sig64, n_sigm, n_rdm, tables):
    """(algorithmic work, unit, bound, peak, peak note) of all launches of `name`."""
    hbm, bf16, bf16s, src = peaks()
    n = prob.norb
    nd = prob.ndet
    nk = lambda ne: ne * (n - ne) + ne  # noqa: E731
    nka, nkb = nk(prob.nalpha), nk(prob.nbeta)
    npair = n * (n + 1) // 2
    nnz_a, nnz_b = tables
    if name == "ab_fp64":
        return 2.0 * nd * nka * nkb * n_sig64, "TFLOP/s", "alu", FP64_PEAK_TFLOPS, "FP64 pipe, nominal"
    if name == "ss_spmm":
        return (2.0 * (nnz_a * prob.nb + nnz_b * prob.na) * n_sig64, "TFLOP/s", "alu", FP64_PEAK_TFLOPS,
                "FP64 pipe, nominal")
    if name == "ss_spmm_f32":
        return (2.0 * (nnz_a * prob.nb + nnz_b * prob.na) * n_sigm, "TFLOP/s", "alu", FP32_PEAK_TFLOPS,
                "FP32 pipe, nominal")
    if name == "ab_mma_bf16x2":
        return (3 * 2.0 * nd * npair * nka * n_sigm, "TFLOP/s", "tensor", bf16s,
                f"bf16 dense sustained ({src})")
    if name == "ab_mma_tf32":
        return (2.0 * nd * npair * nka * n_sigm, "TFLOP/s", "tensor", bf16s * TF32_OVER_BF16,
                f"bf16 dense sustained ({src}) x nominal tf32/bf16 ratio")
    if name == "gram":
        nt = (n * n + 63) // 64  # symmetric Gram: tiles ta <= tb of 64 x 64
        return (2.0 * 64 * 64 * nt * (nt + 1) // 2 * nd * n_rdm, "TFLOP/s", "alu", FP64_PEAK_TFLOPS,
                "FP64 pipe, nominal")
    if name == "ss_mma_bf16x2":
        # one GEMM [H_a | C] [C^T | H_b]^T per vector, 3 BF16 products
        return (3 * 2.0 * prob.na * prob.nb * (prob.na + prob.nb) * n_sigm, "TFLOP/s", "tensor", bf16s,
                f"bf16 dense sustained ({src})")
    if name == "ss_mma_tf32":
        return (2.0 * prob.na * prob.nb * (prob.na + prob.nb) * n_sigm, "TFLOP/s", "tensor",
                bf16s * TF32_OVER_BF16, f"bf16 dense sustained ({src}) x nominal tf32/bf16 ratio")
    if name == "ab_df":
        return (2.0 * nd * nka * nkb * n_sig64, "TFLOP/s", "alu", DF32_PEAK_TFLOPS,
                "FP32 pipe / 6 (12 FP32 operations per double-FP32 multiply-add)")
    if name == "ss_spmm_df":
        return (2.0 * (nnz_a * prob.nb + nnz_b * prob.na) * n_sig64, "TFLOP/s", "alu", DF32_PEAK_TFLOPS,
                "FP32 pipe / 6 (12 FP32 operations per double-FP32 multiply-add)")
    if name == "ab_oz":
        # FORTE_OZ64 alpha-beta term: 26 BF16 digit-pair products of the contraction
        # F[rs][Jb] = sum_k A[rs][k] B[Jb][k] over the n(n+1)/2 pairs and n_kl(alpha)
        return (OZ_PAIRS * 2.0 * nd * npair * nka * n_sig64, "TFLOP/s", "tensor", bf16s,
                f"bf16 dense sustained ({src})")
    if name in ("gram_oz_u", "gram_oz_v"):
        # 26 BF16 digit-pair products (i + j <= 8 of six digits) of the Gram of the
        # symmetric (n(n+1)/2 rows) or antisymmetric (n(n-1)/2 rows) one-body images
        rows = n * (n + 1) // 2 if name == "gram_oz_u" else n * (n - 1) // 2
        return (OZ_PAIRS * 2.0 * rows * rows * nd * n_rdm, "TFLOP/s", "tensor", bf16s,
                f"bf16 dense sustained ({src})")
    return None


def _sig(x, digits=4):
    """Round to `digits` significant digits (keeps the JSON line short)."""
    if x is None or not np.isfinite(x) or x == 0:
        return x
    return float(f"{x:.{digits}g}")


SOLVERS = {
    "fp64": "Davidson-Liu, FP64 sigma and vectors",
    "df32": "Davidson-Liu, double-FP32 sigma, FP64 vectors",
    "oz64": "Davidson-Liu, digit-slice tensor-core sigma, FP64 vectors",
    "bf16x2": "Davidson-Liu on FP32 vectors with the split-BF16 tensor-core sigma to 1e-3, then "
              "Jacobi-Davidson with the digit-slice FP64-class sigma",
    "tf32": "Davidson-Liu on FP32 vectors with the TF32 tensor-core sigma to 1e-2, then "
            "Jacobi-Davidson with the digit-slice FP64-class sigma",
}


def combine_ranks(t_ms, units, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: the units all ranks processed over the
    slowest rank's time.  Returns (max time in ms, summed units, units per second)."""
    if dist is None:
        return t_ms, units, units / (t_ms / 1000.0)
    import torch
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    uu = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    t, u = float(tt.item()), float(uu.item())
    return t, u, u / (t / 1000.0)


def run_ours(args):
    import torch
    import paper_2405_10197_gb300 as fg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    cfg = WORKLOADS[args.workload]
    n, na, nb = cfg["norb"], cfg["nalpha"], cfg["nbeta"]
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    modes = {"fp64": fg.FORTE_FP64, "tf32": fg.FORTE_TF32, "bf16x2": fg.FORTE_BF16X2, "df32": fg.FORTE_DF32,
             "oz64": fg.FORTE_OZ64}
    mode = modes[args.precision]
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    prob = fg.CASProblem(n, na, nb, h, eri, precision=mode, stream=stream)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    nd = prob.ndet
    nroots, tol = 1, args.tol
    g1 = torch.empty(n, n, dtype=torch.float64, device="cuda")
    g2 = torch.empty((n,) * 4, dtype=torch.float64, device="cuda")
    root = torch.empty(nroots, prob.na, prob.nb, dtype=torch.float64, device="cuda")

    def solve(m, t=tol, nr=nroots, out=root):
        fg.forte_set_precision(prob.ctx, m)
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        fg.forte_davidson(prob.ctx, nr, t, allow_not_converged=True)
        d1.record(stream)
        E, rn, it = fg.forte_get_roots(prob.ctx, nr, out)
        return [float(e) for e in E], [float(r) for r in rn], it, (d0, d1)

    # Reference and comparison solves, outside the timed region.  The FP64 reference
    # is converged to a residual of 1e-10 (energy error <= r^2/gap); every other
    # solve's time-to-1e-8 Eh is its time to `tol`, with its energy error against it.
    ttl = None
    if args.fp64_compare:
        details_ref = {}
        fg.forte_set_davidson_params(prob.ctx, 12, 2, args.ref_max_iter, 1e-8)
        E_ref, rn_ref, it_ref, ev = solve(fg.FORTE_FP64, t=args.ref_tol)
        torch.cuda.synchronize()
        ms_ref = ev[0].elapsed_time(ev[1])
        fg.forte_set_davidson_params(prob.ctx, 12, 2, 200, 1e-8)
        # gap to the next root (2-root solve in the mixed mode; bounds the reference error)
        two = torch.empty(2, prob.na, prob.nb, dtype=torch.float64, device="cuda")
        E2, _, _, _ = solve(fg.FORTE_BF16X2, t=1e-6, nr=2, out=two)
        gap = E2[1] - E2[0]
        del two
        cmp = {}
        for name in ("fp64", "tf32"):
            if name == args.precision:
                continue
            if name != "fp64":
                solve(modes[name])  # warm-up (scratch, tables)
            E, rn, it, ev = solve(modes[name])
            torch.cuda.synchronize()
            cmp[name] = {"ms": ev[0].elapsed_time(ev[1]), "err": abs(E[0] - E_ref[0]), "it": it, "rn": rn[0]}
        ttl = {"ref": {"E": E_ref[0], "rn": _sig(rn_ref[0], 3), "it": it_ref, "ms": _sig(ms_ref)},
               "gap": _sig(gap, 6), "cmp": cmp}
        details_ref = {"reference_fp64": {"energy": E_ref[0], "residual": rn_ref[0], "iterations": it_ref,
                                          "ms": ms_ref, "tol": args.ref_tol, "max_iter": args.ref_max_iter},
                       "gap_to_next_root": gap, "comparison_solves": cmp}
    E_ref = ttl["ref"]["E"] if ttl else None

    for _ in range(args.warmup):
        solve(mode)
        fg.forte_rdms(prob.ctx, root[0], g1, g2, n)
    torch.cuda.synchronize()

    s0 = fg.forte_get_counters(prob.ctx)
    clocks = ClockSampler(dev)
    clocks.start()
    fg.forte_profile_enable(prob.ctx, 1)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per_step = []
    ev0.record(stream)
    for _ in range(args.steps):
        E, rn, it, dev_ev = solve(mode)
        fg.forte_rdms(prob.ctx, root[0], g1, g2, n)
        per_step.append((E[0], rn[0], it, dev_ev))
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    fg.forte_profile_enable(prob.ctx, 0)
    t_ms = ev0.elapsed_time(ev1)
    s1 = fg.forte_get_counters(prob.ctx)
    n_sig64, n_sigm = s1[0] - s0[0], s1[1] - s0[1]
    prof = fg.profile_table(prob.ctx)
    launches = sum(v[0] for v in prof.values())
    t_ms, _, value = combine_ranks(t_ms, nd * (n_sig64 + n_sigm), dist, "cuda")

    # rooflines
    traffic = traffic_table()
    nnz = fg_nnz(prob)
    rows = {}
    for name, (cnt, ms) in prof.items():
        w = kernel_work(name, prob, n_sig64, n_sigm, args.steps, nnz)
        if w is None or ms <= 0:
            continue
        work, unit, bound, peak, note = w
        ach = work / (ms / 1000.0) / 1e12
        tr = traffic.get(args.workload, {}).get(name)
        rows[name] = {"kernel": name, "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                      "frac": ach / peak, "traffic": tr["bytes_per_launch"] if tr else None,
                      "peak_note": note, "launches": cnt, "total_ms": ms, "avg_ms": ms / cnt}
    dom_name = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    roof = rows.get(dom_name) or {"kernel": dom_name, "bound": None, "achieved": None, "peak": None,
                                  "unit": None, "frac": None, "traffic": None}
    roof_short = {k: (_sig(v) if isinstance(v, float) else v) for k, v in roof.items()
                  if k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic", "avg_ms")}

    dav = []
    for (E, rn, it, (d0, d1)) in per_step:
        dav.append({"ms": d0.elapsed_time(d1), "energy": E, "residual": rn, "iterations": it,
                    "energy_err_vs_fp64": abs(E - E_ref) if E_ref is not None else None})
    if ttl:
        step_ms = sorted(d["ms"] for d in dav)
        med = step_ms[len(step_ms) // 2]
        ms = {args.precision: _sig(med)}
        err = {args.precision: _sig(max(d["energy_err_vs_fp64"] for d in dav), 2)}
        it = {args.precision: dav[-1]["iterations"]}
        for name, c in ttl["cmp"].items():
            ms[name], err[name], it[name] = _sig(c["ms"]), _sig(c["err"], 2), c["it"]
        # DL: Davidson-Liu with the mode's sigma; DL+JD: Davidson-Liu with the reduced sigma,
        # then Jacobi-Davidson with the FP64-class sigma (details: "solvers")
        ttl_line = {"ref": ttl["ref"], "gap": ttl["gap"], "ms": ms, "err": err, "it": it,
                    "solver": {k: ("DL" if k in ("fp64", "df32", "oz64") else "DL+JD") for k in ms}}
    out = {
        "metric": METRIC, "value": value, "unit": "det/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "tf32": "tf32+f64", "bf16x2": "bf16x2+f64", "df32": "df32",
                  "oz64": "bf16-digits+df32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.workload], "precision": args.precision, "nroots": nroots,
                   "tol": tol, "step": "Davidson to tol + 1-/2-RDM", "l2": "inputs > L2, no flush",
                   "parallelism": f"replicas x{world}"},
        "time_to_1e-8": ttl_line if ttl else None,
        "roofline": roof_short,
        "gpu_launches": launches,
        "clocks": {k: v for k, v in clk.items() if k in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    details = {
        "davidson": dav, "sigma_vectors": {"fp64": n_sig64, "reduced": n_sigm}, "setup_s": t_setup,
        "roofline": roof, "rooflines": rows, "solvers": SOLVERS,
        "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
        "clocks": clk,
    }
    if ttl:
        details.update(details_ref)

    # sigma-only throughput per precision (det/s), outside the timed region
    if args.sigma_rates:
        C = torch.tensor(si.random_vectors(1, prob.na, prob.nb, seed=12), device="cuda")
        S = torch.empty_like(C)
        rates = {}
        for name, m in modes.items():
            fg.forte_set_precision(prob.ctx, m)
            fg.forte_sigma(prob.ctx, C, S, 1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3 if m == fg.FORTE_FP64 else 10
            a.record(stream)
            for _ in range(reps):
                fg.forte_sigma(prob.ctx, C, S, 1)
            b.record(stream)
            torch.cuda.synchronize()
            rates[name] = {"ms": a.elapsed_time(b) / reps, "det_per_s": nd / (a.elapsed_time(b) / reps / 1000.0)}
        details["sigma_rates"] = rates
        fg.forte_set_precision(prob.ctx, mode)

    # end to end through the C ABI: host integrals in, host energies + RDMs out
    if args.e2e_steps > 0:
        h_pin = torch.tensor(h).pin_memory()
        eri_pin = torch.tensor(eri).pin_memory()
        g1_host = torch.empty(n, n, dtype=torch.float64).pin_memory()
        g2_host = torch.empty((n,) * 4, dtype=torch.float64).pin_memory()
        e2e_t, e2e_units = [], 0
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = fg.forte_cas_create(n, na, nb, h_pin.numpy(), eri_pin.numpy())
            fg.forte_set_stream(ctx, stream)
            fg.forte_set_precision(ctx, mode)
            fg.forte_davidson(ctx, nroots, tol, allow_not_converged=True)
            fg.forte_get_roots(ctx, nroots, root)
            fg.forte_rdms(ctx, root[0], g1, g2, n)
            g1_host.copy_(g1, non_blocking=True)
            g2_host.copy_(g2, non_blocking=True)
            torch.cuda.synchronize()
            c = fg.forte_get_counters(ctx)
            fg.forte_destroy(ctx)
            e2e_t.append(time.perf_counter() - t0)
            e2e_units += nd * (c[0] + c[1])
        _, _, e2e_value = combine_ranks(1000.0 * sum(e2e_t), e2e_units, dist, "cuda")
        out["e2e"] = {"value": e2e_value, "unit": "det/s",
                      "h2d_bytes_per_step": 8 * (n * n + n ** 4),
                      "d2h_bytes_per_step": 8 * (nroots + n * n + n ** 4),
                      "s_per_step": _sig(sum(e2e_t) / len(e2e_t))}
        details["e2e_includes"] = ("forte_cas_create from host integrals (strings, tables, CSR, H_II) + "
                                   "Davidson + RDMs + copies of energies and RDMs to host")

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, nrows, dt, thr = oracle_sigma_rate(cfg, seconds=args.ref_seconds)
        out["cpu_baseline"] = {"value": r, "unit": "det/s", "cores": thr, "kind": "oracle",
                               "sample": f"oracle FP64 sigma of {nrows} random rows, {dt:.1f} s"}
    if rank == 0:
        if args.details_out:
            with open(args.details_out, "w") as f:
                json.dump(details, f, indent=1)
        sys.stderr.write("bench details: " + json.dumps(details) + "\n")
        sys.stderr.flush()
        print(json.dumps(out))
    prob.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_kernel_case(args):
    """Small fixed invocation for profilers: build the workload, then run one
    operation twice (the second call is the one to capture)."""
    import torch
    import paper_2405_10197_gb300 as fg
    torch.cuda.set_device(0)
    cfg = WORKLOADS[args.workload]
    n, na, nb = cfg["norb"], cfg["nalpha"], cfg["nbeta"]
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    mode = {"fp64": fg.FORTE_FP64, "tf32": fg.FORTE_TF32, "bf16x2": fg.FORTE_BF16X2, "df32": fg.FORTE_DF32,
            "oz64": fg.FORTE_OZ64}[args.precision]
    prob = fg.CASProblem(n, na, nb, h, eri, precision=mode)
    C = torch.tensor(si.random_vectors(1, prob.na, prob.nb, seed=12), device="cuda")
    out = {"case": args.kernel_case, "workload": args.workload, "precision": args.precision}
    for _ in range(2):
        if args.kernel_case == "sigma":
            S = prob.sigma(C)
            out["max_abs"] = float(S.abs().max())
        else:
            g1, _ = prob.rdms(C[0])
            out["trace_g1"] = float(g1.trace())
    torch.cuda.synchronize()
    prob.close()
    print(json.dumps(out))
    return 0


def run_batch(args):
    """Solves/s of forte_batch_solve on the first `args.batch` instances of the
    batched workload (orbital counts {6,8,10,12}, 1-3 roots, seeds 1000+i), in FP64
    and in the mixed mode, with the autotuner's choices per size class, the
    occupancy of each class launch, the FP64 rate of the tuned per-CTA sigma and an
    oracle check of the n <= 8 instances (dense diagonalisation)."""
    import torch
    import paper_2405_10197_gb300 as fg
    from math import comb
    torch.cuda.set_device(0)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    inst = si.batch_instances()[:args.batch]
    probs = []
    for q in inst:
        h, eri = si.integrals(q["norb"], q["n_l"], q["seed"])
        probs.append(dict(norb=q["norb"], nalpha=q["nalpha"], nbeta=q["nbeta"], nroots=q["nroots"], h=h, eri=eri))
    modes = {"fp64": fg.FORTE_FP64, "tf32": fg.FORTE_TF32, "bf16x2": fg.FORTE_BF16X2, "df32": fg.FORTE_DF32,
             "oz64": fg.FORTE_OZ64}
    mixed = args.precision if args.precision != "fp64" else "bf16x2"
    counts = {n: sum(1 for q in inst if q["norb"] == n) for n in (6, 8, 10, 12)}
    out = {"metric": "batched CASCI solves/s", "unit": "solves/s", "instances": len(probs), "tol": args.tol,
           "orbital_counts": counts, "roots": int(sum(q["nroots"] for q in inst)), "sms": nsm}
    energies = {}
    for name in ("fp64", mixed):
        m = modes[name]
        fg.forte_batch_solve(probs[:8], precision=m, tol=args.tol)  # warm-up (module load, code paths)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E, st = fg.forte_batch_solve(probs, precision=m, tol=args.tol, allow_not_converged=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        energies[name] = E
        tun = []
        for t in fg.forte_batch_tuning():
            n, na, nb = t["norb"], t["nalpha"], t["nbeta"]
            nprob = sum(1 for p in probs if (p["norb"], p["nalpha"], p["nbeta"]) == (n, na, nb))
            NA, NB = comb(n, na), comb(n, nb)
            nk = lambda e: e * (n - e) + e  # noqa: E731
            per_row = lambda e: 1 + e * (n - e) + comb(e, 2) * comb(n - e, 2)  # noqa: E731
            flop = 2.0 * (NA * per_row(na) * NB + NB * per_row(nb) * NA) + 2.0 * NA * NB * nk(na) * nk(nb)
            probed = min(nprob, nsm)
            rate = probed * flop / (t["sigma_ms"] * 1e-3) / 1e12
            entry = dict(t, sigma_ms=_sig(t["sigma_ms"], 4), single_iter_ms=_sig(t["single_iter_ms"], 4),
                         ctas_per_problem_slot=round(nprob / (nsm * t["ctas_per_sm"]), 3))
            if name == "fp64":
                entry["sigma_fp64_tflops"] = _sig(rate, 3)
                entry["frac_of_fp64_pipe_1.25"] = _sig(rate / FP64_PEAK_TFLOPS, 3)
            tun.append(entry)
        big = sum(1 for p in probs if comb(p["norb"], p["nalpha"]) * comb(p["norb"], p["nbeta"]) > 100000)
        out[name] = {"seconds": _sig(dt), "solves_per_s": _sig(len(probs) / dt), "not_converged": int((st != 0).sum()),
                     "not_converged_instances": [dict(index=int(i), norb=probs[i]["norb"], nroots=probs[i]["nroots"],
                                                      status=int(st[i])) for i in np.nonzero(st)[0][:16]],
                     "single_path_above_1e5_det": big, "paths": fg.forte_batch_stats(), "tuning": tun}
    diffs = [float(np.max(np.abs(np.array(a) - np.array(b)))) for a, b in zip(energies["fp64"], energies[mixed])]
    out["max_energy_diff_mixed_vs_fp64"] = max(diffs)
    worst = np.argsort(diffs)[::-1][:5]
    out["largest_diffs"] = [dict(index=int(i), norb=probs[i]["norb"], nroots=probs[i]["nroots"], diff=_sig(diffs[i], 3),
                                 e_fp64=[float(x) for x in energies["fp64"][i]],
                                 e_mixed=[float(x) for x in energies[mixed][i]]) for i in worst[:3]]
    import oracle
    errs = []
    for p, e in zip(probs[:64], energies["fp64"][:64]):
        if p["norb"] <= 8:
            w, _ = oracle.solve_dense(p["norb"], p["nalpha"], p["nbeta"], p["h"], p["eri"], nroots=p["nroots"])
            errs.append(float(np.abs(np.array(e) - w).max()))
    out["oracle_check"] = {"instances": len(errs), "max_abs_err_fp64": max(errs) if errs else None,
                           "sample": "every n <= 8 instance among the first 64 (oracle dense diagonalisation)"}
    out["value"] = out[mixed]["solves_per_s"]
    print(json.dumps(out))
    return 0


def run_sci(args):
    """Determinant-list sigma (selected-CI data path): lists grown from the aufbau
    determinant (it and all its singles and doubles; a third list adds random
    determinants of the sector), one vector, CUDA events around forte_sci_sigma;
    rows sampled against the oracle's matrix elements; the oracle's own list sigma
    timed on a 4,000-determinant head of the first list (same screen: every pair)."""
    import torch
    import paper_2405_10197_gb300 as fg
    import oracle
    torch.cuda.set_device(0)
    cases = [("CAS-size reference list: 24 orbitals, 6a+6b, singles+doubles", 24, 6, 6, 0),
             ("30 orbitals, 10a+10b, singles+doubles", 30, 10, 10, 0),
             ("30 orbitals, 10a+10b, singles+doubles + 150,000 random determinants", 30, 10, 10, 150000)]
    pc = np.vectorize(lambda x: bin(int(x)).count("1"))
    out = {"metric": "determinant-list sigma", "unit": "ms", "cases": []}
    for name, n, na, nb, extra in cases:
        h, eri = si.integrals(n, 2 * n, seed=90 + n)
        words = si.excitation_list(n, na, nb)
        if extra:
            words = np.unique(np.concatenate([words, si.random_determinants(n, na, nb, extra, seed=5)]))
        nd = len(words)
        d = torch.tensor(words.view(np.int64), device="cuda")
        C = torch.tensor(np.random.default_rng(3).normal(size=(1, nd)), device="cuda")
        S = torch.empty_like(C)
        sci = fg.forte_sci_create(n, h, eri)
        try:
            for _ in range(2):
                fg.forte_sci_sigma(sci, d, C, S, 1)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            a.record()
            for _ in range(reps):
                fg.forte_sci_sigma(sci, d, C, S, 1)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
        finally:
            fg.forte_sci_destroy(sci)
        Sh, Ch = S.cpu().numpy()[0], C.cpu().numpy()[0]
        rng = np.random.default_rng(7)
        worst = 0.0
        for i in rng.choice(nd, size=4, replace=False):
            near = np.nonzero(pc(words ^ words[i]) <= 4)[0]
            ref = sum(oracle.hij(n, h, eri, int(words[i]), int(words[j])) * Ch[j] for j in near)
            worst = max(worst, abs(Sh[i] - ref) / max(1.0, abs(ref)))
        out["cases"].append({"workload": name, "n_det": nd, "ms": _sig(ms), "det_per_s": _sig(nd / (ms * 1e-3)),
                             "pair_screens_per_s": _sig(float(nd) * nd / (ms * 1e-3)),
                             "sampled_rows_rel_err_vs_oracle": _sig(worst, 3)})
    # the oracle on a bounded head of the first list
    n, na, nb = 24, 6, 6
    h, eri = si.integrals(n, 2 * n, seed=90 + n)
    words = si.excitation_list(n, na, nb)[:4000]
    C = np.random.default_rng(3).normal(size=(1, len(words)))
    t0 = time.perf_counter()
    oracle.sci_sigma(n, words, h, eri, C)
    dt = time.perf_counter() - t0
    out["cpu_baseline"] = {"kind": "oracle", "cores": oracle.num_threads(), "sample": "oracle.sci_sigma on the first "
                           "4,000 determinants of the 24-orbital list", "pair_screens_per_s": _sig(4000.0 * 4000 / dt),
                           "seconds": _sig(dt)}
    print(json.dumps(out))
    return 0


def run_configs(args):
    """One JSON line per measurement config besides the headline CAS(14,14) step:
    C0 CAS(8,8) FP64 (latency: us per sigma and per iteration), C1 CAS(12,12) 4 roots
    (det/s per 4-vector sigma launch; Davidson to 1e-10 in every precision) and the
    12-site Hubbard ring, C3 CAS(12,12) state-averaged energy gradient (forward +
    backward, central differences along random integral directions), C4 batched
    solves (solves/s, FP64 and BF16x2) and the oracle's own timings on the host."""
    import torch
    import paper_2405_10197_gb300 as fg
    torch.cuda.set_device(0)
    modes = {"fp64": fg.FORTE_FP64, "df32": fg.FORTE_DF32, "oz64": fg.FORTE_OZ64, "tf32": fg.FORTE_TF32,
             "bf16x2": fg.FORTE_BF16X2}

    def ev_time(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def sigma_rates(prob, nvec, reps):
        C = torch.tensor(si.random_vectors(nvec, prob.na, prob.nb, seed=7), device="cuda")
        S = torch.empty_like(C)
        out = {}
        for name, m in modes.items():
            fg.forte_set_precision(prob.ctx, m)
            ms = ev_time(lambda: fg.forte_sigma(prob.ctx, C, S, nvec), reps if m != fg.FORTE_FP64 else max(2, reps // 4))
            out[name] = {"ms_per_launch": ms, "det_per_s": prob.ndet * nvec / (ms / 1000.0)}
        return out

    def solves(prob, nroots, tol, names):
        out = {}
        for name in names:
            fg.forte_set_precision(prob.ctx, modes[name])
            prob.davidson(nroots=nroots, tol=tol)  # warm-up (tables, scratch)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            E, C, rn, it = prob.davidson(nroots=nroots, tol=tol)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out[name] = {"ms": 1000 * dt, "iterations": int(it), "max_residual": float(np.max(rn)),
                         "energies": [float(e) for e in E]}
        ref = out["fp64"]["energies"]
        for name in names:
            out[name]["max_energy_err_vs_fp64"] = float(np.max(np.abs(np.array(out[name]["energies"]) - ref)))
        return out

    lines = []
    # C0
    cfg = si.CAS88
    h, eri = si.integrals(8, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(8, 4, 4, h, eri)
    sr = sigma_rates(prob, 1, 50)
    sv = solves(prob, 1, 1e-10, ["fp64", "df32", "oz64", "bf16x2"])
    c0 = {"config": "C0 CAS(8,8) seed 0, 4,900 determinants", "sigma": sr, "davidson_1e-10": sv,
          "us_per_sigma_fp64": 1000 * sr["fp64"]["ms_per_launch"],
          "us_per_iteration_fp64": 1000 * sv["fp64"]["ms"] / max(1, sv["fp64"]["iterations"])}
    prob.close()
    lines.append(c0)
    # C1
    cfg = si.CAS1212
    h, eri = si.integrals(12, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(12, 6, 6, h, eri)
    c1 = {"config": "C1 CAS(12,12) seed 1, 853,776 determinants, 4 roots",
          "sigma_nvec4": sigma_rates(prob, 4, 10),
          "davidson_4roots_1e-10": solves(prob, 4, 1e-10, ["fp64", "df32", "oz64", "tf32", "bf16x2"])}
    prob.close()
    h, eri = si.hubbard_ring(12, 1.0, 4.0)
    prob = fg.CASProblem(12, 6, 6, h, eri)
    c1["hubbard12_U4_davidson_1e-10"] = solves(prob, 1, 1e-10, ["fp64", "df32", "oz64", "bf16x2"])
    prob.close()
    lines.append(c1)
    # C3: state-averaged gradient, forward + backward, central differences
    cfg = si.CAS1212_SA
    h, eri = si.integrals(12, cfg["n_l"], cfg["seed"])
    w = [1.0 / 3] * 3
    c3 = {"config": "C3 CAS(12,12) seed 3, state average of 3 roots (w = 1/3)"}
    for name in ("fp64", "bf16x2"):
        ht = torch.tensor(h, requires_grad=True)
        et = torch.tensor(eri, requires_grad=True)
        fg.sa_energy(ht, et, 12, 6, 6, w, precision=modes[name], tol=1e-9)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E = fg.sa_energy(ht, et, 12, 6, 6, w, precision=modes[name], tol=1e-9)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        E.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        rng = np.random.default_rng(11)
        dev = []
        for _ in range(args.fd_dirs):
            dh = rng.normal(size=(12, 12)); dh = 0.5 * (dh + dh.T)
            lin = float((ht.grad.numpy() * dh).sum())
            eps = 1e-4
            ep = fg.sa_energy(torch.tensor(h + eps * dh), et.detach(), 12, 6, 6, w, precision=modes[name], tol=1e-10)
            em = fg.sa_energy(torch.tensor(h - eps * dh), et.detach(), 12, 6, 6, w, precision=modes[name], tol=1e-10)
            dev.append(abs((float(ep) - float(em)) / (2 * eps) - lin))
        c3[name] = {"forward_ms": 1000 * (t1 - t0), "backward_ms": 1000 * (t2 - t1), "E_SA": float(E),
                    "fd_directions": args.fd_dirs, "max_fd_deviation_dh": float(max(dev)) if dev else None}
    lines.append(c3)
    # C4: batched solves
    inst = si.batch_instances()[:args.configs_batch]
    probs = []
    for q in inst:
        hq, eq = si.integrals(q["norb"], q["n_l"], q["seed"])
        probs.append(dict(norb=q["norb"], nalpha=q["nalpha"], nbeta=q["nbeta"], nroots=q["nroots"], h=hq, eri=eq))
    fg.forte_batch_solve(probs[:8], precision=fg.FORTE_BF16X2, tol=1e-7)
    c4 = {"config": f"C4 batched: first {len(probs)} of the 512 seeded instances (orbitals "
                    f"{sorted(set(q['norb'] for q in inst))}, 1-3 roots)", "roots": int(sum(q["nroots"] for q in inst))}
    res, sts = {}, {}
    for name in ("fp64", "bf16x2"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E, st = fg.forte_batch_solve(probs, precision=modes[name], tol=1e-7, allow_not_converged=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[name], sts[name] = E, st
        c4[name] = {"seconds": dt, "solves_per_s": len(probs) / dt, "not_converged": int((st != 0).sum()),
                    "not_converged_instances": [int(i) for i in np.nonzero(st != 0)[0]]}
    diffs = [float(np.max(np.abs(np.array(a) - np.array(b)))) for a, b in zip(res["fp64"], res["bf16x2"])]
    both = [d for d, a, b in zip(diffs, sts["fp64"], sts["bf16x2"]) if a == 0 and b == 0]
    c4["max_energy_diff_bf16x2_vs_fp64"] = max(diffs)
    c4["max_energy_diff_where_both_converged"] = max(both) if both else None
    c4["instance_of_max_diff"] = int(np.argmax(diffs))
    lines.append(c4)
    # oracle timings on the host (bounded samples)
    if not args.no_cpu_baseline:
        import oracle
        orc = {"config": "oracle (plain C Slater-Condon, FP64) on this host", "threads": oracle.num_threads()}
        for key, c in (("C0", si.CAS88), ("C1", si.CAS1212)):
            r, nrows, dt, thr = oracle_sigma_rate(c, seconds=5.0)
            orc[key + "_sigma_det_per_s"] = r
        cfg = si.CAS88
        h, eri = si.integrals(8, cfg["n_l"], cfg["seed"])
        t0 = time.perf_counter()
        _, _, _, it_or = oracle.davidson(8, 4, 4, h, eri, nroots=1, tol=1e-10)
        orc["C0_davidson_1e-10_s"] = time.perf_counter() - t0
        # the same textbook Davidson-Liu (reading 6) on the same input: iteration counts
        orc["C0_davidson_1e-10_iterations"] = {"oracle": int(it_or),
                                               "gpu_fp64": int(c0["davidson_1e-10"]["fp64"]["iterations"])}
        lines.append(orc)
    for ln in lines:
        print(json.dumps(ln))
    return 0


def run_extensions(args):
    """One JSON line per extension of the path: X1 the spin-free 3-RDM (FP64 Gram
    work 2 n^6 N_det), X2 an occupation-restricted CAS(14,14) (RAS: at most two
    holes in the lowest four orbitals and two particles in the highest four) and
    X3 the even-S sector of CAS(14,14), each against the unrestricted solve."""
    import torch
    import paper_2405_10197_gb300 as fg
    torch.cuda.set_device(0)
    lines = []

    def ev_ms(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    # X1: 3-RDM of the ground state
    x1 = {"config": "X1 spin-free 3-RDM (FP64, every precision mode)", "cases": []}
    for n, cfg in ((8, si.CAS88), (10, None)):
        h, eri = si.integrals(n, 2 * n, cfg["seed"] if cfg else 10)
        prob = fg.CASProblem(n, n // 2, n // 2, h, eri)
        E, C, rn, it = prob.davidson(nroots=1, tol=1e-8)
        g3 = torch.empty((n,) * 6, dtype=torch.float64, device="cuda")
        ms = ev_ms(lambda: fg.forte_rdm3(prob.ctx, C[0], g3, n), 3)
        flop = 2.0 * n ** 6 * prob.ndet
        x1["cases"].append({"workload": f"CAS({n},{n})", "n_det": prob.ndet, "ms": ms,
                            "gram_fp64_tflops": flop / (ms * 1e-3) / 1e12,
                            "frac_of_nominal_fp64_1.25": flop / (ms * 1e-3) / 1.25e12})
        prob.close()
    lines.append(x1)

    cfg = si.CAS1414
    h, eri = si.integrals(14, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(14, 7, 7, h, eri, precision=fg.FORTE_BF16X2)

    def solve(tag):
        prob.davidson(nroots=1, tol=1e-8)  # warm-up (scratch, tables)
        fg.forte_profile_enable(prob.ctx, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E, C, rn, it = prob.davidson(nroots=1, tol=1e-8)
        torch.cuda.synchronize()
        dt = 1000 * (time.perf_counter() - t0)
        out = {"ms": dt, "iterations": int(it), "energy": float(E[0]), "residual": float(rn[0])}
        for k in ("gas_mask", "spin_proj"):
            nl, kms = fg.forte_profile_query(prob.ctx, k)
            if nl:
                out[k] = {"launches": nl, "ms": kms, "share": kms / dt}
        fg.forte_profile_enable(prob.ctx, 0)
        return out

    C1 = torch.tensor(si.random_vectors(1, prob.na, prob.nb, seed=5), device="cuda")
    S1 = torch.empty_like(C1)
    sig_modes = (("fp64", fg.FORTE_FP64, 2), ("oz64", fg.FORTE_OZ64, 5), ("bf16x2", fg.FORTE_BF16X2, 5))
    sig = {}
    for name, m, reps in sig_modes:
        fg.forte_set_precision(prob.ctx, m)
        sig[name] = {"unrestricted": _sig(ev_ms(lambda: fg.forte_sigma(prob.ctx, C1, S1, 1), reps))}
    fg.forte_set_precision(prob.ctx, fg.FORTE_BF16X2)
    full = solve("full")
    # X2: RAS(2h, 2p); both exact routes of the restricted sigma, then the timed choice
    nd = prob.set_gas((4, 6, 4), (6, 0, 0), (8, 12, 2))
    for name, m, reps in sig_modes:
        fg.forte_set_precision(prob.ctx, m)
        for route, key in ((0, "grid_route"), (1, "kept_route")):
            fg.forte_set_gas_route(prob.ctx, route)
            sig[name][key] = _sig(ev_ms(lambda: fg.forte_sigma(prob.ctx, C1, S1, 1), reps))
        sig[name]["kept_over_unrestricted"] = _sig(sig[name]["kept_route"] / sig[name]["unrestricted"], 3)
    fg.forte_set_gas_route(prob.ctx, -1)
    fg.forte_set_precision(prob.ctx, fg.FORTE_BF16X2)
    gas = solve("gas")
    r64, r32, rms = fg.forte_get_gas_route(prob.ctx)
    names = {-1: "not timed", 0: "full grid", 1: "kept determinants"}
    gas["routes"] = {"fp64_vectors": names[r64], "fp32_vectors": names[r32],
                     "timed_ms": {"fp64_grid": _sig(rms[0]), "fp64_kept": _sig(rms[1]), "fp32_grid": _sig(rms[2]),
                                  "fp32_kept": _sig(rms[3])}}
    lines.append({"config": "X2 CAS(14,14) seed 2 under RAS(2 holes in orbitals 0-3, 2 particles in 10-13), "
                            "BF16x2 Davidson refined to 1e-8", "kept_determinants": nd, "n_det": prob.ndet,
                  "sigma_ms": sig, "davidson": {"unrestricted": full, "restricted": gas}})
    prob.set_gas((), (), ())
    # X3: even-S sector
    prob.set_spin_parity(1)
    even = solve("even")
    prob.set_spin_parity(0)
    lines.append({"config": "X3 CAS(14,14) seed 2, even-S sector vs unrestricted, BF16x2 Davidson refined to 1e-8",
                  "davidson": {"unrestricted": full, "even_S": even}})
    prob.close()
    # X4: adaptive CI at CAS(12,12) seed 1, sigma = 1e-3, in the even-S sector and without
    cfg = si.CAS1212
    h, eri = si.integrals(12, cfg["n_l"], cfg["seed"])
    x4 = {"config": "X4 adaptive CI, CAS(12,12) seed 1, sigma 1e-3, gamma 1, FP64-class screening", "runs": []}
    for parity in (1, 0):
        prob = fg.CASProblem(12, 6, 6, h, eri, precision=fg.FORTE_BF16X2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            e, ec, C, nm, np_, cyc = prob.aci(1e-3, 1.0, 30, 1e-8, parity)
            st = "ok"
        except fg.ForteError as err:
            e = ec = float("nan")
            nm = np_ = cyc = -1
            st = str(err)[:120]
        torch.cuda.synchronize()
        x4["runs"].append({"parity": parity, "seconds": _sig(time.perf_counter() - t0), "E_M": e, "E_corrected": ec,
                           "n_M": nm, "n_P": np_, "cycles": cyc, "status": st})
        prob.close()
    lines.append(x4)
    for ln in lines:
        print(json.dumps(ln))
    return 0


def fg_nnz(prob):
    """Stored entries of the alpha and beta same-spin string Hamiltonians: every
    string within two replacements of a row string (itself, singles, doubles)."""
    from math import comb
    n = prob.norb

    def per_row(ne):
        return 1 + ne * (n - ne) + comb(ne, 2) * comb(n - ne, 2)
    return prob.na * per_row(prob.nalpha), prob.nb * per_row(prob.nbeta)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cas1414")
    ap.add_argument("--precision", choices=["fp64", "tf32", "bf16x2", "df32", "oz64"], default="bf16x2")
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--ref-tol", type=float, default=1e-10,
                    help="residual of the FP64 reference solve behind the time-to-1e-8 comparison")
    ap.add_argument("--ref-max-iter", type=int, default=600)
    ap.add_argument("--details-out", default=None, help="also write the per-kernel details to this JSON file")
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false")
    ap.add_argument("--no-sigma-rates", dest="sigma_rates", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="time forte_batch_solve on the first N instances of the batched workload instead")
    ap.add_argument("--configs", action="store_true",
                    help="measure the other configurations (C0, C1, C3, C4, oracle) instead of the headline step")
    ap.add_argument("--configs-batch", type=int, default=128, help="instances of the batched workload for --configs")
    ap.add_argument("--fd-dirs", type=int, default=4, help="central-difference directions for the C3 gradient check")
    ap.add_argument("--extensions", action="store_true",
                    help="measure the 3-RDM, the occupation restriction and the spin-parity sector")
    ap.add_argument("--sci", action="store_true",
                    help="measure the determinant-list (selected-CI) sigma on reference-grown lists")
    ap.add_argument("--kernel-case", choices=["sigma", "rdm"], default=None,
                    help="profiling helper: run one sigma (or RDM) call twice on the workload and exit")
    args = ap.parse_args(argv)
    if args.steps < 1:
        ap.error("--steps must be >= 1")
    return args


def main():
    args = parse_args()
    if args.kernel_case:
        return run_kernel_case(args)
    if args.batch > 0:
        return run_batch(args)
    if args.configs:
        return run_configs(args)
    if args.extensions:
        return run_extensions(args)
    if args.sci:
        return run_sci(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

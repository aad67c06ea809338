// Batched solve of many independent active-space problems (step a11): each
// problem is an ActiveSpaceMethod instance in the paper's terms (Sec. III,
// ActiveSpaceSolver), so the batch is embarrassingly parallel.
//
// Scheduling: problems are taken largest first (by determinant count) from a
// shared counter by `nworkers` host threads; every worker owns one non-blocking
// CUDA stream, creates the problem's context, runs forte_davidson on its stream
// and frees the context, so device memory stays bounded by the workers' live
// problems while the GPU overlaps the kernels of different problems.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "forte_internal.h"

using namespace forte;

extern "C" int forte_batch_solve(int nprob, const int *norb, const int *nalpha, const int *nbeta,
                                 const int *nroots, const double *const *h, const double *const *eri,
                                 int precision, double tol, int nworkers, double *E_out, int *status_out) {
  clear_error();
  if (nprob < 0 || (nprob > 0 && (!norb || !nalpha || !nbeta || !nroots || !h || !eri || !E_out))) {
    set_error("forte_batch_solve: bad arguments");
    return FORTE_ERR_ARG;
  }
  if (precision != FORTE_FP64 && precision != FORTE_TF32 && precision != FORTE_BF16X2 && precision != FORTE_DF32 &&
      precision != FORTE_OZ64) {
    set_error("forte_batch_solve: unknown precision %d", precision);
    return FORTE_ERR_ARG;
  }
  if (nprob == 0) return FORTE_OK;
  std::vector<long long> offset(nprob + 1, 0), size(nprob, 0);
  for (int i = 0; i < nprob; ++i) {
    if (norb[i] < 1 || norb[i] > 16 || nroots[i] < 1 || nalpha[i] < 0 || nbeta[i] < 0 || nalpha[i] > norb[i] ||
        nbeta[i] > norb[i]) {
      set_error("forte_batch_solve: bad sizes for problem %d", i);
      return FORTE_ERR_ARG;
    }
    offset[i + 1] = offset[i] + nroots[i];
    long long a = 1, b = 1;
    for (int k = 1; k <= nalpha[i]; ++k) a = a * (norb[i] - nalpha[i] + k) / k;
    for (int k = 1; k <= nbeta[i]; ++k) b = b * (norb[i] - nbeta[i] + k) / k;
    size[i] = a * b;
  }
  std::vector<int> order(nprob);
  for (int i = 0; i < nprob; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return size[x] > size[y]; });
  int dev = 0;
  FORTE_CUDA_TRY(cudaGetDevice(&dev));
  const int nw = std::max(1, std::min(nworkers > 0 ? nworkers : 8, nprob));
  std::atomic<int> next(0);
  std::mutex mu;
  int worst = FORTE_OK;
  std::string first_msg;
  auto worker = [&]() {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      std::lock_guard<std::mutex> lock(mu);
      worst = std::max(worst, (int)FORTE_ERR_CUDA);
      if (first_msg.empty()) first_msg = "stream creation failed";
      return;
    }
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= nprob) break;
      const int i = order[k];
      int rc = FORTE_OK;
      forte_ctx *ctx = forte_cas_create(norb[i], nalpha[i], nbeta[i], h[i], eri[i]);
      if (!ctx) rc = FORTE_ERR_ARG;
      if (!rc) rc = forte_set_stream(ctx, st);
      if (!rc) rc = forte_set_precision(ctx, precision);
      if (!rc) rc = forte_davidson(ctx, nroots[i], tol);
      if (rc == FORTE_OK || rc == FORTE_ERR_NOT_CONVERGED) {
        int rc2 = forte_get_roots(ctx, E_out + offset[i], nullptr, nullptr, nullptr);
        if (rc2) rc = rc2;
      }
      if (status_out) status_out[i] = rc;
      if (rc) {
        std::lock_guard<std::mutex> lock(mu);
        if (rc > worst) worst = rc;
        if (first_msg.empty()) first_msg = "problem " + std::to_string(i) + ": " + forte_last_error();
      }
      forte_destroy(ctx);
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> th;
  for (int w = 0; w < nw; ++w) th.emplace_back(worker);
  for (auto &t : th) t.join();
  if (worst) set_error("%s", first_msg.c_str());
  return worst;
}

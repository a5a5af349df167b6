// adjoint.cu - checkpointed rollout and reverse sweep (lbm_record / lbm_backward).
//
// Forward: S_0 = f^eq(rho0, U0, T0) from the fields kept by lbm_init, then
// nsteps stream-collide steps; every k-th state S_0, S_k, S_2k, ... is written
// straight into its own checkpoint buffer by the step that produces it (no
// extra copies).  Reverse: for each segment [c k, min((c+1) k, N)) from the
// last, the states S_ck+1 .. are recomputed from the checkpoint with the same
// kernel (bitwise identical to the forward), then the adjoint steps run from the
// segment's last state down to its first.  Memory: ceil(N/k) + k - 1 states plus
// two adjoint buffers, the uniform sqrt(N) schedule when k ~ sqrt(N).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "../../include/lbm.h"
#include "adjoint.h"
#include "common.h"

using namespace lbm;

namespace {

#define ADJ_CUDA(call)                                              \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ctx_cuda_fail(e_, #call);         \
  } while (0)

size_t state_bytes(const CtxView& v) {
  return (size_t)v.Q * (size_t)v.g.ncell * (size_t)v.ops->elem_bytes;
}

}  // namespace

extern "C" {

int lbm_record(lbm_ctx* ctx, int64_t nsteps, int64_t ckpt_every) {
  if (!ctx) return ctx_fail(LBM_EINVAL, "ctx is NULL");
  CtxView v = ctx_view(ctx);
  if (!v.inited || !v.fields->p) return ctx_fail(LBM_ESTATE, "lbm_record needs lbm_init first");
  if (nsteps < 1 || ckpt_every < 1) return ctx_fail(LBM_EINVAL, "nsteps and ckpt_every must be >= 1");
  Record& r = *v.rec;
  r.valid = false;
  const int64_t k = ckpt_every < nsteps ? ckpt_every : nsteps;
  const int64_t nck = (nsteps + k - 1) / k;
  const size_t sb = state_bytes(v);
  // keep buffers already allocated; grow the lists as needed
  while ((int64_t)r.ckpt.size() < nck) r.ckpt.emplace_back(new DevBuf());
  while ((int64_t)r.ckpt.size() > nck) r.ckpt.pop_back();
  for (auto& b : r.ckpt) {
    int rc = b->ensure(sb, v.stream);
    if (rc) return rc;
  }
  const double* f = static_cast<const double*>(v.fields->p);
  const size_t n = (size_t)v.g.ncell;
  cudaError_t e = v.ops->init(v.model, f, f + n, f + (size_t)(v.D + 1) * n, r.ckpt[0]->p, v.g, v.stream);
  if (e != cudaSuccess) return ctx_cuda_fail(e, "init launch");
  *v.launches += 1;
  void* cur = r.ckpt[0]->p;
  int pp = 0;  // next ping-pong buffer to write
  for (int64_t s = 0; s < nsteps; ++s) {
    void* dst;
    const int64_t nxt = s + 1;
    if (nxt < nsteps && nxt % k == 0) {
      dst = r.ckpt[nxt / k]->p;
    } else {
      if (v.state[pp]->p == cur) pp ^= 1;
      dst = v.state[pp]->p;
      pp ^= 1;
    }
    e = v.ops->step(v.model, cur, dst, v.g, v.omega, v.variant, v.status, v.stream);
    if (e != cudaSuccess) return ctx_cuda_fail(e, "stream_collide launch");
    *v.launches += 1;
    cur = dst;
  }
  *v.cur = (v.state[0]->p == cur) ? 0 : 1;
  *v.steps = nsteps;
  r.final_buf = *v.cur;
  r.nsteps = nsteps;
  r.k = k;
  r.valid = true;
  return LBM_OK;
}

int lbm_release_record(lbm_ctx* ctx) {
  if (!ctx) return ctx_fail(LBM_EINVAL, "ctx is NULL");
  CtxView v = ctx_view(ctx);
  cudaStreamSynchronize(v.stream);
  Record& r = *v.rec;
  r.valid = false;
  r.ckpt.clear();
  r.seg.clear();
  r.nu[0].release();
  r.nu[1].release();
  r.dldrho.release();
  r.omega_acc.release();
  r.omega_out.release();
  r.grads.release();
  return LBM_OK;
}

int lbm_backward(lbm_ctx* ctx, const double* dL_drhoN, double* dL_drho0, double* dL_dU0,
                 double* dL_dT0, double* dL_domega, int where) {
  if (!ctx) return ctx_fail(LBM_EINVAL, "ctx is NULL");
  if (!dL_drhoN) return ctx_fail(LBM_EINVAL, "dL_drhoN is NULL");
  if (where != LBM_HOST && where != LBM_DEVICE) return ctx_fail(LBM_EINVAL, "bad where");
  CtxView v = ctx_view(ctx);
  Record& r = *v.rec;
  if (!r.valid) return ctx_fail(LBM_ESTATE, "lbm_backward needs lbm_record first");
  const size_t n = (size_t)v.g.ncell;
  const size_t sb = state_bytes(v);
  const size_t nb = (size_t)v.Q * n * (size_t)v.ops->adj_elem_bytes;
  const int64_t k = r.k, N = r.nsteps;
  int rc;
  while ((int64_t)r.seg.size() < k - 1) r.seg.emplace_back(new DevBuf());
  for (int64_t j = 0; j < k - 1; ++j)
    if ((rc = r.seg[j]->ensure(sb, v.stream))) return rc;
  const long long nblk = cell_blocks(v.g);
  if ((rc = r.nu[0].ensure(nb, v.stream)) || (rc = r.nu[1].ensure(nb, v.stream)) ||
      (rc = r.dldrho.ensure(n * sizeof(double), v.stream)) ||
      (rc = r.omega_acc.ensure((size_t)nblk * sizeof(double), v.stream)) ||
      (rc = r.omega_out.ensure(sizeof(double), v.stream)))
    return rc;
  ADJ_CUDA(cudaMemcpyAsync(r.dldrho.p, dL_drhoN, n * sizeof(double),
                           where == LBM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                           v.stream));
  ADJ_CUDA(cudaMemsetAsync(r.omega_acc.p, 0, (size_t)nblk * sizeof(double), v.stream));

  // reverse sweep
  int nu_cur = 0;           // buffer holding nu_{n+1} (undefined before the first step)
  bool first = true;
  const int64_t nseg = (N + k - 1) / k;
  std::vector<void*> states((size_t)k);
  for (int64_t c = nseg - 1; c >= 0; --c) {
    const int64_t s0 = c * k;
    const int64_t s1 = (s0 + k < N) ? s0 + k : N;   // states S_s0 .. S_{s1-1}
    states[0] = r.ckpt[c]->p;
    for (int64_t j = 1; j < s1 - s0; ++j) {
      states[j] = r.seg[j - 1]->p;
      cudaError_t e = v.ops->step(v.model, states[j - 1], states[j], v.g, v.omega, v.variant,
                                   v.status, v.stream);
      if (e != cudaSuccess) return ctx_cuda_fail(e, "replay launch");
      *v.launches += 1;
    }
    for (int64_t s = s1 - 1; s >= s0; --s) {
      void* out = r.nu[nu_cur ^ 1].p;
      cudaError_t e = v.ops->adjoint_step(v.model, states[s - s0], first ? nullptr : r.nu[nu_cur].p,
                                          first ? static_cast<const double*>(r.dldrho.p) : nullptr,
                                          out, static_cast<double*>(r.omega_acc.p), v.g, v.omega,
                                          v.stream);
      if (e != cudaSuccess) return ctx_cuda_fail(e, "adjoint launch");
      *v.launches += 1;
      nu_cur ^= 1;
      first = false;
    }
  }
  // gradients with respect to the initial fields
  double *gr = dL_drho0, *gu = dL_dU0, *gt = dL_dT0;
  if (where == LBM_HOST && (dL_drho0 || dL_dU0 || dL_dT0)) {
    if ((rc = r.grads.ensure((size_t)(v.D + 2) * n * sizeof(double), v.stream))) return rc;
    double* b = static_cast<double*>(r.grads.p);
    gr = dL_drho0 ? b : nullptr;
    gu = dL_dU0 ? b + n : nullptr;
    gt = dL_dT0 ? b + (size_t)(v.D + 1) * n : nullptr;
  }
  if (gr || gu || gt) {
    cudaError_t e = v.ops->grad_init(v.model, r.nu[nu_cur].p, static_cast<const double*>(v.fields->p),
                                     gr, gu, gt, v.g, v.stream);
    if (e != cudaSuccess) return ctx_cuda_fail(e, "grad_init launch");
    *v.launches += 1;
  }
  cudaError_t e = launch_sum_reduce(static_cast<const double*>(r.omega_acc.p), nblk,
                                    static_cast<double*>(r.omega_out.p), v.stream);
  if (e != cudaSuccess) return ctx_cuda_fail(e, "omega reduce launch");
  *v.launches += 1;
  if (where == LBM_HOST) {
    if (dL_drho0) ADJ_CUDA(cudaMemcpyAsync(dL_drho0, gr, n * sizeof(double), cudaMemcpyDeviceToHost, v.stream));
    if (dL_dU0) ADJ_CUDA(cudaMemcpyAsync(dL_dU0, gu, (size_t)v.D * n * sizeof(double), cudaMemcpyDeviceToHost, v.stream));
    if (dL_dT0) ADJ_CUDA(cudaMemcpyAsync(dL_dT0, gt, n * sizeof(double), cudaMemcpyDeviceToHost, v.stream));
  }
  if (dL_domega)
    ADJ_CUDA(cudaMemcpyAsync(dL_domega, r.omega_out.p, sizeof(double), cudaMemcpyDeviceToHost, v.stream));
  if (where == LBM_HOST || dL_domega) ADJ_CUDA(cudaStreamSynchronize(v.stream));
  return LBM_OK;
}

}  // extern "C"

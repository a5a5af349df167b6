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
#include <vector>

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

// State of one reverse sweep (shared by both schedules).
struct Sweep {
  CtxView v;
  Record* r;
  int nu_cur = 0;
  bool first = true;
};

int adjoint_at(Sweep& w, const void* state_n) {
  Record& r = *w.r;
  cudaError_t e = w.v.ops->adjoint_step(
      w.v.model, state_n, w.first ? nullptr : r.nu[w.nu_cur].p,
      w.first ? static_cast<const double*>(r.dldrho.p) : nullptr, r.nu[w.nu_cur ^ 1].p,
      static_cast<double*>(r.omega_acc.p), w.v.g, w.v.omega, w.v.stream);
  if (e != cudaSuccess) return ctx_cuda_fail(e, "adjoint launch");
  *w.v.launches += 1;
  w.nu_cur ^= 1;
  w.first = false;
  return LBM_OK;
}

// k >= 1 steps from src (never a work buffer), the last one written to dst.
// Intermediate states alternate between two buffers chosen so that no step reads
// the buffer it writes: counting back from the last step, odd distances use `a`,
// even distances `b`; when dst is a work buffer, `a` is the other work buffer and
// `b` is dst itself (overwritten again by the final step).
int advance(Sweep& w, const void* src, int64_t k, void* dst, void* work0, void* work1) {
  void* a = (dst == work0) ? work1 : work0;
  void* b = (dst == work0) ? work0 : work1;
  const void* cur = src;
  for (int64_t j = 0; j < k; ++j) {
    void* out = (j == k - 1) ? dst : (((k - 1 - j) & 1) ? a : b);
    cudaError_t e = w.v.ops->step(w.v.model, cur, out, w.v.g, w.v.omega, w.v.variant, w.v.status,
                                  nullptr, w.v.stream);
    if (e != cudaSuccess) return ctx_cuda_fail(e, "recompute launch");
    *w.v.launches += 1;
    cur = out;
  }
  return LBM_OK;
}

// Optimal split points for reversing l <= N steps with f <= F free state slots,
// minimising the forward steps recomputed (binomial checkpointing, Griewank 1992;
// this is the plain dynamic programme over its recursion):
//   cost(1, f) = 0,  cost(l, 0) = l (l - 1) / 2   (each state recomputed from the start),
//   cost(l, f) = min over 1 <= m < l of  m + cost(l - m, f - 1) + cost(m, f)
// (advance m steps and store that state, reverse the last l - m steps with one slot
// fewer, then the first m with the same slots).  O(N^2 F) host work; callers fall
// back to bisection beyond a size limit.
void optimal_splits(int64_t N, int64_t F, std::vector<int32_t>* split) {
  const int64_t W = F + 1;
  std::vector<int64_t> cost((size_t)(N + 1) * W, 0);
  split->assign((size_t)(N + 1) * W, 0);
  for (int64_t l = 2; l <= N; ++l) {
    cost[(size_t)(l * W)] = l * (l - 1) / 2;
    for (int64_t f = 1; f <= F; ++f) {
      int64_t best = -1, arg = 1;
      for (int64_t m = 1; m < l; ++m) {
        const int64_t c = m + cost[(size_t)((l - m) * W + f - 1)] + cost[(size_t)(m * W + f)];
        if (best < 0 || c < best) {
          best = c;
          arg = m;
        }
      }
      cost[(size_t)(l * W + f)] = best;
      (*split)[(size_t)(l * W + f)] = (int32_t)arg;
    }
  }
}

// Adjoint steps hi-1 .. lo, with S_lo in s_lo and `used` stored states in use.
// While stored states remain, the range is split at the optimal point (bisection
// if the split table was not built) and the state there is stored; below that,
// each state is recomputed from S_lo.  Work buffers: the context's two population
// buffers.
int reverse_bounded(Sweep& w, int64_t lo, int64_t hi, const void* s_lo, int64_t used) {
  Record& r = *w.r;
  void* w0 = w.v.state[0]->p;
  void* w1 = w.v.state[1]->p;
  const int64_t len = hi - lo;
  if (len == 1) return adjoint_at(w, s_lo);
  int rc;
  if (used < r.max_states) {
    if ((int64_t)r.ckpt.size() <= used) r.ckpt.emplace_back(new DevBuf());
    if ((rc = r.ckpt[used]->ensure((size_t)w.v.Q * (size_t)w.v.g.ncell * (size_t)w.v.ops->elem_bytes,
                                   w.v.stream)))
      return rc;
    const int64_t F = r.max_states - 1, f = r.max_states - used;
    const int64_t mid =
        r.split.empty() ? lo + len / 2 : lo + r.split[(size_t)(len * (F + 1) + f)];
    void* s_mid = r.ckpt[used]->p;
    if ((rc = advance(w, s_lo, mid - lo, s_mid, w0, w1))) return rc;
    if ((rc = reverse_bounded(w, mid, hi, s_mid, used + 1))) return rc;
    return reverse_bounded(w, lo, mid, s_lo, used);
  }
  for (int64_t s = hi - 1; s > lo; --s) {
    if ((rc = advance(w, s_lo, s - lo, w0, w0, w1))) return rc;
    if ((rc = adjoint_at(w, w0))) return rc;
  }
  return adjoint_at(w, s_lo);
}

}  // namespace

extern "C" {

int lbm_record(lbm_ctx* ctx, int64_t nsteps, int64_t ckpt_every) {
  if (!ctx) return ctx_fail(LBM_EINVAL, "ctx is NULL");
  CtxView v = ctx_view(ctx);
  if (!v.inited || !v.fields->p) return ctx_fail(LBM_ESTATE, "lbm_record needs lbm_init first");
  if (v.fixed_ends) return ctx_fail(LBM_EINVAL, "the adjoint does not cover fixed end planes");
  if (v.slab) return ctx_fail(LBM_EINVAL, "the adjoint does not cover slab halo exchanges");
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
  // the last segment's states are computed here anyway: keep them for the reverse sweep
  const int64_t s0_last = ((nsteps - 1) / k) * k;
  while ((int64_t)r.seg.size() < k - 1) r.seg.emplace_back(new DevBuf());
  for (int64_t j = 0; j < nsteps - 1 - s0_last; ++j) {
    int rc = r.seg[j]->ensure(sb, v.stream);
    if (rc) return rc;
  }
  const double* f = static_cast<const double*>(v.fields->p);
  const size_t n = (size_t)v.g.ncell;
  cudaError_t e = v.ops->init(v.model, f, f + n, f + (size_t)(v.D + 1) * n, r.ckpt[0]->p, v.g, 0,
                                 v.g.ncell, v.stream);
  if (e != cudaSuccess) return ctx_cuda_fail(e, "init launch");
  *v.launches += 1;
  void* cur = r.ckpt[0]->p;
  int pp = 0;  // next ping-pong buffer to write
  for (int64_t s = 0; s < nsteps; ++s) {
    void* dst;
    const int64_t nxt = s + 1;
    if (nxt < nsteps && nxt % k == 0) {
      dst = r.ckpt[nxt / k]->p;
    } else if (nxt < nsteps && nxt > s0_last) {
      dst = r.seg[nxt - s0_last - 1]->p;
    } else {
      if (v.state[pp]->p == cur) pp ^= 1;
      dst = v.state[pp]->p;
      pp ^= 1;
    }
    e = v.ops->step(v.model, cur, dst, v.g, v.omega, v.variant, v.status, nullptr, v.stream);
    if (e != cudaSuccess) return ctx_cuda_fail(e, "stream_collide launch");
    *v.launches += 1;
    cur = dst;
  }
  *v.cur = (v.state[0]->p == cur) ? 0 : 1;
  *v.steps = nsteps;
  r.final_buf = *v.cur;
  r.nsteps = nsteps;
  r.k = k;
  r.tail_kept = true;
  r.bounded = false;
  r.valid = true;
  return LBM_OK;
}

int lbm_record_bounded(lbm_ctx* ctx, int64_t nsteps, int64_t max_states) {
  if (!ctx) return ctx_fail(LBM_EINVAL, "ctx is NULL");
  CtxView v = ctx_view(ctx);
  if (!v.inited || !v.fields->p) return ctx_fail(LBM_ESTATE, "lbm_record_bounded needs lbm_init first");
  if (v.fixed_ends) return ctx_fail(LBM_EINVAL, "the adjoint does not cover fixed end planes");
  if (v.slab) return ctx_fail(LBM_EINVAL, "the adjoint does not cover slab halo exchanges");
  if (nsteps < 1 || max_states < 1) return ctx_fail(LBM_EINVAL, "nsteps and max_states must be >= 1");
  Record& r = *v.rec;
  r.valid = false;
  r.seg.clear();
  while (r.ckpt.size() > 1) r.ckpt.pop_back();
  if (r.ckpt.empty()) r.ckpt.emplace_back(new DevBuf());
  int rc = r.ckpt[0]->ensure(state_bytes(v), v.stream);
  if (rc) return rc;
  const double* f = static_cast<const double*>(v.fields->p);
  const size_t n = (size_t)v.g.ncell;
  cudaError_t e = v.ops->init(v.model, f, f + n, f + (size_t)(v.D + 1) * n, r.ckpt[0]->p, v.g, 0,
                                 v.g.ncell, v.stream);
  if (e != cudaSuccess) return ctx_cuda_fail(e, "init launch");
  *v.launches += 1;
  const void* cur = r.ckpt[0]->p;
  for (int64_t s = 0; s < nsteps; ++s) {
    void* dst = v.state[s & 1]->p;
    e = v.ops->step(v.model, cur, dst, v.g, v.omega, v.variant, v.status, nullptr, v.stream);
    if (e != cudaSuccess) return ctx_cuda_fail(e, "stream_collide launch");
    *v.launches += 1;
    cur = dst;
  }
  *v.cur = (nsteps - 1) & 1;
  *v.steps = nsteps;
  r.final_buf = *v.cur;
  r.nsteps = nsteps;
  r.k = nsteps;
  r.tail_kept = false;
  r.bounded = true;
  r.max_states = max_states;
  // optimal splits when the host table is small enough (~0.2 s at the limit)
  const int64_t F = max_states - 1;
  if ((double)nsteps * (double)nsteps * (double)F <= 2e8) optimal_splits(nsteps, F, &r.split);
  else r.split.clear();
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
  if (!r.bounded) {
    while ((int64_t)r.seg.size() < k - 1) r.seg.emplace_back(new DevBuf());
    for (int64_t j = 0; j < k - 1; ++j)
      if ((rc = r.seg[j]->ensure(sb, v.stream))) return rc;
  }
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

  Sweep sw;
  sw.v = v;
  sw.r = &r;
  if (r.bounded) {
    if ((rc = reverse_bounded(sw, 0, N, r.ckpt[0]->p, 1))) return rc;
    // the context's buffers served as work space: leave the initial state in them
    ADJ_CUDA(cudaMemcpyAsync(v.state[0]->p, r.ckpt[0]->p, sb, cudaMemcpyDeviceToDevice, v.stream));
    *v.cur = 0;
    *v.steps = 0;
  }
  // reverse sweep (uniform checkpoints)
  int& nu_cur = sw.nu_cur;  // buffer holding nu_{n+1} (undefined before the first step)
  bool& first = sw.first;
  const int64_t nseg = r.bounded ? 0 : (N + k - 1) / k;
  std::vector<void*> states((size_t)k);
  for (int64_t c = nseg - 1; c >= 0; --c) {
    const int64_t s0 = c * k;
    const int64_t s1 = (s0 + k < N) ? s0 + k : N;   // states S_s0 .. S_{s1-1}
    states[0] = r.ckpt[c]->p;
    // the last segment was kept by lbm_record (only on the first reverse sweep:
    // later segments' replays reuse the same buffers)
    const bool kept = r.tail_kept && c == nseg - 1;
    for (int64_t j = 1; j < s1 - s0; ++j) {
      states[j] = r.seg[j - 1]->p;
      if (kept) continue;
      cudaError_t e = v.ops->step(v.model, states[j - 1], states[j], v.g, v.omega, v.variant,
                                   v.status, nullptr, v.stream);
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
  if (!r.bounded) r.tail_kept = (nseg == 1);   // seg[] now holds segment 0's states
  if (r.bounded) r.valid = false;               // S_N is no longer in the context buffers
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

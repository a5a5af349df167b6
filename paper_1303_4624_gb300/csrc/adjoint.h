// adjoint.h - host-side types shared by lbm_api.cu and adjoint.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <vector>

#include "../../include/lbm.h"
#include "common.h"

namespace lbm {

// One device allocation, made through the caller's allocator when one is set.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  lbm_free_fn free_fn = nullptr;
  void* user = nullptr;
  void* stream = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf();
  void release();
  int ensure(size_t nbytes, cudaStream_t st);
};

// A checkpointed rollout: S_0, S_k, S_2k, ... and the buffers of the reverse sweep.
struct Record {
  bool valid = false;
  int64_t nsteps = 0;
  int64_t k = 0;
  int final_buf = 0;                            // state buffer holding S_N
  bool tail_kept = false;                       // seg[] holds the last segment's states
  bool bounded = false;                         // lbm_record_bounded: bisection schedule
  int64_t max_states = 0;                       // stored-state budget of the bounded schedule
  // optimal split points of the bounded schedule: split[l * (F + 1) + f] = how far to
  // advance before storing, for l steps to reverse with f free state slots (empty:
  // bisection); F = max_states - 1
  std::vector<int32_t> split;
  std::vector<std::unique_ptr<DevBuf>> ckpt;    // ceil(nsteps / k) states
  std::vector<std::unique_ptr<DevBuf>> seg;     // k - 1 replayed states
  DevBuf nu[2];                                 // adjoint ping-pong, Q * cells of the adjoint type
  DevBuf dldrho;                                // dL/drho_N staging (FP64)
  DevBuf omega_acc;                             // per-block partial sums of dL/domega
  DevBuf omega_out;                             // 1 double
  DevBuf grads;                                 // host-output staging (D + 2) * cells FP64
};

struct CtxView {
  int model, storage, D, Q;
  const StorageOps* ops;
  Grid g;
  double omega;
  cudaStream_t stream;
  DevBuf* state[2];
  int* cur;
  DevBuf* fields;
  bool inited;
  int64_t* steps;
  int64_t* launches;
  Record* rec;
  int variant;      // stream-collide kernel variant the context uses
  int* status;      // device status flag
  bool fixed_ends;  // fixed-state end planes active (no adjoint for them)
  bool slab;        // a slab of a decomposed grid (no adjoint across the halo exchange)
};

int ctx_fail(int code, const char* msg);
int ctx_cuda_fail(cudaError_t e, const char* what);
const ModelConst* ctx_model_const(int model);
CtxView ctx_view(lbm_ctx* c);
// Unique id of the CUDA context current on the calling thread (0 if none is current
// or the driver cannot tell).  A device reset destroys the primary context, and the
// next one has a new id: per-device set-up keyed by this id is redone after a reset.
unsigned long long current_context_id();

}  // namespace lbm

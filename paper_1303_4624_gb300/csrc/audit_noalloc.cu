// audit_noalloc.cu - conservation audit of caller-owned populations, with no
// device allocation (lbm_audit_noalloc in include/lbm.h).
//
// Some callers cannot call cudaMalloc: code whose device memory is owned in full
// by another allocator (a framework's memory pool that has reserved the GPU
// and does not expect outside allocations), or code in the middle of a time
// loop that must not pay for the device-wide synchronisation that cudaMalloc /
// cudaFree can cause.  For them this file runs the same per-block audit kernel
// and fixed-order reduction as lbm_audit, but on caller-owned input and output
// buffers, with the per-block partial sums kept in a file-scope __device__
// array instead of a context-owned allocation.
//
// The array is a static device symbol: every GPU that loads the library holds
// it (512 KiB) until the process exits.  Host code cannot use the symbol's name
// as a device address, so set-up takes the address with cudaGetSymbolAddress,
// once per device, with that device current.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/lbm.h"
#include "adjoint.h"
#include "kernels.cuh"

namespace {

using namespace lbm;

// Largest grid the static scratch serves: one slot row per 256-cell block.
constexpr int kNoAllocMaxBlocks = 8192;                          // 2,097,152 cells
static __device__ __align__(256) double g_audit_scratch[kNoAllocMaxBlocks * kAuditSlots];

struct DeviceSetup {
  int dev;
  unsigned long long ctx_id;   // the context the set-up was made in (0: unknown)
  double* scratch;             // device address of g_audit_scratch on `dev`
};
std::mutex g_mu;
std::vector<DeviceSetup> g_setup;

// Once per device and context, with that device current: the scratch address and
// this translation unit's copy of the constant-memory model tables.  Keyed by the
// context's id as well as the device, so that a device reset (which destroys the
// context, its module and its constant memory) leads to a fresh set-up.
int setup_current_device(double** scratch) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ctx_cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_mu);
  const unsigned long long id = current_context_id();
  for (const auto& s : g_setup)
    if (s.dev == dev && s.ctx_id == id) {
      *scratch = s.scratch;
      return LBM_OK;
    }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_audit_scratch);   // also makes the primary context current
  if (e != cudaSuccess) return ctx_cuda_fail(e, "cudaGetSymbolAddress(g_audit_scratch)");
  const ModelConst* m0 = ctx_model_const(0);
  const ModelConst* m1 = ctx_model_const(1);
  if (!m0 || !m1) return ctx_fail(LBM_EINVAL, "model table solve failed");
  ModelConst both[2] = {*m0, *m1};
  e = cudaMemcpyToSymbol(c_mc, both, sizeof both);
  if (e != cudaSuccess) return ctx_cuda_fail(e, "constant table upload");
  const float unit[2] = {1.0f, -1.0f};
  e = cudaMemcpyToSymbol(c_unit, unit, sizeof unit);
  if (e != cudaSuccess) return ctx_cuda_fail(e, "constant table upload");
  const unsigned long long now = current_context_id();
  for (auto it = g_setup.begin(); it != g_setup.end();)
    it = (it->dev == dev) ? g_setup.erase(it) : it + 1;
  g_setup.push_back({dev, now, static_cast<double*>(p)});
  *scratch = static_cast<double*>(p);
  return LBM_OK;
}

// True when p is device (or managed) memory of device `dev`.  Asks the driver
// about the pointer; allocates nothing.
bool is_device_pointer(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

template <class S>
cudaError_t launch(int model, const void* h, const Grid& g, double* scratch, double* out,
                   cudaStream_t st) {
  const int nb = moment_blocks(g.ncell);
  if (model == 0)
    k_moments<0, S><<<nb, kMomentThreads, 0, st>>>(static_cast<const S*>(h), g, nullptr, nullptr,
                                                   nullptr, scratch, 0, g.ncell);
  else
    k_moments<1, S><<<nb, kMomentThreads, 0, st>>>(static_cast<const S*>(h), g, nullptr, nullptr,
                                                   nullptr, scratch, 0, g.ncell);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_audit_reduce<<<1, 256, 0, st>>>(scratch, nb, out);
  return cudaGetLastError();
}

}  // namespace

extern "C" int lbm_audit_noalloc(int model, int storage, const int64_t dims[3], const void* h,
                                 size_t h_bytes, double* out, void* stream) {
  if (model != LBM_D2Q33 && model != LBM_D3Q95) return ctx_fail(LBM_EINVAL, "unknown model");
  if (storage < LBM_FP64 || storage > LBM_BF16DEV) return ctx_fail(LBM_EINVAL, "unknown storage");
  if (!dims || !h || !out) return ctx_fail(LBM_EINVAL, "dims, h and out are required");
  for (int k = 0; k < 3; ++k)
    if (dims[k] < 1 || dims[k] > 65535) return ctx_fail(LBM_EINVAL, "dims must be in [1, 65535]");
  if (model == LBM_D2Q33 && dims[2] != 1) return ctx_fail(LBM_EINVAL, "D2Q33 needs Nz == 1");
  const long long ncell = (long long)dims[0] * dims[1] * dims[2];
  if (moment_blocks(ncell) > kNoAllocMaxBlocks) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "lbm_audit_noalloc serves at most %d cells (static scratch); got %lld",
             kNoAllocMaxBlocks * kMomentThreads, ncell);
    return ctx_fail(LBM_EINVAL, msg);
  }
  const size_t esize = storage == LBM_FP64 ? 8 : (storage == LBM_FP32 ? 4 : 2);
  const size_t need = (size_t)(model == LBM_D2Q33 ? Model<0>::Q : Model<1>::Q) * (size_t)ncell * esize;
  if (h_bytes < need) {
    char msg[160];
    snprintf(msg, sizeof msg, "h holds %zu bytes; the grid's populations need %zu", h_bytes, need);
    return ctx_fail(LBM_EINVAL, msg);
  }
  double* scratch = nullptr;
  int rc = setup_current_device(&scratch);
  if (rc) return rc;
  int dev = 0;
  cudaError_t de = cudaGetDevice(&dev);
  if (de != cudaSuccess) return ctx_cuda_fail(de, "cudaGetDevice");
  if (!is_device_pointer(h, dev) || !is_device_pointer(out, dev))
    return ctx_fail(LBM_EINVAL, "h and out must be device memory of the current device");
  Grid g;
  g.nx = (int)dims[0];
  g.ny = (int)dims[1];
  g.nz = (int)dims[2];
  g.nxy = g.nx * g.ny;
  g.ncell = ncell;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (storage) {
    case LBM_FP64: e = launch<double>(model, h, g, scratch, out, st); break;
    case LBM_FP32: e = launch<float>(model, h, g, scratch, out, st); break;
    case LBM_FP16DEV: e = launch<__half>(model, h, g, scratch, out, st); break;
    default: e = launch<__nv_bfloat16>(model, h, g, scratch, out, st); break;
  }
  if (e != cudaSuccess) return ctx_cuda_fail(e, "audit launch");
  return LBM_OK;
}

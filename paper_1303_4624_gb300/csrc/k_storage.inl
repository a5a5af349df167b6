// k_storage.inl - launchers of one storage form.  Included by k_fp64.cu,
// k_fp32.cu, k_fp16.cu and k_bf16.cu after defining LBM_STORE (element type) and
// LBM_OPS (name of the StorageOps table).
#include <algorithm>
#include <mutex>

#include "kernels.cuh"
#include "stream_collide_tma.cuh"
#include "stream_collide_pair.cuh"
#include "adjoint_kernels.cuh"

namespace lbm {
namespace {

using S = LBM_STORE;

cudaError_t upload(const ModelConst* mc2) {
  const float unit[2] = {1.0f, -1.0f};
  cudaError_t e = cudaMemcpyToSymbol(c_unit, unit, sizeof unit);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_mc, mc2, 2 * sizeof(ModelConst));
}

template <int M>
cudaError_t init_m(const double* rho, const double* U, const double* T, void* dst, const Grid& g,
                   long long begin, long long end, cudaStream_t st) {
  const int bs = 256;
  const long long nb = (end - begin + bs - 1) / bs;
  if (nb <= 0) return cudaSuccess;
  k_init<M, S><<<(unsigned)nb, bs, 0, st>>>(rho, U, T, static_cast<S*>(dst), g, begin, end);
  return cudaGetLastError();
}

// TMA-kernel configuration per model and storage type: pipeline depth, resident CTAs
// per SM the registers are capped for, and whether the results go out through a
// shared-memory tile and bulk stores (16-bit forms) or straight from the threads.
// Shared memory per CTA = STAGES x (stage of Q shifted row segments) + output tile:
// D3Q95 FP16 2 x 25,440 B (4 CTAs per SM); D2Q33 FP16 3 x 8,864 + 8,448 B.
template <int M, class T>
struct TmaCfg {
  static constexpr int kStages = 2;
  static constexpr int kMinBlocks = (M == 1) ? 2 : 3;     // FP32
  static constexpr bool kOutSmem = false;
};
template <int M>
struct TmaCfg<M, double> {
  static constexpr int kStages = 2;
  static constexpr int kMinBlocks = (M == 1) ? 1 : 2;
  static constexpr bool kOutSmem = false;
};
// 16-bit forms: D3Q95 stores straight from the threads with 4 CTAs (128 registers)
// per SM (measured at 512 x 256 x 256: 8.6 GLUPS, against 5.5 with the
// shared-memory output tile and bulk stores, whose two block barriers per chunk
// leave the warps waiting on warp 0's copy work); D2Q33 keeps the output tile.
template <int M>
struct TmaCfg<M, __half> {
  static constexpr int kStages = (M == 1) ? 2 : 3;
  static constexpr int kMinBlocks = (M == 1) ? 4 : 6;
  static constexpr bool kOutSmem = (M == 0);
};
template <int M>
struct TmaCfg<M, __nv_bfloat16> : TmaCfg<M, __half> {};

template <int M>
struct TmaKernel {
  using C = TmaCfg<M, S>;
  using Smem = TmaSmem<M, S, C::kStages, C::kOutSmem>;
  static constexpr auto kern = k_stream_collide_tma<M, S, C::kStages, C::kMinBlocks, C::kOutSmem>;
};

struct LaunchCache {
  int dev = -1;
  int grid = 0;
};
std::mutex g_tma_mu;
LaunchCache g_tma_cache[2][16];

// Shared-memory opt-in and the persistent grid (resident CTAs per SM x SMs), once
// per device and model.
template <int M>
cudaError_t prepare_tma_m(int* grid_out) {
  using K = TmaKernel<M>;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_tma_mu);
  LaunchCache& lc = g_tma_cache[M][dev & 15];
  if (lc.dev != dev) {
    e = cudaFuncSetAttribute(K::kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::Smem::kBytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, K::kern, kTmaW, K::Smem::kBytes);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    lc.grid = per_sm * sms;
    lc.dev = dev;
  }
  if (grid_out) *grid_out = lc.grid;
  return cudaSuccess;
}

cudaError_t prepare_tma(int m) {
  return m == 0 ? prepare_tma_m<0>(nullptr) : prepare_tma_m<1>(nullptr);
}

template <int M>
cudaError_t step_tma_m(const void* src, void* dst, const Grid& g, double omega, int* status,
                       const StepTest* test, cudaStream_t st) {
  using K = TmaKernel<M>;
  int cap = 0;
  cudaError_t e = prepare_tma_m<M>(&cap);
  if (e != cudaSuccess) return e;
  const long long nchunks = (long long)((g.nx + kTmaW - 1) / kTmaW) * g.ny * g.nz;
  const int grid = (int)(nchunks < cap ? nchunks : cap);
  TmaTest t;
  t.stall_chunk = test ? test->stall_chunk : -1;
  t.limit_ns = test ? test->limit_ns : 1000000000ull;   // 1 s: far beyond any copy's latency
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kTmaW);
  cfg.dynamicSmemBytes = K::Smem::kBytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, K::kern, static_cast<const S*>(src), static_cast<S*>(dst), g,
                            omega, (int)nchunks, status, t);
}

// The pair kernel (16-bit forms): 64-thread blocks of 128 cells, like the direct
// kernel's grid.
template <int M>
cudaError_t step_pair_m(const void* src, void* dst, const Grid& g, double omega, int rev,
                        cudaStream_t st) {
  const int cells = 2 * kPairThreads;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((g.nx + cells - 1) / cells), (unsigned)g.ny, (unsigned)g.nz);
  cfg.blockDim = dim3(kPairThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  auto kern = rev ? k_stream_collide_pair<M, S, true, false> : k_stream_collide_pair<M, S, false, false>;
  if constexpr (PairNarrow<M>::value) {
    if ((unsigned long long)Model<M>::Q * (unsigned long long)g.ncell <= 0xFFFFFFFFull)
      kern = rev ? k_stream_collide_pair<M, S, true, true> : k_stream_collide_pair<M, S, false, true>;
  }
  return cudaLaunchKernelEx(&cfg, kern, static_cast<const S*>(src), static_cast<S*>(dst), g, omega);
}

// The direct kernel for this grid: 32-bit element indices (where the form uses
// them) when Q ncell fits them.
using DirectFn = void (*)(const S*, S*, Grid, double);
template <int M>
DirectFn direct_kernel(const Grid& g, int rev) {
  if constexpr (DirectNarrow<M, S>::value) {
    if ((unsigned long long)Model<M>::Q * (unsigned long long)g.ncell <= 0xFFFFFFFFull)
      return rev ? k_stream_collide<M, S, true, true> : k_stream_collide<M, S, false, true>;
  }
  return rev ? k_stream_collide<M, S, true, false> : k_stream_collide<M, S, false, false>;
}

template <int M>
cudaError_t step_m(const void* src, void* dst, const Grid& g, double omega, int variant, int* status,
                   const StepTest* test, cudaStream_t st) {
  const int rev = (variant & kStepReverse) ? 1 : 0;
  variant &= ~kStepReverse;
  if (variant == kVariantTma) return step_tma_m<M>(src, dst, g, omega, status, test, st);
  if constexpr (sizeof(S) == 2) {
    if (variant == kVariantPair) return step_pair_m<M>(src, dst, g, omega, rev, st);
  }
  if constexpr (!std::is_same<S, double>::value) {
    if (variant == kVariantSplit) {
      constexpr int cells = kSplitThreads / 2;
      const dim3 grid((unsigned)((g.nx + cells - 1) / cells), (unsigned)g.ny, (unsigned)g.nz);
      k_stream_collide_split<M, S><<<grid, kSplitThreads, 0, st>>>(
          static_cast<const S*>(src), static_cast<S*>(dst), g, omega);
      return cudaGetLastError();
    }
  }
  const int bx = cell_block_x(g.nx);
  const dim3 grid((unsigned)((g.nx + bx - 1) / bx), (unsigned)g.ny, (unsigned)g.nz);
#ifndef LBM_NO_PDL
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(bx);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, direct_kernel<M>(g, rev), static_cast<const S*>(src),
                            static_cast<S*>(dst), g, omega);
#else
  direct_kernel<M>(g, rev)<<<grid, bx, 0, st>>>(static_cast<const S*>(src), static_cast<S*>(dst), g,
                                                omega);
  return cudaGetLastError();
#endif
}

template <int M>
cudaError_t moments_m(const void* src, const Grid& g, double* rho, double* U, double* T,
                      double* partials, long long block0, long long nblocks, cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  const long long end = std::min(g.ncell, (block0 + nblocks) * (long long)kMomentThreads);
  k_moments<M, S><<<(unsigned)nblocks, kMomentThreads, 0, st>>>(static_cast<const S*>(src), g, rho,
                                                                U, T, partials, block0, end);
  return cudaGetLastError();
}

template <int M>
cudaError_t get_f_m(const void* src, double* f, const Grid& g, cudaStream_t st) {
  k_get_f<M, S><<<1024, 256, 0, st>>>(static_cast<const S*>(src), f, g);
  return cudaGetLastError();
}

template <int M>
cudaError_t set_f_m(const double* f, void* dst, const Grid& g, cudaStream_t st) {
  k_set_f<M, S><<<1024, 256, 0, st>>>(f, static_cast<S*>(dst), g);
  return cudaGetLastError();
}

#include "k_adjoint.inl"

cudaError_t fix_ends(void* state, const Grid& g, int axis, int width, const void* tmpl, int Q,
                     cudaStream_t st) {
  k_fix_ends<S><<<256, 256, 0, st>>>(static_cast<S*>(state), g, axis, width,
                                     static_cast<const S*>(tmpl), Q);
  return cudaGetLastError();
}

cudaError_t halo_copy(void* state, void* buf, const int* segs, int nseg, long long plane,
                      long long ncell, int to_buf, cudaStream_t st) {
  const long long n = (long long)nseg * plane;
  const long long nb = (n + 255) / 256;
  k_halo_copy<S><<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, st>>>(
      static_cast<S*>(state), static_cast<S*>(buf), reinterpret_cast<const int2*>(segs), nseg, plane,
      ncell, to_buf);
  return cudaGetLastError();
}

cudaError_t init(int m, const double* rho, const double* U, const double* T, void* dst,
                 const Grid& g, long long begin, long long end, cudaStream_t st) {
  return m == 0 ? init_m<0>(rho, U, T, dst, g, begin, end, st)
                : init_m<1>(rho, U, T, dst, g, begin, end, st);
}
cudaError_t step(int m, const void* src, void* dst, const Grid& g, double omega, int variant,
                 int* status, const StepTest* test, cudaStream_t st) {
  return m == 0 ? step_m<0>(src, dst, g, omega, variant, status, test, st)
                : step_m<1>(src, dst, g, omega, variant, status, test, st);
}
cudaError_t moments(int m, const void* src, const Grid& g, double* rho, double* U, double* T,
                    double* partials, long long block0, long long nblocks, cudaStream_t st) {
  return m == 0 ? moments_m<0>(src, g, rho, U, T, partials, block0, nblocks, st)
                : moments_m<1>(src, g, rho, U, T, partials, block0, nblocks, st);
}
cudaError_t get_f(int m, const void* src, double* f, const Grid& g, cudaStream_t st) {
  return m == 0 ? get_f_m<0>(src, f, g, st) : get_f_m<1>(src, f, g, st);
}
cudaError_t set_f(int m, const double* f, void* dst, const Grid& g, cudaStream_t st) {
  return m == 0 ? set_f_m<0>(f, dst, g, st) : set_f_m<1>(f, dst, g, st);
}

}  // namespace

const StorageOps LBM_OPS = {(int)sizeof(S), upload,       init,      step,         prepare_tma,
                            moments,        get_f,        set_f,     fix_ends,     halo_copy,
                            (int)sizeof(L), adjoint_step, grad_init};

}  // namespace lbm

// stream_collide_pair.cuh - two cells per thread on the paired FP32 instructions
// (sm_103a), for the FP16 / BF16 deviation forms.
//
// The 16-bit forms move half the bytes of the FP32 form, so one thread per cell
// leaves them bound by instruction issue: each cell update costs ~2300
// instructions, more than half of them FP32 arithmetic (moments, temperature,
// equilibrium, relaxation).  Here a thread updates the two neighbouring cells
// x and x + 1 of a row together:
//   * every FP32 operation of cell_collide runs once on a float2 (lane .x cell x,
//     lane .y cell x + 1) through the paired instructions (__fadd2_rn,
//     __fmul2_rn, __ffma2_rn), each lane rounded exactly as the scalar operation,
//     so the results are bitwise those of the one-cell kernels;
//   * the two cells' populations of a direction are adjacent in memory: for even
//     e_x the pair (x - e_x, x + 1 - e_x) is one aligned 32-bit load; for odd e_x
//     it is two 16-bit loads (the second may wrap to x = 0), packed;
//   * the Q populations stay packed (one 32-bit register per direction for both
//     cells) and are unpacked to float2 where they are used;
//   * each direction's two results leave as one packed, aligned 32-bit store.
// Needs Nx even (so that x and x + 1 share a row and pairs start 4-byte aligned).
#pragma once

#include "kernels.cuh"

namespace lbm {

template <class S>
struct PairCodec;
// dec() is volatile inline PTX on purpose: each population is decoded where it is
// used (once for the moments, once for the relaxation), so only the packed pair
// stays live in between; a decode the compiler could merge would keep two FP32
// registers per direction alive instead of one packed register and spill.
template <>
struct PairCodec<__half> {
  using P = __half2;
  static __device__ __forceinline__ float2 dec(P v) {
    float2 r;
    asm volatile("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
                 "cvt.f32.f16 %0, lo;\n\tcvt.f32.f16 %1, hi;\n\t}"
                 : "=f"(r.x), "=f"(r.y)
                 : "r"(*reinterpret_cast<const uint32_t*>(&v)));
    return r;
  }
  static __device__ __forceinline__ P enc(float2 v) { return __float22half2_rn(v); }
  static __device__ __forceinline__ P make(__half lo, __half hi) { return __halves2half2(lo, hi); }
};
template <>
struct PairCodec<__nv_bfloat16> {
  using P = __nv_bfloat162;
  static __device__ __forceinline__ float2 dec(P v) {
    float2 r;
    asm volatile("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
                 "cvt.f32.bf16 %0, lo;\n\tcvt.f32.bf16 %1, hi;\n\t}"
                 : "=f"(r.x), "=f"(r.y)
                 : "r"(*reinterpret_cast<const uint32_t*>(&v)));
    return r;
  }
  static __device__ __forceinline__ P enc(float2 v) { return __float22bfloat162_rn(v); }
  static __device__ __forceinline__ P make(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return __halves2bfloat162(lo, hi);
  }
};

#ifndef LBM_PAIR_THREADS
#define LBM_PAIR_THREADS 64
#endif
constexpr int kPairThreads = LBM_PAIR_THREADS;     // 2 cells per thread

// Resident 64-thread blocks per SM the registers are capped for: D2Q33 128
// registers at 8 (16 warps per SM); D3Q95 168 at 6 (12 warps per SM).
#ifndef LBM_PAIR_MINB_D3Q95
#define LBM_PAIR_MINB_D3Q95 6
#endif
#ifndef LBM_PAIR_MINB_D2Q33
#define LBM_PAIR_MINB_D2Q33 8
#endif
template <int M>
struct PairMinBlocks {
  static constexpr int value = M == 1 ? LBM_PAIR_MINB_D3Q95 : LBM_PAIR_MINB_D2Q33;
};
// 32-bit element indices (see k_stream_collide's NARROW) for D3Q95 when Q ncell fits
// them: 11.9 against 11.4 GLUPS in FP16 at 512x256x256; D2Q33 measured slower with
// them (37.6 against 38.3 GLUPS at 4096x2048).
template <int M>
struct PairNarrow {
  static constexpr bool value = M == 1;
};

// The Q packed pairs stay in registers between the gather and their two uses.
// D3Q95 (CHAIN): the relaxation decodes direction i's pair only once the previous
// direction's result exists (the packed pair is OR-ed with that result masked by a
// zero read from constant memory, which the compiler cannot see through).  Without
// the dependency the compiler decodes the pairs ahead of their use: 190 more live
// registers, so the kernel needed 255 registers (8 warps per SM) and still spilled;
// with it, 168 (12 warps per SM).  One extra integer instruction per direction; the
// values, and so the results, are unchanged.  D2Q33 fits without it, and measured
// slower with it (36.8-37.8 against 38.3 GLUPS at 4096x2048).
// REV: walk the blocks in reverse order (see k_stream_collide).
template <int M, class S, bool REV, bool NARROW>
__global__ void __launch_bounds__(kPairThreads, PairMinBlocks<M>::value)
    k_stream_collide_pair(const S* __restrict__ src, S* __restrict__ dst, Grid g, double omega) {
  using Mo = Model<M>;
  using PC = PairCodec<S>;
  using P = typename PC::P;
  constexpr int D = Mo::D, RR = Mo::R, Q = Mo::Q;
  constexpr bool CHAIN = M == 1;
  wait_prior_grid();
  allow_next_grid();
  const int bx = REV ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
  const int x = 2 * (bx * kPairThreads + (int)threadIdx.x);
  if (x >= g.nx) return;
  const int y = REV ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
  const int z = REV ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z;
  int xo[2 * RR + 1], yo[2 * RR + 1], zo[2 * RR + 1];
  neighbour_offsets<D, RR>(x, y, z, g.nx, g.ny, g.nz, g.nxy, xo, yo, zo);
  // a1 + a2 gather: Q packed pairs.  For even e_x the pair (x - e_x, x + 1 - e_x) is
  // one aligned 32-bit read; for odd e_x two 16-bit reads (the second may wrap to
  // x = 0), packed.
  P h2[Q];
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ex = Mo::vs.e[i][0], ey = Mo::vs.e[i][1], ez = Mo::vs.e[i][2];
    const int xs = xo[ex + RR];                    // (x - e_x) mod Nx
    if constexpr (NARROW) {
      const uint32_t row = (uint32_t)i * (uint32_t)g.ncell + (uint32_t)(zo[ez + RR] + yo[ey + RR]);
      if constexpr ((ex & 1) == 0) {
        h2[i] = __ldg(reinterpret_cast<const P*>(src + (row + (uint32_t)xs)));
      } else {
        const int xs1 = (xs + 1 == g.nx) ? 0 : xs + 1;     // (x + 1 - e_x) mod Nx
        h2[i] = PC::make(__ldg(src + (row + (uint32_t)xs)), __ldg(src + (row + (uint32_t)xs1)));
      }
    } else {
      const S* row = src + (size_t)i * (size_t)g.ncell + (zo[ez + RR] + yo[ey + RR]);
      if constexpr ((ex & 1) == 0) {
        h2[i] = __ldg(reinterpret_cast<const P*>(row + xs));   // xs even: aligned pair
      } else {
        const int xs1 = (xs + 1 == g.nx) ? 0 : xs + 1;     // (x + 1 - e_x) mod Nx
        h2[i] = PC::make(__ldg(row + xs), __ldg(row + xs1));
      }
    }
  });
  S* const obase = dst + (((size_t)z * g.ny + y) * g.nx + x);
  const uint32_t zmask = __float_as_uint(c_unit[0]) ^ 0x3f800000u;   // 0
  uint32_t last = 0;                                                   // last stored pair
  cell_collide_with2<M, S, float2>(
      [&](auto I) { return PC::dec(h2[decltype(I)::value]); },
      [&](auto I) {
        if constexpr (CHAIN) {
          const uint32_t b =
              *reinterpret_cast<const uint32_t*>(&h2[decltype(I)::value]) | (last & zmask);
          return PC::dec(*reinterpret_cast<const P*>(&b));
        } else {
          return PC::dec(h2[decltype(I)::value]);
        }
      },
      omega,
      [&](auto I, float2 v) {
        constexpr int i = decltype(I)::value;
        const P pv = PC::enc(v);
        if constexpr (CHAIN) last = *reinterpret_cast<const uint32_t*>(&pv);
        if constexpr (NARROW)
          *reinterpret_cast<P*>(dst + ((uint32_t)i * (uint32_t)g.ncell +
                                       (uint32_t)((z * g.ny + y) * g.nx + x))) = pv;
        else
          *reinterpret_cast<P*>(obase + (size_t)i * (size_t)g.ncell) = pv;
      });
}

}  // namespace lbm

// kernels.cuh - sm_103a kernels of the thermal LBM hot path (templates).
//
// Included by one translation unit per storage form (k_fp64.cu, k_fp32.cu,
// k_fp16.cu, k_bf16.cu); each gets its own copy of the constant-memory model
// table and instantiates every kernel for D2Q33 and D3Q95.
//
// State layout (HBM): structure of arrays, h[i][cell] with cell = (z*Ny + y)*Nx + x,
// two buffers (ping-pong).  The stored value is the deviation h_i = f_i / w_i - 1
// from the rest state (rho0 = 1, u = 0, theta = 1 where f_i^eq = w_i).
//
// Notation (unit-variance variables of the Hermite expansion): xi_i = a e_i with
// a = sqrt(2) c; u = a U_lattice; theta = T / T0 with T0 = 1/(2 c^2).  The
// fourth-order Hermite equilibrium (Formula 1 with m = N = 4, expansion about
// u = 0, theta = 1) written as a polynomial in s = xi_i . u for one direction is
//     f_i^eq / (w_i rho) = A0 + A1 s + A2 s^2 + s^3/6 + s^4/24
// where, with q = |u|^2, t = theta - 1 and x2 = |xi_i|^2 (the same for every
// member of a symmetry group),
//     A0 = 1 - q/2 + t(x2-D)/2 + [3q^2 + 6t(D+2-x2)q + 3t^2(x2^2 - 2(D+2)x2 + D(D+2))]/24
//     A1 = 1 - q/2 + t(x2-D-2)/2
//     A2 = 1/2 - q/4 + t(x2-D-4)/4.
// The even part A0 + A2 s^2 + s^4/24 is shared by the two members of an
// opposite pair (s -> -s); the odd part A1 s + s^3/6 changes sign.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "common.h"
#include "velset.cuh"

namespace lbm {

static __constant__ ModelConst c_mc[2];

// ----------------------------------------------------------------- storage codecs
template <class S>
struct Codec;
template <>
struct Codec<double> {
  using R = double;
  static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
  static __device__ __forceinline__ double enc(double v) { return v; }
};
template <>
struct Codec<float> {
  using R = float;
  static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
  static __device__ __forceinline__ float enc(double v) { return (float)v; }
};
template <>
struct Codec<__half> {
  using R = float;
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ __half enc(double v) { return __double2half(v); }
};
template <>
struct Codec<__nv_bfloat16> {
  using R = float;
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
  }
  static __device__ __forceinline__ __nv_bfloat16 enc(double v) { return __double2bfloat16(v); }
};
template <class S>
__device__ __forceinline__ double to_double(S v) {
  if constexpr (std::is_same<S, __half>::value)
    return (double)__half2float(v);
  else if constexpr (std::is_same<S, __nv_bfloat16>::value)
    return (double)__bfloat162float(v);
  else
    return (double)v;
}

// ----------------------------------------------------------------- helpers
template <int I, int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    sfor<I + 1, N>(f);
  }
}

// True modulo for |v| up to a few multiples of n (grids smaller than the reach are legal).
__device__ __forceinline__ int wrapi(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

template <class R>
__device__ __forceinline__ R gW(const ModelConst& mc, int g) {
  if constexpr (std::is_same<R, double>::value) return mc.W[g]; else return mc.Wf[g];
}
template <class R>
__device__ __forceinline__ R gX2(const ModelConst& mc, int g) {
  if constexpr (std::is_same<R, double>::value) return mc.X2[g]; else return mc.X2f[g];
}

// Kahan compensated accumulation: the running error is kept in c (true sum ~ s - c).
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Coefficients of A0, A1, A2 as functions of the group's x2 (see file header).
template <class R, int D>
struct EqCoef {
  R K0, K1, K2, L0, L1, M0, M1;
  __device__ __forceinline__ EqCoef(R q, R t) {
    K0 = R(1) - q * R(0.5) - t * R(0.5 * D) + q * q * R(0.125) + t * q * R(0.25 * (D + 2)) +
         t * t * R(0.125 * D * (D + 2));
    K1 = t * R(0.5) - t * q * R(0.25) - t * t * R(0.25 * (D + 2));
    K2 = t * t * R(0.125);
    L0 = R(1) - q * R(0.5) - t * R(0.5 * (D + 2));
    L1 = t * R(0.5);
    M0 = R(0.5) - q * R(0.25) - t * R(0.25 * (D + 4));
    M1 = t * R(0.25);
  }
  __device__ __forceinline__ R A0(R x2) const { return K0 + x2 * (K1 + x2 * K2); }
  __device__ __forceinline__ R A1(R x2) const { return L0 + L1 * x2; }
  __device__ __forceinline__ R A2(R x2) const { return M0 + M1 * x2; }
};

// ----------------------------------------------------------------- fused stream-collide
// One thread per cell, x fastest across the block; blockIdx.y / z give the row.
// a1 pull-gather  g_i(x) = F_i((x - e_i) mod N)         (Q loads, coalesced along x)
// a2 decode       f_i = w_i (1 + h_i)                    (kept as h_i)
// a3 moments      rho - 1 = sum w_i h_i, j = sum w_i h_i xi_i, E - D = sum w_i h_i |xi_i|^2
//                 (rest moments sum w = 1, sum w xi = 0, sum w |xi|^2 = D are exact)
// a4 temperature  theta = (E/rho - |u|^2)/D in FP64
// a5 equilibrium  per group A0, A1, A2; per pair the even / odd parts in s
// a6 BGK          h_i' = (1 - omega) h_i + omega (rho P_i - 1), stored at x
template <int M, class S>
__global__ void __launch_bounds__(128)
    k_stream_collide(const S* __restrict__ src, S* __restrict__ dst, Grid g, double omega) {
  using Mo = Model<M>;
  using Rt = typename Codec<S>::R;
  constexpr int Q = Mo::Q, D = Mo::D, RR = Mo::R, NP = Mo::NP, G = Mo::G;
  constexpr bool kComp = std::is_same<Rt, float>::value;
  const ModelConst& mc = c_mc[M];

  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;

  int xo[2 * RR + 1], yo[2 * RR + 1], zo[2 * RR + 1];
  sfor<0, 2 * RR + 1>([&](auto K) {
    constexpr int k = decltype(K)::value;
    xo[k] = wrapi(x - (k - RR), g.nx);
    yo[k] = wrapi(y - (k - RR), g.ny) * g.nx;
    if constexpr (D == 3) zo[k] = wrapi(z - (k - RR), g.nz) * g.nxy; else zo[k] = 0;
  });

  // a1 + a2: gather
  Rt h[Q];
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ex = Mo::vs.e[i][0], ey = Mo::vs.e[i][1], ez = Mo::vs.e[i][2];
    const int cell = zo[ez + RR] + yo[ey + RR] + xo[ex + RR];
    h[i] = Codec<S>::ld(src + (size_t)i * (size_t)g.ncell + cell);
  });

  // a3: moments (deviation form)
  Rt rs = gW<Rt>(mc, 0) * h[0], rc = Rt(0), es = Rt(0), ec = Rt(0);
  Rt jx = Rt(0), jy = Rt(0), jz = Rt(0);
  sfor<0, NP>([&](auto P) {
    constexpr int p = decltype(P)::value;
    constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
    constexpr int gg = Mo::vs.grp[ip];
    constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
    const Rt sp = h[ip] + h[im];
    const Rt dm = h[ip] - h[im];
    const Rt tr = gW<Rt>(mc, gg) * sp;
    const Rt te = gX2<Rt>(mc, gg) * tr;
    if constexpr (kComp) {
      kahan_add(rs, rc, tr);
      kahan_add(es, ec, te);
    } else {
      rs += tr;
      es += te;
    }
    const Rt tj = gW<Rt>(mc, gg) * dm;
    if constexpr (ex != 0) jx += Rt(ex) * tj;
    if constexpr (ey != 0) jy += Rt(ey) * tj;
    if constexpr (ez != 0) jz += Rt(ez) * tj;
  });

  // a4: FP64 temperature recovery
  const double rho = 1.0 + ((double)rs - (double)rc);
  const double E = (double)D + ((double)es - (double)ec);
  const double ir = 1.0 / rho;
  const double ux = mc.a * (double)jx * ir;
  const double uy = mc.a * (double)jy * ir;
  const double uz = (D == 3) ? mc.a * (double)jz * ir : 0.0;
  const double qd = ux * ux + uy * uy + uz * uz;
  const double theta = (E * ir - qd) * (1.0 / D);

  // a5 + a6: equilibrium and BGK
  const EqCoef<Rt, D> cf((Rt)qd, (Rt)(theta - 1.0));
  const Rt uax = (Rt)(mc.a * ux), uay = (Rt)(mc.a * uy), uaz = (Rt)(mc.a * uz);
  const Rt om1 = (Rt)(1.0 - omega);
  const Rt wr = (Rt)(omega * rho);
  const Rt nw = (Rt)(-omega);
  const size_t self = ((size_t)z * g.ny + y) * g.nx + x;

  Rt A0[G], A1[G], A2[G];
  sfor<0, G>([&](auto GG) {
    constexpr int gg = decltype(GG)::value;
    const Rt x2 = gX2<Rt>(mc, gg);
    A0[gg] = cf.A0(x2);
    A1[gg] = cf.A1(x2);
    A2[gg] = cf.A2(x2);
  });

  {
    const Rt hn = om1 * h[0] + (wr * cf.K0 + nw);
    Codec<S>::st(dst + self, hn);
  }
  sfor<0, NP>([&](auto P) {
    constexpr int p = decltype(P)::value;
    constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
    constexpr int gg = Mo::vs.grp[ip];
    constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
    Rt s = Rt(0);
    if constexpr (ex != 0) s += Rt(ex) * uax;
    if constexpr (ey != 0) s += Rt(ey) * uay;
    if constexpr (ez != 0) s += Rt(ez) * uaz;
    const Rt s2 = s * s;
    const Rt ev = s2 * (s2 * Rt(1.0 / 24.0) + A2[gg]) + A0[gg];
    const Rt od = s * (s2 * Rt(1.0 / 6.0) + A1[gg]);
    const Rt base = wr * ev + nw;
    const Rt wod = wr * od;
    const Rt hp = om1 * h[ip] + (base + wod);
    const Rt hm = om1 * h[im] + (base - wod);
    Codec<S>::st(dst + (size_t)ip * (size_t)g.ncell + self, hp);
    Codec<S>::st(dst + (size_t)im * (size_t)g.ncell + self, hm);
  });
}

// ----------------------------------------------------------------- equilibrium init (FP64)
// h_i = rho P_i(u, theta) - 1 for the fields rho, U (lattice), T (lattice) of each cell.
template <int M, class S>
__global__ void __launch_bounds__(256)
    k_init(const double* __restrict__ rho, const double* __restrict__ U,
           const double* __restrict__ T, S* __restrict__ dst, Grid g) {
  using Mo = Model<M>;
  constexpr int D = Mo::D, NP = Mo::NP;
  const ModelConst& mc = c_mc[M];
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.ncell) return;
  const double r = rho[idx];
  const double ux = mc.a * U[idx];
  const double uy = mc.a * U[g.ncell + idx];
  const double uz = (D == 3) ? mc.a * U[2 * g.ncell + idx] : 0.0;
  const double theta = T[idx] / mc.T0;
  const EqCoef<double, D> cf(ux * ux + uy * uy + uz * uz, theta - 1.0);
  const double uax = mc.a * ux, uay = mc.a * uy, uaz = mc.a * uz;
  dst[idx] = Codec<S>::enc(r * cf.K0 - 1.0);
  sfor<0, NP>([&](auto P) {
    constexpr int p = decltype(P)::value;
    constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
    constexpr int gg = Mo::vs.grp[ip];
    constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
    const double x2 = mc.X2[gg];
    const double s = ex * uax + ey * uay + ez * uaz;
    const double s2 = s * s;
    const double ev = cf.A0(x2) + s2 * (cf.A2(x2) + s2 * (1.0 / 24.0));
    const double od = s * (cf.A1(x2) + s2 * (1.0 / 6.0));
    dst[(size_t)ip * g.ncell + idx] = Codec<S>::enc(r * (ev + od) - 1.0);
    dst[(size_t)im * g.ncell + idx] = Codec<S>::enc(r * (ev - od) - 1.0);
  });
}

// ----------------------------------------------------------------- moments + audit (FP64)
// Per cell rho = sum f, rho U = sum f e, D rho T = sum f |e|^2 - rho |U|^2 (lattice
// units), f_i = w_i (1 + h_i).  Each block also writes 8 FP64 audit partials:
// mass, momentum (3), energy, min f/w, non-finite count, cells.

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <int M, class S>
__global__ void __launch_bounds__(kMomentThreads)
    k_moments(const S* __restrict__ src, Grid g, double* __restrict__ rho_out,
              double* __restrict__ U_out, double* __restrict__ T_out,
              double* __restrict__ partials) {
  using Mo = Model<M>;
  constexpr int D = Mo::D, Q = Mo::Q;
  const ModelConst& mc = c_mc[M];
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc[kAuditSlots] = {0, 0, 0, 0, 0, 1e300, 0, 0};
  if (idx < g.ncell) {
    double r = 0, mx = 0, my = 0, mz = 0, e2 = 0, mn = 1e300, bad = 0;
    sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int ex = Mo::vs.e[i][0], ey = Mo::vs.e[i][1], ez = Mo::vs.e[i][2];
      const double hv = to_double(src[(size_t)i * g.ncell + idx]);
      const double f = mc.w[i] * (1.0 + hv);
      if (!isfinite(hv)) bad += 1.0;
      mn = fmin(mn, 1.0 + hv);
      r += f;
      mx += ex * f;
      my += ey * f;
      mz += ez * f;
      e2 += (ex * ex + ey * ey + ez * ez) * f;
    });
    const double Ux = mx / r, Uy = my / r, Uz = mz / r;
    const double Tl = (e2 / r - (Ux * Ux + Uy * Uy + Uz * Uz)) / D;
    if (rho_out) rho_out[idx] = r;
    if (U_out) {
      U_out[idx] = Ux;
      U_out[g.ncell + idx] = Uy;
      if (D == 3) U_out[2 * g.ncell + idx] = Uz;
    }
    if (T_out) T_out[idx] = Tl;
    acc[0] = r; acc[1] = mx; acc[2] = my; acc[3] = mz; acc[4] = 0.5 * e2;
    acc[5] = mn; acc[6] = bad; acc[7] = 1.0;
  }
  __shared__ double sh[kMomentThreads / 32][kAuditSlots];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kAuditSlots; ++k) {
    const double v = (k == 5) ? warp_min(acc[k]) : warp_sum(acc[k]);
    if (lane == 0) sh[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kAuditSlots) {
    const int k = threadIdx.x;
    double v = sh[0][k];
    for (int w = 1; w < kMomentThreads / 32; ++w) v = (k == 5) ? fmin(v, sh[w][k]) : v + sh[w][k];
    partials[(size_t)blockIdx.x * kAuditSlots + k] = v;
  }
}

// Fixed-order reduction of the audit partials by one block of 256 threads.
static __global__ void __launch_bounds__(256) k_audit_reduce(const double* __restrict__ partials,
                                                      int nblocks, double* __restrict__ out) {
  double acc[kAuditSlots] = {0, 0, 0, 0, 0, 1e300, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < kAuditSlots; ++k) {
      const double v = partials[(size_t)b * kAuditSlots + k];
      acc[k] = (k == 5) ? fmin(acc[k], v) : acc[k] + v;
    }
  __shared__ double sh[8][kAuditSlots];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kAuditSlots; ++k) {
    const double v = (k == 5) ? warp_min(acc[k]) : warp_sum(acc[k]);
    if (lane == 0) sh[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kAuditSlots) {
    const int k = threadIdx.x;
    double v = sh[0][k];
    for (int w = 1; w < 8; ++w) v = (k == 5) ? fmin(v, sh[w][k]) : v + sh[w][k];
    out[k] = v;
  }
}

// ----------------------------------------------------------------- population I/O (FP64)
template <int M, class S>
__global__ void k_get_f(const S* __restrict__ src, double* __restrict__ f, Grid g) {
  const ModelConst& mc = c_mc[M];
  const long long n = (long long)Model<M>::Q * g.ncell;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k / g.ncell);
    f[k] = mc.w[i] * (1.0 + to_double(src[k]));
  }
}

template <int M, class S>
__global__ void k_set_f(const double* __restrict__ f, S* __restrict__ dst, Grid g) {
  const ModelConst& mc = c_mc[M];
  const long long n = (long long)Model<M>::Q * g.ncell;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k / g.ncell);
    dst[k] = Codec<S>::enc(f[k] / mc.w[i] - 1.0);
  }
}

}  // namespace lbm

namespace lbm {

// ----------------------------------------------------------------- adjoint
// Discrete adjoint of one pull stream-collide step (exact transpose, arithmetic
// type L = FP32 or FP64).  Variables are derivatives with respect to the
// physical populations f.  With nu_n(x, j) = dL/dg^(n)_j(x) for the populations
// gathered by step n and lambda_{n+1}(x, i) = dL/dS_{n+1}(x, i) = nu_{n+1}(x + e_i, i):
//   nu_n(x, j) = (1 - omega) lambda_j + omega (alpha + beta . xi_j + gamma |xi_j|^2)
// because f^eq depends on g only through M = (rho, j, E) with dM/dg_j = (1, xi_j, |xi_j|^2)
// (the collision Jacobian has rank D + 2 beyond its diagonal).  alpha, beta,
// gamma = sum_i lambda_i d f_i^eq / dM, through f_i^eq = w_i rho P(s_i; q, t):
//   dP/ds = A1 + 2 A2 s + s^2/2 + s^3/6
//   dP/dq = Bq - s/2 - s^2/4,            Bq = -1/2 + q/4 + t (D+2-x2)/4
//   dP/dt = Bt + Ct s + Dt s^2,          Bt = (x2-D)/2 + (D+2-x2) q/4 + t (x2^2 - 2(D+2) x2 + D(D+2))/4
//                                        Ct = (x2-D-2)/2, Dt = (x2-D-4)/4
// and the chain rule from (rho, u, theta) to M:
//   d u/d rho = -u/rho, d u/d j = 1/rho, d theta/d rho = (q - D theta)/(D rho),
//   d theta/d j = -2 u/(D rho), d theta/d E = 1/(D rho).
// dL/domega of the step is sum_i lambda_i (f_i^eq - g_i) = rho Lrho - sum_i lambda_i w_i (1 + h_i).
template <class R, int D>
struct EqGrad {
  R q, t;
  __device__ __forceinline__ EqGrad(R q_, R t_) : q(q_), t(t_) {}
  __device__ __forceinline__ R Bq(R x2) const {
    return R(-0.5) + q * R(0.25) + t * (R(D + 2) - x2) * R(0.25);
  }
  __device__ __forceinline__ R Bt(R x2) const {
    return (x2 - R(D)) * R(0.5) + (R(D + 2) - x2) * q * R(0.25) +
           t * (x2 * x2 - R(2 * (D + 2)) * x2 + R(D * (D + 2))) * R(0.25);
  }
  static __device__ __forceinline__ R Ct(R x2) { return (x2 - R(D + 2)) * R(0.5); }
  static __device__ __forceinline__ R Dt(R x2) { return (x2 - R(D + 4)) * R(0.25); }
};

template <class R>
__device__ __forceinline__ void comp_add(R& s, R& c, R x) {
  if constexpr (std::is_same<R, float>::value) kahan_add(s, c, x); else s += x;
}

__device__ __forceinline__ double block_sum_128(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  return r;
}

template <int M, class S, class L, bool kFirst>
__global__ void __launch_bounds__(128)
    k_adjoint(const S* __restrict__ state, const L* __restrict__ nu_next,
              const double* __restrict__ dldrho, L* __restrict__ nu_out,
              double* __restrict__ omega_acc, Grid g, double omega) {
  using Mo = Model<M>;
  using Rt = L;
  constexpr int Q = Mo::Q, D = Mo::D, RR = Mo::R, NP = Mo::NP, G = Mo::G;
  const ModelConst& mc = c_mc[M];
  __shared__ double sh[4];

  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  const bool active = x < g.nx;
  double om_part = 0.0;
  if (active) {
    int xo[2 * RR + 1], yo[2 * RR + 1], zo[2 * RR + 1];
    sfor<0, 2 * RR + 1>([&](auto K) {
      constexpr int k = decltype(K)::value;
      xo[k] = wrapi(x - (k - RR), g.nx);
      yo[k] = wrapi(y - (k - RR), g.ny) * g.nx;
      if constexpr (D == 3) zo[k] = wrapi(z - (k - RR), g.nz) * g.nxy; else zo[k] = 0;
    });
    const size_t self = ((size_t)z * g.ny + y) * g.nx + x;
    Rt lam[Q];
    Rt l1 = Rt(0);
    if constexpr (kFirst) l1 = (Rt)dldrho[self];
    // pass 1: lambda (gathered from x + e_i), forward moments of g (gathered from x - e_i)
    Rt rs, rc = Rt(0), es = Rt(0), ec = Rt(0), jx = Rt(0), jy = Rt(0), jz = Rt(0), sg;
    {
      const Rt h0 = (Rt)Codec<S>::ld(state + self);
      lam[0] = kFirst ? l1 : nu_next[self];
      rs = gW<Rt>(mc, 0) * h0;
      sg = gW<Rt>(mc, 0) * lam[0] * (Rt(1) + h0);
    }
    sfor<0, NP>([&](auto P) {
      constexpr int p = decltype(P)::value;
      constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
      constexpr int gg = Mo::vs.grp[ip];
      constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
      const int cm = zo[ez + RR] + yo[ey + RR] + xo[ex + RR];   // x - e_ip
      const int cp = zo[RR - ez] + yo[RR - ey] + xo[RR - ex];   // x + e_ip
      const Rt hp = (Rt)Codec<S>::ld(state + (size_t)ip * g.ncell + cm);
      const Rt hm = (Rt)Codec<S>::ld(state + (size_t)im * g.ncell + cp);
      if constexpr (kFirst) {
        lam[ip] = l1;
        lam[im] = l1;
      } else {
        lam[ip] = nu_next[(size_t)ip * g.ncell + cp];
        lam[im] = nu_next[(size_t)im * g.ncell + cm];
      }
      const Rt w = gW<Rt>(mc, gg);
      const Rt tr = w * (hp + hm);
      comp_add(rs, rc, tr);
      comp_add(es, ec, gX2<Rt>(mc, gg) * tr);
      const Rt tj = w * (hp - hm);
      if constexpr (ex != 0) jx += Rt(ex) * tj;
      if constexpr (ey != 0) jy += Rt(ey) * tj;
      if constexpr (ez != 0) jz += Rt(ez) * tj;
      sg += w * (lam[ip] * (Rt(1) + hp) + lam[im] * (Rt(1) + hm));
    });
    const double rho = 1.0 + ((double)rs - (double)rc);
    const double E = (double)D + ((double)es - (double)ec);
    const double ir = 1.0 / rho;
    const double ux = mc.a * (double)jx * ir, uy = mc.a * (double)jy * ir;
    const double uz = (D == 3) ? mc.a * (double)jz * ir : 0.0;
    const double qd = ux * ux + uy * uy + uz * uz;
    const double theta = (E * ir - qd) * (1.0 / D);
    const Rt q = (Rt)qd, t = (Rt)(theta - 1.0);
    const EqCoef<Rt, D> cf(q, t);
    const EqGrad<Rt, D> gr(q, t);
    const Rt uax = (Rt)(mc.a * ux), uay = (Rt)(mc.a * uy), uaz = (Rt)(mc.a * uz);

    // pass 2: contractions with lambda
    Rt Lr = gW<Rt>(mc, 0) * lam[0] * cf.K0;
    Rt Sq = gW<Rt>(mc, 0) * lam[0] * gr.Bq(Rt(0));
    Rt St = gW<Rt>(mc, 0) * lam[0] * gr.Bt(Rt(0));
    Rt Vx = Rt(0), Vy = Rt(0), Vz = Rt(0);
    sfor<0, NP>([&](auto P) {
      constexpr int p = decltype(P)::value;
      constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
      constexpr int gg = Mo::vs.grp[ip];
      constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
      const Rt x2 = gX2<Rt>(mc, gg);
      const Rt w = gW<Rt>(mc, gg);
      Rt s = Rt(0);
      if constexpr (ex != 0) s += Rt(ex) * uax;
      if constexpr (ey != 0) s += Rt(ey) * uay;
      if constexpr (ez != 0) s += Rt(ez) * uaz;
      const Rt s2 = s * s;
      const Rt A1 = cf.A1(x2), A2 = cf.A2(x2);
      const Rt Pe = cf.A0(x2) + s2 * (A2 + s2 * Rt(1.0 / 24.0));
      const Rt Po = s * (A1 + s2 * Rt(1.0 / 6.0));
      const Rt Pse = A1 + s2 * Rt(0.5);
      const Rt Pso = s * (Rt(2) * A2 + s2 * Rt(1.0 / 6.0));
      const Rt Pqe = gr.Bq(x2) - s2 * Rt(0.25);
      const Rt Pqo = s * Rt(-0.5);
      const Rt Pte = gr.Bt(x2) + EqGrad<Rt, D>::Dt(x2) * s2;
      const Rt Pto = EqGrad<Rt, D>::Ct(x2) * s;
      const Rt ls = lam[ip] + lam[im], ld = lam[ip] - lam[im];
      Lr += w * (ls * Pe + ld * Po);
      Sq += w * (ls * Pqe + ld * Pqo);
      St += w * (ls * Pte + ld * Pto);
      const Rt v = w * (ld * Pse + ls * Pso);
      if constexpr (ex != 0) Vx += Rt(ex) * v;
      if constexpr (ey != 0) Vy += Rt(ey) * v;
      if constexpr (ez != 0) Vz += Rt(ez) * v;
    });
    // chain rule to the moments (FP64 scalars)
    const double Lux = rho * (mc.a * (double)Vx + 2.0 * ux * (double)Sq);
    const double Luy = rho * (mc.a * (double)Vy + 2.0 * uy * (double)Sq);
    const double Luz = (D == 3) ? rho * (mc.a * (double)Vz + 2.0 * uz * (double)Sq) : 0.0;
    const double Lt = rho * (double)St;
    const double iDr = ir * (1.0 / D);
    const double alpha = (double)Lr - (ux * Lux + uy * Luy + uz * Luz) * ir + Lt * (qd - D * theta) * iDr;
    const double bx = Lux * ir - 2.0 * Lt * ux * iDr;
    const double by = Luy * ir - 2.0 * Lt * uy * iDr;
    const double bz = Luz * ir - 2.0 * Lt * uz * iDr;
    const double gam = Lt * iDr;
    om_part = rho * (double)Lr - (double)sg;

    // pass 3: nu_n(x, j)
    const Rt om1 = (Rt)(1.0 - omega);
    const Rt oa = (Rt)(omega * alpha), og = (Rt)(omega * gam);
    const Rt obx = (Rt)(omega * mc.a * bx), oby = (Rt)(omega * mc.a * by),
             obz = (Rt)(omega * mc.a * bz);
    nu_out[self] = om1 * lam[0] + oa;
    sfor<0, NP>([&](auto P) {
      constexpr int p = decltype(P)::value;
      constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
      constexpr int gg = Mo::vs.grp[ip];
      constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
      const Rt ev = oa + og * gX2<Rt>(mc, gg);
      Rt od = Rt(0);
      if constexpr (ex != 0) od += Rt(ex) * obx;
      if constexpr (ey != 0) od += Rt(ey) * oby;
      if constexpr (ez != 0) od += Rt(ez) * obz;
      nu_out[(size_t)ip * g.ncell + self] = om1 * lam[ip] + (ev + od);
      nu_out[(size_t)im * g.ncell + self] = om1 * lam[im] + (ev - od);
    });
  }
  const double bsum = block_sum_128(om_part, sh);
  if (threadIdx.x == 0) {
    const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    omega_acc[b] += bsum;
  }
}

// dL/d(rho0, U0, T0): lambda_0(x, i) = nu0(x + e_i, i) contracted with the
// derivatives of f_i^eq(rho, u, theta) at the initial fields (FP64).
template <int M, class L>
__global__ void __launch_bounds__(128)
    k_grad_init(const L* __restrict__ nu0, const double* __restrict__ fields,
                double* __restrict__ d_rho, double* __restrict__ d_U, double* __restrict__ d_T,
                Grid g) {
  using Mo = Model<M>;
  constexpr int D = Mo::D, RR = Mo::R, NP = Mo::NP;
  const ModelConst& mc = c_mc[M];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  int xo[2 * RR + 1], yo[2 * RR + 1], zo[2 * RR + 1];
  sfor<0, 2 * RR + 1>([&](auto K) {
    constexpr int k = decltype(K)::value;
    xo[k] = wrapi(x - (k - RR), g.nx);
    yo[k] = wrapi(y - (k - RR), g.ny) * g.nx;
    if constexpr (D == 3) zo[k] = wrapi(z - (k - RR), g.nz) * g.nxy; else zo[k] = 0;
  });
  const size_t self = ((size_t)z * g.ny + y) * g.nx + x;
  const size_t n = (size_t)g.ncell;
  const double rho = fields[self];
  const double ux = mc.a * fields[n + self], uy = mc.a * fields[2 * n + self];
  const double uz = (D == 3) ? mc.a * fields[3 * n + self] : 0.0;
  const double theta = fields[(size_t)(D + 1) * n + self] / mc.T0;
  const double q = ux * ux + uy * uy + uz * uz, t = theta - 1.0;
  const EqCoef<double, D> cf(q, t);
  const EqGrad<double, D> gr(q, t);
  const double uax = mc.a * ux, uay = mc.a * uy, uaz = mc.a * uz;
  const double l0 = (double)nu0[self];
  double Lr = mc.W[0] * l0 * cf.K0, Sq = mc.W[0] * l0 * gr.Bq(0.0), St = mc.W[0] * l0 * gr.Bt(0.0);
  double Vx = 0, Vy = 0, Vz = 0;
  sfor<0, NP>([&](auto P) {
    constexpr int p = decltype(P)::value;
    constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
    constexpr int gg = Mo::vs.grp[ip];
    constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
    const int cm = zo[ez + RR] + yo[ey + RR] + xo[ex + RR];
    const int cp = zo[RR - ez] + yo[RR - ey] + xo[RR - ex];
    const double lp = (double)nu0[(size_t)ip * n + cp];
    const double lm = (double)nu0[(size_t)im * n + cm];
    const double x2 = mc.X2[gg], w = mc.W[gg];
    const double s = ex * uax + ey * uay + ez * uaz, s2 = s * s;
    const double A1 = cf.A1(x2), A2 = cf.A2(x2);
    const double Pe = cf.A0(x2) + s2 * (A2 + s2 / 24.0), Po = s * (A1 + s2 / 6.0);
    const double Pse = A1 + 0.5 * s2, Pso = s * (2.0 * A2 + s2 / 6.0);
    const double Pqe = gr.Bq(x2) - 0.25 * s2, Pqo = -0.5 * s;
    const double Pte = gr.Bt(x2) + EqGrad<double, D>::Dt(x2) * s2, Pto = EqGrad<double, D>::Ct(x2) * s;
    const double ls = lp + lm, ld = lp - lm;
    Lr += w * (ls * Pe + ld * Po);
    Sq += w * (ls * Pqe + ld * Pqo);
    St += w * (ls * Pte + ld * Pto);
    const double v = w * (ld * Pse + ls * Pso);
    Vx += ex * v;
    Vy += ey * v;
    Vz += ez * v;
  });
  if (d_rho) d_rho[self] = Lr;
  if (d_U) {
    d_U[self] = mc.a * rho * (mc.a * Vx + 2.0 * ux * Sq);
    d_U[n + self] = mc.a * rho * (mc.a * Vy + 2.0 * uy * Sq);
    if (D == 3) d_U[2 * n + self] = mc.a * rho * (mc.a * Vz + 2.0 * uz * Sq);
  }
  if (d_T) d_T[self] = rho * St / mc.T0;
}

// Fixed-order sum of n FP64 partials by one block of 256 threads.
static __global__ void __launch_bounds__(256) k_sum_reduce(const double* __restrict__ partials,
                                                           long long n, double* __restrict__ out) {
  double acc = 0;
  for (long long b = threadIdx.x; b < n; b += blockDim.x) acc += partials[b];
  __shared__ double sh[8];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0;
    for (int w = 0; w < 8; ++w) v += sh[w];
    *out = v;
  }
}

}  // namespace lbm

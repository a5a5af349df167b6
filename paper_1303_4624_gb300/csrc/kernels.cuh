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
// {1, -1}, written by the host with the model tables.  The paired-FP32 path adds
// and subtracts through FMAs with these factors (see xadd): the compiler cannot
// know their values, so it cannot merge a preceding paired multiply into the add.
static __constant__ float c_unit[2];

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

// Arithmetic types: double (FP64 form), float (one cell per thread) and float2 (two
// cells per thread: lane .x is one cell, lane .y the next; every operation below
// acts on each lane exactly as the float operation does, through the paired FP32
// instructions of sm_100+, so both lanes round as the scalar code would).
template <class R>
struct IsPair : std::false_type {};
template <>
struct IsPair<float2> : std::true_type {};

// A constant in the arithmetic type.
template <class R>
__device__ __forceinline__ R cst(double v) {
  if constexpr (IsPair<R>::value) return make_float2((float)v, (float)v); else return (R)v;
}
template <class R>
__device__ __forceinline__ R splat(float v) {
  if constexpr (IsPair<R>::value) return make_float2(v, v); else return (R)v;
}

template <class R>
__device__ __forceinline__ R gW(const ModelConst& mc, int g) {
  if constexpr (std::is_same<R, double>::value) return mc.W[g]; else return splat<R>(mc.Wf[g]);
}
template <class R>
__device__ __forceinline__ R gA(const ModelConst& mc) {
  if constexpr (std::is_same<R, double>::value) return mc.a; else return splat<R>(mc.af);
}
template <class R>
__device__ __forceinline__ R gX2(const ModelConst& mc, int g) {
  if constexpr (std::is_same<R, double>::value) return mc.X2[g]; else return splat<R>(mc.X2f[g]);
}

// Explicitly rounded arithmetic for the stream-collide path.  The compiler never
// fuses or reorders these (unlike a * b + c, which it may contract into an FMA
// differently in each kernel), so every kernel variant performs the identical
// operation sequence and their results agree bit for bit.
// Paired adds and subtracts are written as a * 1 + b and b * (-1) + a with the
// factors read from constant memory: measured on this GPU, a paired multiply whose
// only use is a paired add is merged into one fused multiply-add even when both are
// written with explicit round-to-nearest, which would round once where the scalar
// code rounds twice.  An FMA by a factor the compiler cannot see keeps the two
// roundings (x * 1 and b * -1 are exact), at the cost of no extra instruction.
template <class R>
__device__ __forceinline__ R xadd(R a, R b) {
  if constexpr (std::is_same<R, float>::value) return __fadd_rn(a, b);
  else if constexpr (IsPair<R>::value) return __ffma2_rn(a, make_float2(c_unit[0], c_unit[0]), b);
  else return __dadd_rn(a, b);
}
template <class R>
__device__ __forceinline__ R xsub(R a, R b) {
  if constexpr (std::is_same<R, float>::value) return __fsub_rn(a, b);
  else if constexpr (IsPair<R>::value) return __ffma2_rn(b, make_float2(c_unit[1], c_unit[1]), a);
  else return __dsub_rn(a, b);
}
template <class R>
__device__ __forceinline__ R xmul(R a, R b) {
  if constexpr (std::is_same<R, float>::value) return __fmul_rn(a, b);
  else if constexpr (IsPair<R>::value) return __fmul2_rn(a, b);
  else return __dmul_rn(a, b);
}
template <class R>
__device__ __forceinline__ R xfma(R a, R b, R c) {
  if constexpr (std::is_same<R, float>::value) return __fmaf_rn(a, b, c);
  else if constexpr (IsPair<R>::value) return __ffma2_rn(a, b, c);
  else return __fma_rn(a, b, c);
}
// -a (exact)
template <class R>
__device__ __forceinline__ R xneg(R a) {
  if constexpr (IsPair<R>::value) return make_float2(-a.x, -a.y); else return -a;
}
// 1 / a by the hardware approximation (per lane)
__device__ __forceinline__ float xrcp_approx(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ float2 xrcp_approx(float2 a) {
  return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y));
}

// Kahan compensated accumulation: the running error is kept in c (true sum ~ s - c).
template <class R>
__device__ __forceinline__ void kahan_add(R& s, R& c, R x) {
  const R y = xsub(x, c);
  const R t = xadd(s, y);
  c = xsub(xsub(t, s), y);
  s = t;
}

// Coefficients of A0, A1, A2 as functions of the group's x2 (see file header):
//   A0 - 1 = K0m1 + x2 (K1 + x2 K2),  A1 = L0 + L1 x2,  A2 = M0 + M1 x2, with
//   K0m1 = q (q/8 - 1/2) + t (t D(D+2)/8 + q (D+2)/4 - D/2)   (A0 - 1 at x2 = 0,
//          formed without the leading 1 so that P - 1 keeps the precision of the deviation)
//   K1 = t (1/2 - q/4 - t (D+2)/4),  K2 = t^2/8,
//   L0 = 1 - q/2 - t (D+2)/2,  L1 = t/2,  M0 = 1/2 - q/4 - t (D+4)/4,  M1 = t/4.
template <class R, int D>
struct EqCoef {
  R K0, K0m1, K1, K2, L0, L1, M0, M1;
  __device__ __forceinline__ EqCoef(R q, R t) {
    K0m1 = xfma(t, xfma(t, cst<R>(0.125 * D * (D + 2)), xfma(q, cst<R>(0.25 * (D + 2)), cst<R>(-0.5 * D))),
                xmul(q, xfma(q, cst<R>(0.125), cst<R>(-0.5))));
    K0 = xadd(cst<R>(1), K0m1);
    K1 = xmul(t, xfma(t, cst<R>(-0.25 * (D + 2)), xfma(q, cst<R>(-0.25), cst<R>(0.5))));
    K2 = xmul(xmul(t, t), cst<R>(0.125));
    L0 = xfma(t, cst<R>(-0.5 * (D + 2)), xfma(q, cst<R>(-0.5), cst<R>(1)));
    L1 = xmul(t, cst<R>(0.5));
    M0 = xfma(t, cst<R>(-0.25 * (D + 4)), xfma(q, cst<R>(-0.25), cst<R>(0.5)));
    M1 = xmul(t, cst<R>(0.25));
  }
  __device__ __forceinline__ R A0(R x2) const { return xfma(x2, xfma(x2, K2, K1), K0); }
  __device__ __forceinline__ R A0m1(R x2) const { return xfma(x2, xfma(x2, K2, K1), K0m1); }
  __device__ __forceinline__ R A1(R x2) const { return xfma(L1, x2, L0); }
  __device__ __forceinline__ R A2(R x2) const { return xfma(M1, x2, M0); }
};

// acc + K v for a compile-time integer K.  K = +-1 is written as an add or a
// subtract (the same rounding as the FMA by +-1): the compiler turns an FMA by a
// literal +-1 into an add anyway, and a plain paired add would then be open to the
// merge described at xadd.
template <int K, class R>
__device__ __forceinline__ R xaxpy(R v, R acc) {
  if constexpr (K == 1) return xadd(acc, v);
  else if constexpr (K == -1) return xsub(acc, v);
  else return xfma(cst<R>(K), v, acc);
}

// s = e . v for a compile-time integer lattice vector e.
template <class R, int EX, int EY, int EZ>
__device__ __forceinline__ R edot(R vx, R vy, R vz) {
  R s = cst<R>(0);
  bool first = true;
  if constexpr (EX != 0) { s = xmul(cst<R>(EX), vx); first = false; }
  if constexpr (EY != 0) { s = first ? xmul(cst<R>(EY), vy) : xaxpy<EY>(vy, s); first = false; }
  if constexpr (EZ != 0) { s = first ? xmul(cst<R>(EZ), vz) : xaxpy<EZ>(vz, s); }
  return s;
}

// ----------------------------------------------------------------- fused stream-collide
// Steps of one cell update (shared by the direct-gather and the staged kernel):
// a1 pull-gather  g_i(x) = F_i((x - e_i) mod N)         (the caller's load functor)
// a2 decode       f_i = w_i (1 + h_i), kept as h_i
// a3 moments      rho - 1 = sum w_i h_i, j = sum w_i h_i xi_i, E - D = sum w_i h_i |xi_i|^2
//                 (the rest-state moments sum w = 1, sum w xi = 0, sum w |xi|^2 = D are
//                 exact); opposite pairs are summed first; the rho and E sums are
//                 Kahan-compensated in FP32
// a4 temperature  theta - 1 = ((E - D rho) / rho - |u|^2) / D: in double-float on the
//                 FP32 pipe for the FP32, FP16 and BF16 forms (rho - 1, E - D rho and
//                 1/rho carried as hi + lo pairs; one Newton step r' = r + r (1 - rho r)
//                 refines the FP32 estimate of 1/rho), in FP64 for the FP64 form
//                 (cell_state)
// a5 equilibrium  per group A0, A1, A2; per pair the even / odd parts in s
// a6 BGK          h_i' = h_i + omega (h_i^eq - h_i) with h_i^eq = rho P_i - 1 (see
//                 half_collide for the two algebraic forms), handed to the store functor
// Partial moments of one half of the directions (rest + pairs [P0, P1) when REST).
// Every kernel forms the moments as the same two halves, first [0, NP/2) with the
// rest direction, then [NP/2, NP), combined in that order, so that the direct,
// staged and split kernels produce bitwise identical results.
template <class Rt>
struct HalfMoments {
  Rt rs, rc, es, ec, jx, jy, jz;   // Kahan sums (rs, es) with compensations (rc, ec)
};

// SHELL = false: every +/- pair's contribution enters the compensated rho and E sums.
// SHELL = true (FP16 / BF16 forms): the equal-weight deviations of one symmetry
// shell are first summed in plain FP32 (error ~ n 2^-24 |h|, far below the 2^-11
// rounding of the stored values) and each shell's total enters the compensated
// sums, so the compensation spans the five decades of weights across shells.
template <int M, class Rt, int P0, int P1, bool REST, bool SHELL, class Get>
__device__ __forceinline__ HalfMoments<Rt> half_moments(Get&& hv) {
  using Mo = Model<M>;
  const ModelConst& mc = c_mc[M];
  HalfMoments<Rt> m;
  m.rs = REST ? xmul(gW<Rt>(mc, 0), hv(std::integral_constant<int, 0>{})) : cst<Rt>(0);
  m.rc = m.es = m.ec = m.jx = m.jy = m.jz = cst<Rt>(0);
  Rt shell = cst<Rt>(0);
  sfor<P0, P1>([&](auto P) {
    constexpr int p = decltype(P)::value;
    constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
    constexpr int gg = Mo::vs.grp[ip];
    constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
    constexpr bool first = (p == P0) || (Mo::vs.grp[ip - 2] != gg);
    constexpr bool last = (p + 1 == P1) || (Mo::vs.grp[ip + 2] != gg);
    const Rt hp = hv(std::integral_constant<int, ip>{});
    const Rt hm = hv(std::integral_constant<int, im>{});
    const Rt sp = xadd(hp, hm);
    if constexpr (SHELL) {
      shell = first ? sp : xadd(shell, sp);
      if constexpr (last) {
        const Rt tr = xmul(gW<Rt>(mc, gg), shell);
        kahan_add(m.rs, m.rc, tr);
        kahan_add(m.es, m.ec, xmul(gX2<Rt>(mc, gg), tr));
      }
    } else {
      const Rt tr = xmul(gW<Rt>(mc, gg), sp);
      const Rt te = xmul(gX2<Rt>(mc, gg), tr);
      if constexpr (!std::is_same<Rt, double>::value) {
        kahan_add(m.rs, m.rc, tr);
        kahan_add(m.es, m.ec, te);
      } else {
        m.rs = xadd(m.rs, tr);
        m.es = xadd(m.es, te);
      }
    }
    const Rt tj = xmul(gW<Rt>(mc, gg), xsub(hp, hm));
    if constexpr (ex != 0) m.jx = xaxpy<ex>(tj, m.jx);
    if constexpr (ey != 0) m.jy = xaxpy<ey>(tj, m.jy);
    if constexpr (ez != 0) m.jz = xaxpy<ez>(tj, m.jz);
  });
  return m;
}

// Double-float (hi + lo) arithmetic on the FP32 pipe.  On this GPU the FP64 pipe
// issues about 1/64 of the FP32 rate (two FP64 lanes per SM per clock), so a few
// dozen FP64 operations per cell already bound a kernel below HBM speed; the
// temperature recovery and the audit sums use double-float instead.  two_sum is
// Knuth's error-free addition (s + e = a + b exactly); ff_add adds two
// double-float numbers and renormalises with Dekker's fast two-sum; the result
// keeps about 44 significant bits.
struct FF {
  float hi, lo;
};
template <class R>
__device__ __forceinline__ void two_sum(R a, R b, R& s, R& e) {
  s = xadd(a, b);
  const R bb = xsub(s, a);
  e = xadd(xsub(a, xsub(s, bb)), xsub(b, bb));
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = xadd(e, xadd(a.lo, b.lo));
  const float h = xadd(s, e);
  return {h, xsub(e, xsub(h, s))};
}
__device__ __forceinline__ double ff_to_double(FF v) { return (double)v.hi + (double)v.lo; }

// Cell state from the two halves.  theta - 1 is recovered in double-float on the
// FP32 pipe for the FP32-arithmetic forms (Rt = float: FP32, FP16 and BF16 storage)
// and in FP64 for the FP64 form (Rt = double).  The energy difference E - D rho
// cancels badly where the gas is hot and dense (behind a shock), so it is formed
// with FP64-grade precision in every form, whatever the storage rounding.
template <class Rt>
struct CellState {
  Rt q, t, uax, uay, uaz;   // |u|^2, theta - 1, a u
  Rt rho, rdev;             // rho, rho - 1
  Rt wr, wrd;               // omega rho, omega (rho - 1)
};

template <int M, class Rt>
__device__ __forceinline__ CellState<Rt> cell_state(const HalfMoments<Rt>& A,
                                                    const HalfMoments<Rt>& B, double omega) {
  constexpr int D = Model<M>::D;
  const ModelConst& mc = c_mc[M];
  CellState<Rt> c;
  if constexpr (!std::is_same<Rt, double>::value) {
    // FP32-arithmetic forms (Rt = float, or float2 for two cells): rho - 1 and
    // E - D rho as double-float (hi, lo) on the FP32 pipe
    const Rt one = cst<Rt>(1.0), Dv = cst<Rt>(D);
    Rt rd_hi, rd_lo, ed_hi, ed_lo, rho_hi, rho_lo;
    two_sum(A.rs, B.rs, rd_hi, rd_lo);
    rd_lo = xsub(rd_lo, xadd(A.rc, B.rc));
    two_sum(A.es, B.es, ed_hi, ed_lo);
    ed_lo = xsub(ed_lo, xadd(A.ec, B.ec));
    two_sum(one, rd_hi, rho_hi, rho_lo);
    rho_lo = xadd(rho_lo, rd_lo);
    const Rt rho_r = xadd(rho_hi, rho_lo);
    const Rt r0 = xrcp_approx(rho_r);
    const Rt ir = xfma(r0, xsub(xfma(xneg(rho_hi), r0, one), xmul(rho_lo, r0)), r0);
    const Rt ir_lo = xmul(ir, xsub(xfma(xneg(rho_hi), ir, one), xmul(rho_lo, ir)));
    const Rt a = gA<Rt>(mc);
    const Rt jx = xadd(A.jx, B.jx), jy = xadd(A.jy, B.jy), jz = xadd(A.jz, B.jz);
    const Rt ux = xmul(xmul(a, jx), ir), uy = xmul(xmul(a, jy), ir);
    const Rt uz = (D == 3) ? xmul(xmul(a, jz), ir) : cst<Rt>(0.0);
    c.q = xfma(ux, ux, xfma(uy, uy, xmul(uz, uz)));
    // E - D rho = ed - D rd (the product's rounding error recovered by FMA)
    const Rt ph = xmul(Dv, rd_hi);
    const Rt pl = xfma(Dv, rd_lo, xfma(Dv, rd_hi, xneg(ph)));
    Rt sh, se;
    two_sum(ed_hi, xneg(ph), sh, se);
    const Rt dl = xadd(se, xsub(ed_lo, pl));
    const Rt dh = xadd(sh, dl);
    const Rt dlo = xsub(dl, xsub(dh, sh));
    // (E - D rho) / rho as double-float, then theta - 1 = (that - |u|^2) / D
    const Rt xh = xmul(dh, ir);
    const Rt xl = xfma(dh, ir_lo, xfma(dlo, ir, xfma(dh, ir, xneg(xh))));
    // v = x - q as double-float; t = v / D rounded to nearest: a product with the
    // FP32-rounded 1/D alone is biased (it rounds 1/3 up), which would heat or cool
    // every cell by a fixed fraction of an ulp per step; one FMA residual step
    // removes it
    Rt vh, ve;
    two_sum(xh, xneg(c.q), vh, ve);
    const Rt vl = xadd(ve, xl);
    const Rt third = cst<Rt>(1.0 / D);
    const Rt y = xmul(xadd(vh, vl), third);
    c.t = xfma(xadd(xfma(xneg(Dv), y, vh), vl), third, y);
    c.uax = xmul(a, ux);
    c.uay = xmul(a, uy);
    c.uaz = xmul(a, uz);
    c.rho = rho_r;
    c.rdev = xadd(rd_hi, rd_lo);
    const Rt om = cst<Rt>(omega);
    c.wr = xmul(om, rho_r);
    c.wrd = xmul(om, c.rdev);
    return c;
  } else {
    // FP64 form: everything in FP64
    const double rd = xadd(A.rs, B.rs);
    const double ed = xadd(A.es, B.es);
    const double jx = xadd(A.jx, B.jx), jy = xadd(A.jy, B.jy), jz = xadd(A.jz, B.jz);
    const double rho = xadd(1.0, rd);
    const double ir = 1.0 / rho;
    const double a = gA<double>(mc);
    const double ux = xmul(xmul(a, jx), ir), uy = xmul(xmul(a, jy), ir);
    const double uz = (D == 3) ? xmul(xmul(a, jz), ir) : 0.0;
    c.q = xfma(ux, ux, xfma(uy, uy, xmul(uz, uz)));
    // theta - 1 = ((E - D rho) / rho - |u|^2) / D
    c.t = xmul(xfma(xfma(-(double)D, rd, ed), ir, -c.q), 1.0 / D);
    c.uax = xmul(a, ux);
    c.uay = xmul(a, uy);
    c.uaz = xmul(a, uz);
    c.rho = rho;
    c.rdev = rd;
    c.wr = xmul(omega, rho);
    c.wrd = xmul(omega, rd);
    return c;
  }
}

// Equilibrium + BGK of pairs [P0, P1) (and the rest direction when REST), with
// h_i^eq = (rho - 1) + rho (P_i - 1):
//   EXACT = true:  h_i' = h_i + omega (h_i^eq - h_i)   (FP32 / FP64 forms).  The
//                  equilibrium is an exact fixed point whatever the rounding of omega;
//                  with (1 - omega) h + omega h^eq the two rounded factors need not
//                  sum to one and a uniform region drifts by their difference every
//                  step (about 1e-5 in rho after 200 steps at omega = 1.8 in FP32).
//   EXACT = false: h_i' = (1 - omega) h_i + omega (rho - 1) + omega rho (P_i - 1)
//                  (FP16 / BF16 forms: two instructions fewer per pair; the drift is
//                  far below the storage rounding).
template <int M, class Rt, int P0, int P1, bool REST, bool EXACT, class Get, class Store>
__device__ __forceinline__ void half_collide(const CellState<Rt>& c, double omega, Get&& hv,
                                             Store&& st) {
  using Mo = Model<M>;
  constexpr int D = Mo::D;
  const ModelConst& mc = c_mc[M];
  const EqCoef<Rt, D> cf(c.q, c.t);
  const Rt om = cst<Rt>(omega);
  const Rt om1 = cst<Rt>(1.0 - omega);
  const Rt wr24 = xmul(c.wr, cst<Rt>(1.0 / 24.0)), wr6 = xmul(c.wr, cst<Rt>(1.0 / 6.0));
  if constexpr (REST) {
    const Rt h0 = hv(std::integral_constant<int, 0>{});
    if constexpr (EXACT)
      st(std::integral_constant<int, 0>{}, xfma(om, xsub(xfma(c.rho, cf.K0m1, c.rdev), h0), h0));
    else
      st(std::integral_constant<int, 0>{}, xfma(om1, h0, xfma(c.wr, cf.K0m1, c.wrd)));
  }
  sfor<P0, P1>([&](auto P) {
    constexpr int p = decltype(P)::value;
    constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
    constexpr int gg = Mo::vs.grp[ip];
    constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
    const Rt x2 = gX2<Rt>(mc, gg);
    const Rt s = edot<Rt, ex, ey, ez>(c.uax, c.uay, c.uaz);
    const Rt s2 = xmul(s, s);
    const Rt hp = hv(std::integral_constant<int, ip>{});
    const Rt hm = hv(std::integral_constant<int, im>{});
    if constexpr (EXACT) {
      const Rt ev = xfma(s2, xfma(s2, cst<Rt>(1.0 / 24.0), cf.A2(x2)), cf.A0m1(x2));
      const Rt od = xmul(s, xfma(s2, cst<Rt>(1.0 / 6.0), cf.A1(x2)));
      const Rt be = xfma(c.rho, ev, c.rdev);      // even part of h^eq
      const Rt bo = xmul(c.rho, od);              // odd part of h^eq
      st(std::integral_constant<int, ip>{}, xfma(om, xsub(xadd(be, bo), hp), hp));
      st(std::integral_constant<int, im>{}, xfma(om, xsub(xsub(be, bo), hm), hm));
    } else {
      // omega rho folded into the shell's coefficients: base = omega h^eq's even
      // part, wod = its odd part
      const Rt base = xfma(s2, xfma(s2, wr24, xmul(c.wr, cf.A2(x2))), xfma(c.wr, cf.A0m1(x2), c.wrd));
      const Rt wod = xmul(s, xfma(s2, wr6, xmul(c.wr, cf.A1(x2))));
      st(std::integral_constant<int, ip>{}, xfma(om1, hp, xadd(base, wod)));
      st(std::integral_constant<int, im>{}, xfma(om1, hm, xsub(base, wod)));
    }
  });
}

// Arithmetic options per storage form: FP32 / FP64 storage keep per-pair Kahan sums
// and the exact-fixed-point relaxation; FP16 / BF16 storage use per-shell
// compensation and the two-term relaxation (see half_moments / half_collide).
template <class S>
struct FormOpts {
  static constexpr bool kShell = sizeof(S) == 2;
  static constexpr bool kExact = sizeof(S) >= 4;
};

// a3 - a6 of one cell (Rt = float / double) or of two cells (Rt = float2, one per
// lane) from its gathered, decoded populations: hv(I) returns direction I's value,
// st(I, v) stores direction I's result.  The arithmetic options follow the storage
// form S.
// hm(I) serves the moments (a3), hr(I) the relaxation (a6): both return the same
// values (the pair kernel's relaxation getter adds an ordering dependency).
template <int M, class S, class Rt, class GetM, class GetR, class Store>
__device__ __forceinline__ void cell_collide_with2(GetM&& hm, GetR&& hr, double omega,
                                                   Store&& st) {
  using Mo = Model<M>;
  constexpr int NP = Mo::NP, NH = NP / 2;
  constexpr bool SH = FormOpts<S>::kShell, EX = FormOpts<S>::kExact;
  // a3, a4
  const HalfMoments<Rt> A = half_moments<M, Rt, 0, NH, true, SH>(hm);
  const HalfMoments<Rt> B = half_moments<M, Rt, NH, NP, false, SH>(hm);
  const CellState<Rt> c = cell_state<M, Rt>(A, B, omega);
  // a5, a6
  half_collide<M, Rt, 0, NH, true, EX>(c, omega, hr, st);
  half_collide<M, Rt, NH, NP, false, EX>(c, omega, hr, st);
}
template <int M, class S, class Rt, class Get, class Store>
__device__ __forceinline__ void cell_collide_with(Get&& hv, double omega, Store&& st) {
  cell_collide_with2<M, S, Rt>(hv, hv, omega, st);
}

// a3 - a6 of one cell from its gathered, decoded populations h[Q].
template <int M, class S, class Store>
__device__ __forceinline__ void cell_collide(const typename Codec<S>::R (&h)[Model<M>::Q],
                                             double omega, Store&& st) {
  using Rt = typename Codec<S>::R;
  cell_collide_with<M, S, Rt>([&](auto I) { return h[decltype(I)::value]; }, omega, st);
}

// One cell update: a1 + a2 through the load functor (all Q loads issued before any
// use), then cell_collide.
template <int M, class S, class Load, class Store>
__device__ __forceinline__ void cell_update(Load&& ld, double omega, Store&& st) {
  using Rt = typename Codec<S>::R;
  Rt h[Model<M>::Q];
  sfor<0, Model<M>::Q>([&](auto I) { h[decltype(I)::value] = ld(I); });
  cell_collide<M, S>(h, omega, st);
}

// Periodic index for -n <= v < 2n (one correction each way).
__device__ __forceinline__ int wrap1(int v, int n) {
  v += (v < 0) ? n : 0;
  v -= (v >= n) ? n : 0;
  return v;
}

// Row offsets of the periodic neighbours x - k, y - k, z - k for k in [-R, R]
// (index k + R): one correction each way when every extent is at least the reach,
// a true modulo otherwise (grids smaller than the reach are legal).
template <int D, int RR>
__device__ __forceinline__ void neighbour_offsets(int x, int y, int z, int nx, int ny, int nz,
                                                  int nxy, int* xo, int* yo, int* zo) {
  if (nx >= RR && ny >= RR && (D == 2 || nz >= RR)) {
    sfor<0, 2 * RR + 1>([&](auto K) {
      constexpr int k = decltype(K)::value;
      xo[k] = wrap1(x - (k - RR), nx);
      yo[k] = wrap1(y - (k - RR), ny) * nx;
      if constexpr (D == 3) zo[k] = wrap1(z - (k - RR), nz) * nxy; else zo[k] = 0;
    });
  } else {
    sfor<0, 2 * RR + 1>([&](auto K) {
      constexpr int k = decltype(K)::value;
      xo[k] = wrapi(x - (k - RR), nx);
      yo[k] = wrapi(y - (k - RR), ny) * nx;
      if constexpr (D == 3) zo[k] = wrapi(z - (k - RR), nz) * nxy; else zo[k] = 0;
    });
  }
}

// Direct-gather kernel: one thread per cell, x fastest across the block,
// blockIdx.y / z give the row; Q loads per thread straight from HBM / L2.
// LBM_DIRECT_MINB: resident 128-thread blocks per SM the D3Q95 register budget is
// cut for (128 registers at 4: 16 warps per SM; measured best for the FP32 and
// FP16 forms).  D2Q33's 33 populations fit fewer registers without spilling, and
// more resident warps pay: 8 blocks (64 registers) for FP32, 6 (80 registers) for
// the 16-bit forms (4096 x 2048: +4.6 % and +12.8 % over 4 blocks).  The FP64
// form keeps 2 (D3Q95's 95 doubles need 190 registers).
#ifndef LBM_DIRECT_MINB
#define LBM_DIRECT_MINB 4
#endif
template <int M, class S>
struct DirectMinBlocks {
  static constexpr int value = std::is_same<S, double>::value
                                   ? 2
                                   : (Model<M>::Q == 33 ? (sizeof(S) == 4 ? 8 : 6) : LBM_DIRECT_MINB);
};
// 4-byte global -> shared copy (cp.async, L1-allocating) and the wait for all of
// this thread's outstanding copies.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
// Close the group of this thread's cp.async copies issued since the last commit, and
// wait until at most N of its committed groups are still in flight.
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Launched with programmatic stream serialization: the next step's grid may be
// scheduled while this one drains; griddepcontrol.wait holds every thread until
// the previous grid has completed and its writes are visible (a no-op when the
// launch has no programmatic dependency).
__device__ __forceinline__ void wait_prior_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_next_grid() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// REV: walk the blocks in reverse order (the block scheduler issues blocks in
// increasing index order), so that a step following a forward step starts on the
// cells written last, still resident in L2.
// NARROW (FP32 D3Q95, when every element index of a state copy, Q ncell, fits 32
// bits): each population's element index i ncell + row offset + column is formed
// in 32 bits and scaled into the 64-bit base in one instruction, instead of adding
// 64-bit offsets per population: 2404 instead of 2710 instructions per cell
// (measured), which lifts the HBM-bound FP32 kernel from 0.966 to 1.00 of the
// measured copy bandwidth.  The 16-bit forms, bound by instruction issue, measured
// slower with it (the index multiply-adds compete with the FP32 arithmetic for the
// FMA pipe), and keep the 64-bit form.
template <int M, class S>
struct DirectNarrow {
  static constexpr bool value = M == 1 && std::is_same<S, float>::value;
};
template <int M, class S, bool REV, bool NARROW>
__global__ void __launch_bounds__(128, DirectMinBlocks<M, S>::value)
    k_stream_collide(const S* __restrict__ src, S* __restrict__ dst, Grid g, double omega) {
  using Mo = Model<M>;
  constexpr int D = Mo::D, RR = Mo::R;
  wait_prior_grid();
  allow_next_grid();
  const int bx = REV ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
  const int x = bx * blockDim.x + threadIdx.x;
  if (x >= g.nx) return;
  const int y = REV ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
  const int z = REV ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z;
  int xo[2 * RR + 1], yo[2 * RR + 1], zo[2 * RR + 1];
  neighbour_offsets<D, RR>(x, y, z, g.nx, g.ny, g.nz, g.nxy, xo, yo, zo);
  if constexpr (NARROW) {
    const uint32_t nc = (uint32_t)g.ncell;
    const uint32_t self = (uint32_t)((z * g.ny + y) * g.nx + x);
    cell_update<M, S>(
        [&](auto I) {
          constexpr int i = decltype(I)::value;
          constexpr int ex = Mo::vs.e[i][0], ey = Mo::vs.e[i][1], ez = Mo::vs.e[i][2];
          const uint32_t e = (uint32_t)i * nc + (uint32_t)(zo[ez + RR] + yo[ey + RR]) +
                             (uint32_t)xo[ex + RR];
          return Codec<S>::ld(src + e);
        },
        omega,
        [&](auto I, typename Codec<S>::R v) {
          Codec<S>::st(dst + ((uint32_t)decltype(I)::value * nc + self), v);
        });
  } else {
    const size_t self = ((size_t)z * g.ny + y) * g.nx + x;
    cell_update<M, S>(
        [&](auto I) {
          constexpr int i = decltype(I)::value;
          constexpr int ex = Mo::vs.e[i][0], ey = Mo::vs.e[i][1], ez = Mo::vs.e[i][2];
          const int cell = zo[ez + RR] + yo[ey + RR] + xo[ex + RR];
          return Codec<S>::ld(src + (size_t)i * (size_t)g.ncell + cell);
        },
        omega,
        [&](auto I, typename Codec<S>::R v) {
          Codec<S>::st(dst + (size_t)decltype(I)::value * (size_t)g.ncell + self, v);
        });
  }
}

// ----------------------------------------------------------------- split kernel
// Warp-pair kernel: the Q directions of each cell are split between two warps that
// handle the same 32 cells (warp 2k: the rest direction and pairs [0, NP/2), warp
// 2k+1: pairs [NP/2, NP)), which halves the registers a thread holds and doubles
// the warps an SM keeps resident.  Each warp forms the partial moments of its
// half; the two halves are exchanged through shared memory behind a named
// 64-thread barrier and combined in a fixed order (first half, then second), so
// both warps hold identical moments; each then evaluates the equilibrium and the
// BGK update for its own directions.  Same arithmetic per direction as cell_update.
#ifndef LBM_SPLIT_MINB
#define LBM_SPLIT_MINB 3
#endif
constexpr int kSplitThreads = 256;                 // 4 warp pairs = 128 cells per block

__device__ __forceinline__ void pair_barrier(int id) {
  asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

template <int M, class S, int HALF, class Load, class Store>
__device__ __forceinline__ void half_update(Load&& ld, double omega, Store&& st,
                                            float (*xch)[2][8][32], int pair, int lane) {
  using Mo = Model<M>;
  using Rt = typename Codec<S>::R;
  static_assert(std::is_same<Rt, float>::value, "split kernel is for the FP32-arithmetic forms");
  constexpr int NP = Mo::NP, NH = NP / 2;
  constexpr int P0 = HALF == 0 ? 0 : NH, P1 = HALF == 0 ? NH : NP;
  constexpr int I0 = HALF == 0 ? 0 : 1 + 2 * NH;   // first direction index of this half
  constexpr int NV = 1 + 2 * P1 - I0;               // directions held by this half
  Rt h[NV];
  sfor<I0, 1 + 2 * P1>([&](auto I) { h[decltype(I)::value - I0] = ld(I); });
  auto hv = [&](auto I) { return h[decltype(I)::value - I0]; };
  const HalfMoments<Rt> mine = half_moments<M, Rt, P0, P1, HALF == 0, FormOpts<S>::kShell>(hv);
  // exchange the partial moments of the two halves
  float* w = &xch[pair][HALF][0][lane];
  w[0] = mine.rs; w[32] = mine.rc; w[64] = mine.es; w[96] = mine.ec;
  w[128] = mine.jx; w[160] = mine.jy; w[192] = mine.jz;
  pair_barrier(1 + pair);
  HalfMoments<Rt> A, B;
  const float* a = &xch[pair][0][0][lane];
  const float* b = &xch[pair][1][0][lane];
  A.rs = a[0]; A.rc = a[32]; A.es = a[64]; A.ec = a[96]; A.jx = a[128]; A.jy = a[160]; A.jz = a[192];
  B.rs = b[0]; B.rc = b[32]; B.es = b[64]; B.ec = b[96]; B.jx = b[128]; B.jy = b[160]; B.jz = b[192];
  const CellState<Rt> c = cell_state<M, Rt>(A, B, omega);
  half_collide<M, Rt, P0, P1, HALF == 0, FormOpts<S>::kExact>(c, omega, hv, st);
}

template <int M, class S>
__global__ void __launch_bounds__(kSplitThreads, LBM_SPLIT_MINB)
    k_stream_collide_split(const S* __restrict__ src, S* __restrict__ dst, Grid g, double omega) {
  using Mo = Model<M>;
  constexpr int D = Mo::D, RR = Mo::R;
  __shared__ float xch[kSplitThreads / 64][2][8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = warp >> 1, half = warp & 1;
  const int xw = blockIdx.x * (kSplitThreads / 2) + pair * 32;   // first cell of the pair
  if (xw >= g.nx) return;                                        // the whole pair is idle
  const int x = xw + lane;
  const bool active = x < g.nx;
  const int y = blockIdx.y, z = blockIdx.z;
  int xo[2 * RR + 1], yo[2 * RR + 1], zo[2 * RR + 1];
  const int xa = active ? x : xw;
  neighbour_offsets<D, RR>(xa, y, z, g.nx, g.ny, g.nz, g.nxy, xo, yo, zo);
  const size_t self = ((size_t)z * g.ny + y) * g.nx + xa;
  auto ld = [&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ex = Mo::vs.e[i][0], ey = Mo::vs.e[i][1], ez = Mo::vs.e[i][2];
    const int cell = zo[ez + RR] + yo[ey + RR] + xo[ex + RR];
    return Codec<S>::ld(src + (size_t)i * (size_t)g.ncell + cell);
  };
  auto st = [&](auto I, float v) {
    if (active) Codec<S>::st(dst + (size_t)decltype(I)::value * (size_t)g.ncell + self, v);
  };
  if (half == 0)
    half_update<M, S, 0>(ld, omega, st, xch, pair, lane);
  else
    half_update<M, S, 1>(ld, omega, st, xch, pair, lane);
}

// ----------------------------------------------------------------- equilibrium init
// h_i = rho P_i(u, theta) - 1 for the fields rho, U (lattice), T (lattice) of each cell,
// rounded once to the storage type.  FP64 for the FP64 form; double-float on the FP32
// pipe for the FP32, FP16 and BF16 forms, whose ~48 significant bits round to the
// same value as FP64 except within 2^-44 relative of a rounding boundary.  The five
// FP64 inputs are split into double-float once and everything else runs on the FP32
// pipe: on this GPU the FP64 pipe issues 1/64 of the FP32 rate, and the FP64 form of
// the 95 direction polynomials is bound by it (~38 ms for 33.5 M cells; with the
// shell coefficients alone in FP64, ~13 ms; all in double-float, 6.7 ms).

// double-float helpers (FMA products, Knuth / Dekker sums; see ff_add)
__device__ __forceinline__ FF ff_from(double d) {
  const float hi = __double2float_rn(d);
  return {hi, __double2float_rn(d - (double)hi)};
}
__device__ __forceinline__ FF ff_renorm(float p, float e) {
  const float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_renorm(p, e);
}
// a times an FP32 constant c
__device__ __forceinline__ FF ff_mulc(FF a, float c) {
  const float p = __fmul_rn(c, a.hi);
  float e = __fmaf_rn(c, a.hi, -p);
  e = __fmaf_rn(c, a.lo, e);
  return ff_renorm(p, e);
}
template <int K>
__device__ __forceinline__ FF ff_scale(FF a) {
  if constexpr (K == 1) return a;
  else if constexpr (K == -1) return {-a.hi, -a.lo};
  else return ff_mulc(a, (float)K);
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ FF ff_const(float c) { return {c, 0.f}; }

// hi + lo rounded once to the storage type.  FP32: one add.  FP16 / BF16: round hi,
// unless hi is exactly halfway between two neighbours of the 16-bit format (FP32
// holds those midpoints exactly), where the sign of lo decides; since hi is hi + lo
// rounded to FP32, no other case can put hi and hi + lo on opposite sides of a
// midpoint.
template <class S>
__device__ __forceinline__ S ff_round(FF v);
template <>
__device__ __forceinline__ float ff_round<float>(FF v) {
  return __fadd_rn(v.hi, v.lo);
}
template <>
__device__ __forceinline__ __half ff_round<__half>(FF v) {
  const __half a = __float2half_rd(v.hi), b = __float2half_ru(v.hi);
  if (v.lo != 0.f && __half_as_ushort(a) != __half_as_ushort(b) &&
      v.hi == 0.5f * (__half2float(a) + __half2float(b)))
    return v.lo > 0.f ? b : a;
  return __float2half_rn(v.hi);
}
template <>
__device__ __forceinline__ __nv_bfloat16 ff_round<__nv_bfloat16>(FF v) {
  const __nv_bfloat16 a = __float2bfloat16_rd(v.hi), b = __float2bfloat16_ru(v.hi);
  if (v.lo != 0.f && __bfloat16_as_ushort(a) != __bfloat16_as_ushort(b) &&
      v.hi == 0.5f * (__bfloat162float(a) + __bfloat162float(b)))
    return v.lo > 0.f ? b : a;
  return __float2bfloat16_rn(v.hi);
}

// s = e . (a u) as double-float for a compile-time lattice vector e
template <int EX, int EY, int EZ>
__device__ __forceinline__ FF ff_edot(FF vx, FF vy, FF vz) {
  FF s = {0.f, 0.f};
  bool first = true;
  if constexpr (EX != 0) { s = ff_scale<EX>(vx); first = false; }
  if constexpr (EY != 0) { s = first ? ff_scale<EY>(vy) : ff_add(s, ff_scale<EY>(vy)); first = false; }
  if constexpr (EZ != 0) { s = first ? ff_scale<EZ>(vz) : ff_add(s, ff_scale<EZ>(vz)); }
  return s;
}

// Cells [begin, end) of the grid (U and the populations strided by g.ncell).
template <int M, class S>
__global__ void __launch_bounds__(256)
    k_init(const double* __restrict__ rho, const double* __restrict__ U,
           const double* __restrict__ T, S* __restrict__ dst, Grid g, long long begin,
           long long end) {
  using Mo = Model<M>;
  constexpr int D = Mo::D, NP = Mo::NP;
  const ModelConst& mc = c_mc[M];
  const long long idx = begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= end) return;
  if constexpr (!std::is_same<S, double>::value) {
    // the coefficients of EqCoef (see there), with rho folded in per shell:
    //   h_i = (rho - 1) + rho (A0 - 1) + rho A2 s^2 + rho s^4 / 24 + s (rho A1 + rho s^2 / 6)
    constexpr double kSixth = 1.0 / 6.0, kTwentyFourth = 1.0 / 24.0;
    constexpr float c6h = (float)kSixth, c6l = (float)(kSixth - (double)c6h);
    constexpr float c24h = (float)kTwentyFourth, c24l = (float)(kTwentyFourth - (double)c24h);
    const FF a = {mc.af, mc.alo};
    const FF r = ff_from(rho[idx]);
    const FF ux = ff_mul(ff_from(U[idx]), a);
    const FF uy = ff_mul(ff_from(U[g.ncell + idx]), a);
    const FF uz = (D == 3) ? ff_mul(ff_from(U[2 * g.ncell + idx]), a) : FF{0.f, 0.f};
    const FF q = ff_add(ff_add(ff_mul(ux, ux), ff_mul(uy, uy)), ff_mul(uz, uz));
    const FF t = ff_add(ff_mul(ff_from(T[idx]), FF{mc.iT0f, mc.iT0lo}), ff_const(-1.f));
    const FF K0m1 =
        ff_add(ff_mul(t, ff_add(ff_add(ff_mulc(t, 0.125f * D * (D + 2)), ff_mulc(q, 0.25f * (D + 2))),
                                ff_const(-0.5f * D))),
               ff_mul(q, ff_add(ff_mulc(q, 0.125f), ff_const(-0.5f))));
    const FF K1 = ff_mul(t, ff_add(ff_add(ff_mulc(t, -0.25f * (D + 2)), ff_mulc(q, -0.25f)),
                                   ff_const(0.5f)));
    const FF K2 = ff_mulc(ff_mul(t, t), 0.125f);
    const FF L0 = ff_add(ff_add(ff_mulc(t, -0.5f * (D + 2)), ff_mulc(q, -0.5f)), ff_const(1.f));
    const FF L1 = ff_mulc(t, 0.5f);
    const FF M0 = ff_add(ff_add(ff_mulc(t, -0.25f * (D + 4)), ff_mulc(q, -0.25f)), ff_const(0.5f));
    const FF M1 = ff_mulc(t, 0.25f);
    const FF rm1 = ff_add(r, ff_const(-1.f));
    const FF vx = ff_mul(ux, a), vy = ff_mul(uy, a), vz = ff_mul(uz, a);
    const FF r6 = ff_mul(r, FF{c6h, c6l}), r24 = ff_mul(r, FF{c24h, c24l});
    {
      const FF h0 = ff_add(rm1, ff_mul(r, K0m1));
      dst[idx] = ff_round<S>(h0);   // one rounding to the storage type
    }
    FF R0 = {0.f, 0.f}, R1 = R0, R2 = R0;
    sfor<0, NP>([&](auto P) {
      constexpr int p = decltype(P)::value;
      constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
      constexpr int gg = Mo::vs.grp[ip];
      constexpr bool first = (p == 0) || (Mo::vs.grp[ip - 2] != gg);
      constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
      if constexpr (first) {   // the shell's coefficients, once per shell
        const FF x2 = {mc.X2f[gg], mc.X2lo[gg]};
        const FF A0m1 = ff_add(K0m1, ff_mul(x2, ff_add(K1, ff_mul(x2, K2))));
        R0 = ff_add(rm1, ff_mul(r, A0m1));
        R1 = ff_mul(r, ff_add(L0, ff_mul(L1, x2)));
        R2 = ff_mul(r, ff_add(M0, ff_mul(M1, x2)));
      }
      const FF s = ff_edot<ex, ey, ez>(vx, vy, vz);
      const FF s2 = ff_mul(s, s);
      const FF ev = ff_add(R0, ff_mul(s2, ff_add(R2, ff_mul(s2, r24))));
      const FF od = ff_mul(s, ff_add(R1, ff_mul(s2, r6)));
      const FF hp = ff_add(ev, od);
      const FF hm = ff_add(ev, ff_neg(od));
      dst[(size_t)ip * g.ncell + idx] = ff_round<S>(hp);
      dst[(size_t)im * g.ncell + idx] = ff_round<S>(hm);
    });
    return;
  }
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

// ----------------------------------------------------------------- moments + audit
// Per cell rho = sum f, rho U = sum f e, D rho T = sum f |e|^2 - rho |U|^2 (lattice
// units), f_i = w_i (1 + h_i), written as FP64.  Each block also writes 8 FP64 audit
// partials: mass, momentum (3), energy, min f/w, non-finite count, cells.  The FP64
// form sums in FP64 (k_moments below); the other forms use moments_fp32_forms.

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ----------------------------------------------------------------- moments, FP32 forms
// Resident 256-thread blocks per SM the FP32-form moments kernel is register-capped
// for (64 registers a thread at 4; measured best among 2 to 6).
#ifndef LBM_MOM_MINB
#define LBM_MOM_MINB 4
#endif

// Moments of the FP32 / FP16 / BF16 forms, one thread per cell: the collision's own
// compensated sums (deviation form, +/- pairs first; rho - 1 and E - D as
// double-float, j in FP32), then
//   rho = 1 + rd,  U = j / rho,  T = T0 (1 + ((ed - D rd) / rho - |U|^2 / T0) / D)
// in FP32 (rho as double-float), written as FP64.  The audit terms of the 256
// cells of a block are summed in double-float per warp and in FP64 across warps:
//   mass = n + sum rd,  momentum = sum j,  energy = T0 (D n + sum ed) / 2
// (rest-state moments: sum w = 1, sum w xi = 0, sum w |xi|^2 = D).
template <int M, class S>
__device__ __forceinline__ void moments_fp32_forms(const S* __restrict__ src, const Grid& g,
                                                   long long idx, long long end, long long block,
                                                   double* __restrict__ rho_out,
                                                   double* __restrict__ U_out,
                                                   double* __restrict__ T_out,
                                                   double* __restrict__ partials) {
  using Mo = Model<M>;
  constexpr int D = Mo::D, Q = Mo::Q, NH = Mo::NP / 2;
  constexpr bool SH = sizeof(S) == 2;
  const ModelConst& mc = c_mc[M];
  FF srd = {0.f, 0.f}, sed = {0.f, 0.f}, sjx = {0.f, 0.f}, sjy = {0.f, 0.f}, sjz = {0.f, 0.f};
  float hmin = 3.0e38f, bad = 0.f, cnt = 0.f;
  if (idx < end) {
    auto hv = [&](auto I) {
      const float v = Codec<S>::ld(src + (size_t)decltype(I)::value * (size_t)g.ncell + idx);
      hmin = fminf(hmin, v);
      return v;
    };
    const HalfMoments<float> A = half_moments<M, float, 0, NH, true, SH>(hv);
    const HalfMoments<float> B = half_moments<M, float, NH, Mo::NP, false, SH>(hv);
    // rs - rc carries the compensated sum of each half; combine the halves exactly
    two_sum(A.rs, B.rs, srd.hi, srd.lo);
    srd.lo = xsub(srd.lo, xadd(A.rc, B.rc));
    two_sum(A.es, B.es, sed.hi, sed.lo);
    sed.lo = xsub(sed.lo, xadd(A.ec, B.ec));
    sjx.hi = xadd(A.jx, B.jx);
    sjy.hi = xadd(A.jy, B.jy);
    sjz.hi = (D == 3) ? xadd(A.jz, B.jz) : 0.f;
    FF rho;
    two_sum(1.0f, srd.hi, rho.hi, rho.lo);
    rho.lo = xadd(rho.lo, srd.lo);
    const float r0 = __fdividef(1.0f, rho.hi);
    const float ir = xfma(r0, xfma(-rho.hi, r0, 1.0f), r0);   // one Newton step for 1/rho
    const float Ux = xmul(sjx.hi, ir), Uy = xmul(sjy.hi, ir), Uz = xmul(sjz.hi, ir);
    const float U2 = xfma(Ux, Ux, xfma(Uy, Uy, xmul(Uz, Uz)));
    const float T0f = mc.T0f;
    const float dE = xadd(xfma(-(float)D, srd.hi, sed.hi), xfma(-(float)D, srd.lo, sed.lo));
    const float t = xmul(xsub(xmul(dE, ir), xmul(U2, mc.iT0f)), cst<float>(1.0 / D));
    if (rho_out) rho_out[idx] = ff_to_double(rho);
    if (U_out) {
      U_out[idx] = (double)Ux;
      U_out[g.ncell + idx] = (double)Uy;
      if (D == 3) U_out[2 * g.ncell + idx] = (double)Uz;
    }
    if (T_out) T_out[idx] = (double)xfma(T0f, t, T0f);
    if (!isfinite(srd.hi) || !isfinite(sed.hi)) {
      // a NaN or Inf population poisons both sums: count them one by one
      for (int i = 0; i < Q; ++i)
        if (!isfinite((float)Codec<S>::ld(src + (size_t)i * (size_t)g.ncell + idx))) bad = xadd(bad, 1.0f);
    }
    cnt = 1.f;
  }
  // Block sums: every thread's terms go to shared memory and warp w reduces audit
  // slot w over the block's cells (lane l takes cells l, l + 32, ..., then a
  // shuffle tree), double-float for the sums, in a fixed order (deterministic).
  constexpr int NT = kMomentThreads;
  static_assert(NT / 32 == kAuditSlots, "one warp per audit slot");
  __shared__ float shv[2 * kAuditSlots][NT];   // slot k: hi in row 2k, lo in row 2k + 1
  __shared__ FF res[kAuditSlots];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const FF terms[kAuditSlots] = {srd, sjx, sjy, sjz, sed, {hmin, 0.f}, {bad, 0.f}, {cnt, 0.f}};
#pragma unroll
  for (int k = 0; k < kAuditSlots; ++k) {
    shv[2 * k][tid] = terms[k].hi;
    shv[2 * k + 1][tid] = terms[k].lo;
  }
  __syncthreads();
  const bool is_min = wid == 5;
  FF v = {shv[2 * wid][lane], shv[2 * wid + 1][lane]};
  for (int c = lane + 32; c < NT; c += 32) {
    const FF w = {shv[2 * wid][c], shv[2 * wid + 1][c]};
    if (is_min) v.hi = fminf(v.hi, w.hi);
    else v = ff_add(v, w);
  }
  for (int o = 16; o > 0; o >>= 1) {
    FF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    if (is_min) v.hi = fminf(v.hi, w.hi);
    else v = ff_add(v, w);
  }
  if (lane == 0) res[wid] = v;
  __syncthreads();
  if (tid < kAuditSlots) {
    const int k = tid;
    const float n = res[7].hi;                                   // exact: at most 256
    double d = ff_to_double(res[k]);
    if (k == 0) d += (double)n;                                  // mass = n + sum (rho - 1)
    if (k == 4) d = 0.5 * mc.T0 * ((double)D * (double)n + d);   // energy
    if (k == 5) d = (n > 0.f) ? 1.0 + d : 1e300;                 // min f / w over the block
    partials[(size_t)block * kAuditSlots + k] = d;
  }
}

template <class S>
struct MomMinBlocks {
  static constexpr int value = std::is_same<S, double>::value ? 1 : LBM_MOM_MINB;
};
// Blocks block0, block0 + 1, ... of kMomentThreads cells each, cells below end (the
// audit partials of block b go to slot b, so a launch over part of the grid writes
// the same partials as the whole-grid launch writes for those blocks).
template <int M, class S>
__global__ void __launch_bounds__(kMomentThreads, MomMinBlocks<S>::value)
    k_moments(const S* __restrict__ src, Grid g, double* __restrict__ rho_out,
              double* __restrict__ U_out, double* __restrict__ T_out,
              double* __restrict__ partials, long long block0, long long end) {
  using Mo = Model<M>;
  constexpr int D = Mo::D, Q = Mo::Q;
  const ModelConst& mc = c_mc[M];
  const long long block = block0 + blockIdx.x;
  const long long idx = block * blockDim.x + threadIdx.x;
  double acc[kAuditSlots] = {0, 0, 0, 0, 0, 1e300, 0, 0};
  if constexpr (!std::is_same<S, double>::value) {
    moments_fp32_forms<M, S>(src, g, idx, end, block, rho_out, U_out, T_out, partials);
    return;
  } else if (idx < end) {
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
    partials[(size_t)block * kAuditSlots + k] = v;
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

// ----------------------------------------------------------------- fixed end planes
// The shock tube's end conditions: after a step, the cells with coordinate
// < width (side 0) or >= N - width (side 1) along `axis` take the populations of
// template cell `side` (the discrete equilibrium of that side's state).
template <class S>
__global__ void k_fix_ends(S* __restrict__ state, Grid g, int axis, int width,
                           const S* __restrict__ tmpl, int Q) {
  const int n_ax = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
  const long long per_layer = g.ncell / n_ax;
  const long long total = 2LL * width * per_layer;
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < total;
       b += (long long)gridDim.x * blockDim.x) {
    const long long layer = b / per_layer;            // 0 .. 2 width - 1
    const long long r = b - layer * per_layer;        // position within the plane
    const int side = layer < width ? 0 : 1;
    const int c_ax = side == 0 ? (int)layer : n_ax - 2 * width + (int)layer;
    long long cell;
    if (axis == 2) {
      cell = (long long)c_ax * g.nxy + r;
    } else if (axis == 1) {
      const long long z = r / g.nx, x = r - z * g.nx;
      cell = (z * g.ny + c_ax) * g.nx + x;
    } else {
      cell = r * g.nx + c_ax;                        // r runs over (z, y) rows
    }
    for (int i = 0; i < Q; ++i) state[(size_t)i * g.ncell + cell] = tmpl[2 * i + side];
  }
}

// ----------------------------------------------------------------- slab halo copy
// Domain decomposition along the slowest axis: `segs` lists (direction, local plane)
// pairs; segment j occupies elements [j * plane, (j + 1) * plane) of the message.
// to_buf: state -> message (pack), else message -> state (unpack).
template <class S>
__global__ void k_halo_copy(S* __restrict__ state, S* __restrict__ buf, const int2* __restrict__ segs,
                            int nseg, long long plane, long long ncell, int to_buf) {
  const long long n = (long long)nseg * plane;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const long long j = k / plane;
    const long long c = k - j * plane;
    const int2 sg = segs[j];
    const size_t off = (size_t)sg.x * (size_t)ncell + (size_t)sg.y * (size_t)plane + (size_t)c;
    if (to_buf) buf[k] = state[off];
    else state[off] = buf[k];
  }
}

}  // namespace lbm

// adjoint_kernels.cuh - sm_103a kernels of the discrete adjoint (templates).
//
// Included by k_storage.inl after kernels.cuh (which supplies the model table,
// codecs, equilibrium coefficients and helpers).
#pragma once

#include "kernels.cuh"

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


// Pairs [first, end) of symmetry group g (g >= 1) in storage order.
template <int M>
struct ShellPairs {
  static constexpr int first(int g) {
    int p = 0;
    while (p < Model<M>::NP && Model<M>::vs.grp[1 + 2 * p] != g) ++p;
    return p;
  }
  static constexpr int end(int g) {
    int p = first(g);
    while (p < Model<M>::NP && Model<M>::vs.grp[1 + 2 * p] == g) ++p;
    return p;
  }
};

// Passes 2 and 3 as loops over each shell's pairs (lattice vectors read from
// constant memory) instead of fully unrolled over all pairs: a smaller kernel for
// the instruction cache.  Needs lambda in shared memory or uniform (FP32 adjoint).
#ifndef LBM_ADJ_SHELL_LOOP
#define LBM_ADJ_SHELL_LOOP 1
#endif

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

#ifndef LBM_ADJ_MINB
#define LBM_ADJ_MINB 4
#endif
// The FP32 adjoint commits its lambda copies in this many groups and waits for each
// just before pass 1 needs it, so the later groups' latency overlaps pass 1 (1.75
// adjoint steps per forward step against 1.78 with one wait for all; 2, 3 or 6
// groups measured 1.76).
// Unroll factor of the shell loops of passes 2 and 3 (1.74 adjoint steps per forward
// step at 2, 1.75 at 1, 1.78 at 3).
#ifndef LBM_ADJ_UNROLL
#define LBM_ADJ_UNROLL 2
#endif
constexpr int kAdjUnroll = LBM_ADJ_UNROLL;
#ifndef LBM_ADJ_GROUPS
#define LBM_ADJ_GROUPS 4
#endif
#ifndef LBM_ADJ_LAM_SMEM
#define LBM_ADJ_LAM_SMEM 1
#endif
template <class S>
struct AdjMinBlocks {
  static constexpr int value = std::is_same<S, double>::value ? 1 : LBM_ADJ_MINB;
};
// FP32 adjoint: the Q gathered lambda_i of a thread live in dynamic shared memory
// (lambda_i of thread t at word i * 128 + t: conflict-free), which leaves the
// registers to the gather offsets and the sums (Q floats in registers on top of
// them spill at 128 registers a thread).  The FP64 adjoint keeps them in registers.
template <class L>
struct AdjLamSmem {
  static constexpr bool value = std::is_same<L, float>::value && LBM_ADJ_LAM_SMEM;
};
constexpr int kAdjThreads = 128;
template <int M, class L>
constexpr int adj_smem_bytes() {
  return AdjLamSmem<L>::value ? Model<M>::Q * kAdjThreads * (int)sizeof(L) : 0;
}
// Address of population i at a cell: the element index in 32 bits when every index
// of a state copy fits them (NARROW), which saves the per-population 64-bit offset
// arithmetic; else the population's array first, then the cell.  (A macro: passed
// through a helper function, the 64-bit form compiled to a different register
// allocation, 168 registers with spills against 128 without.)
#define LBM_POP(base, i, cell)                                                                \
  (NARROW ? (base) + (uint32_t)((uint32_t)(i) * (uint32_t)g.ncell + (uint32_t)(cell))         \
          : (base) + (size_t)(i) * g.ncell + (cell))
template <int M, class S, class L, bool kFirst, bool NARROW>
__global__ void __launch_bounds__(kAdjThreads, AdjMinBlocks<S>::value)
    k_adjoint(const S* __restrict__ state, const L* __restrict__ nu_next,
              const double* __restrict__ dldrho, L* __restrict__ nu_out,
              double* __restrict__ omega_acc, Grid g, double omega) {
  using Mo = Model<M>;
  using Rt = L;
  constexpr int Q = Mo::Q, D = Mo::D, RR = Mo::R, NP = Mo::NP;
  constexpr bool kSm = AdjLamSmem<L>::value;
  // the lambda copies are committed in kGroups groups of kPerGroup pairs; pass 1
  // waits for each group just before its first pair
  constexpr int kGroups = LBM_ADJ_GROUPS;
  constexpr int kPerGroup = (NP + kGroups - 1) / kGroups;
  const ModelConst& mc = c_mc[M];
  __shared__ double sh[4];
  extern __shared__ __align__(16) unsigned char adj_dyn[];
  wait_prior_grid();     // programmatic launch: the previous step's writes are visible after this
  allow_next_grid();

  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  const bool active = x < g.nx;
  double om_part = 0.0;
  if (active) {
    int xo[2 * RR + 1], yo[2 * RR + 1], zo[2 * RR + 1];
    neighbour_offsets<D, RR>(x, y, z, g.nx, g.ny, g.nz, g.nxy, xo, yo, zo);
    const size_t self = ((size_t)z * g.ny + y) * g.nx + x;
    Rt l1 = Rt(0);
    if constexpr (kFirst) l1 = (Rt)dldrho[self];
    // lambda_i(x) = nu_next(x + e_i, i): one value per direction for the first step
    // of the sweep (dL/drho_N, the same for every i), else gathered.
    Rt lam_r[(kSm || kFirst) ? 1 : Q];
    const Rt* const lam_s = reinterpret_cast<const Rt*>(adj_dyn) + threadIdx.x;
    auto lam = [&](int i) -> Rt {
      if constexpr (kFirst) return l1;
      else if constexpr (kSm) return lam_s[i * kAdjThreads];
      else return lam_r[i];
    };
    if constexpr (kSm && !kFirst) {
      // FP32: the lambda gather goes global -> shared by cp.async, which holds no
      // registers while in flight; each thread waits for its own copies only.
      Rt* const dst = reinterpret_cast<Rt*>(adj_dyn) + threadIdx.x;
      cp_async4(dst, nu_next + self);
      sfor<0, NP>([&](auto P) {
        constexpr int p = decltype(P)::value;
        constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
        constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
        const int cm = zo[ez + RR] + yo[ey + RR] + xo[ex + RR];   // x - e_ip
        const int cp = zo[RR - ez] + yo[RR - ey] + xo[RR - ex];   // x + e_ip
        cp_async4(dst + ip * kAdjThreads, LBM_POP(nu_next, ip, cp));
        cp_async4(dst + im * kAdjThreads, LBM_POP(nu_next, im, cm));
        if constexpr (kGroups > 1 && (p % kPerGroup == kPerGroup - 1 || p + 1 == NP))
          cp_async_commit();
      });
      if constexpr (kGroups <= 1) cp_async_wait_all();
    }
    // pass 1: forward moments of g (gathered from x - e_i) and sum lambda_i f_i
    Rt rs, es = Rt(0), jx = Rt(0), jy = Rt(0), jz = Rt(0), sg;
    {
      const Rt h0 = (Rt)Codec<S>::ld(state + self);
      if constexpr (kSm && !kFirst && kGroups > 1) cp_async_wait_group<kGroups - 1>();
      if constexpr (!kSm && !kFirst) lam_r[0] = nu_next[self];
      rs = gW<Rt>(mc, 0) * h0;
      sg = gW<Rt>(mc, 0) * lam(0) * (Rt(1) + h0);
    }
    // Shell by shell: the weight and |xi|^2 are common to a shell, so the pair
    // terms are summed unweighted and each shell's totals are weighted once.
    Rt gs = Rt(0), gjx = Rt(0), gjy = Rt(0), gjz = Rt(0), gsg = Rt(0);
    sfor<0, NP>([&](auto P) {
      constexpr int p = decltype(P)::value;
      constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
      constexpr int gg = Mo::vs.grp[ip];
      constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
      constexpr bool first = (p == 0) || (Mo::vs.grp[ip - 2] != gg);
      constexpr bool last = (p + 1 == NP) || (Mo::vs.grp[ip + 2] != gg);
      if constexpr (kSm && !kFirst && kGroups > 1 && p > 0 && p % kPerGroup == 0)
        cp_async_wait_group<kGroups - 1 - p / kPerGroup>();
      const int cm = zo[ez + RR] + yo[ey + RR] + xo[ex + RR];   // x - e_ip
      const int cp = zo[RR - ez] + yo[RR - ey] + xo[RR - ex];   // x + e_ip
      const Rt hp = (Rt)Codec<S>::ld(LBM_POP(state, ip, cm));
      const Rt hm = (Rt)Codec<S>::ld(LBM_POP(state, im, cp));
      if constexpr (!kSm && !kFirst) {
        lam_r[ip] = *LBM_POP(nu_next, ip, cp);
        lam_r[im] = *LBM_POP(nu_next, im, cm);
      }
      if constexpr (first) gs = gjx = gjy = gjz = gsg = Rt(0);
      const Rt sp = hp + hm, dm = hp - hm;
      gs += sp;
      if constexpr (ex != 0) gjx += Rt(ex) * dm;
      if constexpr (ey != 0) gjy += Rt(ey) * dm;
      if constexpr (ez != 0) gjz += Rt(ez) * dm;
      const Rt lp = lam(ip), lm = lam(im);
      gsg += lp * hp + lm * hm + (lp + lm);               // lambda_p f_p / w + lambda_m f_m / w
      if constexpr (last) {
        const Rt w = gW<Rt>(mc, gg);
        const Rt tr = w * gs;
        rs += tr;
        es += gX2<Rt>(mc, gg) * tr;
        jx += w * gjx;
        jy += w * gjy;
        jz += w * gjz;
        sg += w * gsg;
      }
    });
    // Linearisation point: the forward moments and temperature of g.  Plain sums in
    // the arithmetic type suffice here (they fix where the Jacobian is taken, to
    // ~1e-7 relative in FP32; the gradients are compared at 1e-4).
    const Rt rho_r = Rt(1) + rs;
    Rt ir_r;
    if constexpr (std::is_same<Rt, float>::value) ir_r = __fdividef(1.0f, rho_r);
    else ir_r = 1.0 / rho_r;
    const double rho_d = (double)rho_r;
    const Rt ux = gA<Rt>(mc) * jx * ir_r;
    const Rt uy = gA<Rt>(mc) * jy * ir_r;
    const Rt uz = (D == 3) ? gA<Rt>(mc) * jz * ir_r : Rt(0);
    const Rt q = ux * ux + uy * uy + uz * uz;
    const Rt t = ((es - Rt(D) * rs) * ir_r - q) * Rt(1.0 / D);
    const Rt theta = Rt(1) + t;
    const EqCoef<Rt, D> cf(q, t);
    const EqGrad<Rt, D> gr(q, t);
    const Rt a_r = gA<Rt>(mc);
    const Rt uax = a_r * ux, uay = a_r * uy, uaz = a_r * uz;

    // pass 2: contractions with lambda
    Rt Lr = gW<Rt>(mc, 0) * lam(0) * cf.K0;
    Rt Sq = gW<Rt>(mc, 0) * lam(0) * gr.Bq(Rt(0));
    Rt St = gW<Rt>(mc, 0) * lam(0) * gr.Bt(Rt(0));
    Rt Vx = Rt(0), Vy = Rt(0), Vz = Rt(0);
    // Per shell, with ls = lambda_p + lambda_m, ld = lambda_p - lambda_m and s = xi_p . u:
    //   sum ls P = A0 m0 + A2 m2 + m4 / 24 + A1 n1 + n3 / 6,
    //   sum ls dP/dq = Bq m0 - m2 / 4 - n1 / 2,  sum ls dP/dt = Bt m0 + Dt m2 + Ct n1,
    // with m0 = sum ls, m2 = sum ls s^2, m4 = sum ls s^4, n1 = sum ld s, n3 = sum ld s^3;
    // the vector term keeps one v = ld (A1 + s^2/2) + ls s (2 A2 + s^2/6) per pair.
    Rt m0 = Rt(0), m2 = Rt(0), m4 = Rt(0), n1 = Rt(0), n3 = Rt(0);
    Rt gvx = Rt(0), gvy = Rt(0), gvz = Rt(0);
    constexpr bool kLoop = LBM_ADJ_SHELL_LOOP && (kSm || kFirst);
    if constexpr (kLoop) {
      sfor<1, Mo::G>([&](auto Gi) {
        constexpr int gg = decltype(Gi)::value;
        const Rt x2 = gX2<Rt>(mc, gg);
        const Rt A1 = cf.A1(x2), A2 = cf.A2(x2);
        m0 = m2 = m4 = n1 = n3 = gvx = gvy = gvz = Rt(0);
#pragma unroll kAdjUnroll
        for (int p = ShellPairs<M>::first(gg); p < ShellPairs<M>::end(gg); ++p) {
          const int ip = 1 + 2 * p, im = 2 + 2 * p;
          const Rt ex = mc.ef[ip][0], ey = mc.ef[ip][1], ez = mc.ef[ip][2];
          const Rt s = ex * uax + ey * uay + ez * uaz;
          const Rt s2 = s * s;
          const Rt lp = lam(ip), lm = lam(im);
          const Rt ls = lp + lm, ld = lp - lm;
          const Rt tl = ls * s2, tu = ld * s;
          m0 += ls;
          m2 += tl;
          m4 += tl * s2;
          n1 += tu;
          n3 += tu * s2;
          const Rt v = ld * (A1 + s2 * Rt(0.5)) + (ls * s) * (Rt(2) * A2 + s2 * Rt(1.0 / 6.0));
          gvx += ex * v;
          gvy += ey * v;
          gvz += ez * v;
        }
        const Rt w = gW<Rt>(mc, gg);
        Lr += w * (cf.A0(x2) * m0 + A2 * m2 + m4 * Rt(1.0 / 24.0) + A1 * n1 + n3 * Rt(1.0 / 6.0));
        Sq += w * (gr.Bq(x2) * m0 - m2 * Rt(0.25) - n1 * Rt(0.5));
        St += w * (gr.Bt(x2) * m0 + EqGrad<Rt, D>::Dt(x2) * m2 + EqGrad<Rt, D>::Ct(x2) * n1);
        Vx += w * gvx;
        Vy += w * gvy;
        Vz += w * gvz;
      });
    } else
    sfor<0, NP>([&](auto P) {
      constexpr int p = decltype(P)::value;
      constexpr int ip = 1 + 2 * p, im = 2 + 2 * p;
      constexpr int gg = Mo::vs.grp[ip];
      constexpr int ex = Mo::vs.e[ip][0], ey = Mo::vs.e[ip][1], ez = Mo::vs.e[ip][2];
      constexpr bool first = (p == 0) || (Mo::vs.grp[ip - 2] != gg);
      constexpr bool last = (p + 1 == NP) || (Mo::vs.grp[ip + 2] != gg);
      const Rt x2 = gX2<Rt>(mc, gg);
      const Rt A1 = cf.A1(x2), A2 = cf.A2(x2);
      Rt s = Rt(0);
      if constexpr (ex != 0) s += Rt(ex) * uax;
      if constexpr (ey != 0) s += Rt(ey) * uay;
      if constexpr (ez != 0) s += Rt(ez) * uaz;
      const Rt s2 = s * s;
      const Rt lp = lam(ip), lm = lam(im);
      const Rt ls = lp + lm, ld = lp - lm;
      const Rt tl = ls * s2, tu = ld * s;
      if constexpr (first) m0 = m2 = m4 = n1 = n3 = gvx = gvy = gvz = Rt(0);
      m0 += ls;
      m2 += tl;
      m4 += tl * s2;
      n1 += tu;
      n3 += tu * s2;
      const Rt v = ld * (A1 + s2 * Rt(0.5)) + (ls * s) * (Rt(2) * A2 + s2 * Rt(1.0 / 6.0));
      if constexpr (ex != 0) gvx += Rt(ex) * v;
      if constexpr (ey != 0) gvy += Rt(ey) * v;
      if constexpr (ez != 0) gvz += Rt(ez) * v;
      if constexpr (last) {
        const Rt w = gW<Rt>(mc, gg);
        Lr += w * (cf.A0(x2) * m0 + A2 * m2 + m4 * Rt(1.0 / 24.0) + A1 * n1 + n3 * Rt(1.0 / 6.0));
        Sq += w * (gr.Bq(x2) * m0 - m2 * Rt(0.25) - n1 * Rt(0.5));
        St += w * (gr.Bt(x2) * m0 + EqGrad<Rt, D>::Dt(x2) * m2 + EqGrad<Rt, D>::Ct(x2) * n1);
        Vx += w * gvx;
        Vy += w * gvy;
        Vz += w * gvz;
      }
    });
    // chain rule to the moments (arithmetic type; the omega term in FP64)
    const Rt Lux = rho_r * (a_r * Vx + Rt(2) * ux * Sq);
    const Rt Luy = rho_r * (a_r * Vy + Rt(2) * uy * Sq);
    const Rt Luz = (D == 3) ? rho_r * (a_r * Vz + Rt(2) * uz * Sq) : Rt(0);
    const Rt Lt = rho_r * St;
    const Rt iDr = ir_r * Rt(1.0 / D);
    const Rt alpha = Lr - (ux * Lux + uy * Luy + uz * Luz) * ir_r + Lt * (q - Rt(D) * theta) * iDr;
    const Rt bx = Lux * ir_r - Rt(2) * Lt * ux * iDr;
    const Rt by = Luy * ir_r - Rt(2) * Lt * uy * iDr;
    const Rt bz = Luz * ir_r - Rt(2) * Lt * uz * iDr;
    const Rt gam = Lt * iDr;
    om_part = fma(rho_d, (double)Lr, -(double)sg);

    // pass 3: nu_n(x, j)
    const Rt om1 = (Rt)(1.0 - omega);
    const Rt om = (Rt)omega;
    const Rt oa = om * alpha, og = om * gam;
    const Rt obx = om * a_r * bx, oby = om * a_r * by, obz = om * a_r * bz;
    nu_out[self] = om1 * lam(0) + oa;
    if constexpr (kLoop) {
      sfor<1, Mo::G>([&](auto Gi) {
        constexpr int gg = decltype(Gi)::value;
        const Rt ev = oa + og * gX2<Rt>(mc, gg);
#pragma unroll kAdjUnroll
        for (int p = ShellPairs<M>::first(gg); p < ShellPairs<M>::end(gg); ++p) {
          const int ip = 1 + 2 * p, im = 2 + 2 * p;
          const Rt od = mc.ef[ip][0] * obx + mc.ef[ip][1] * oby + mc.ef[ip][2] * obz;
          *LBM_POP(nu_out, ip, self) = om1 * lam(ip) + (ev + od);
          *LBM_POP(nu_out, im, self) = om1 * lam(im) + (ev - od);
        }
      });
    } else
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
      *LBM_POP(nu_out, ip, self) = om1 * lam(ip) + (ev + od);
      *LBM_POP(nu_out, im, self) = om1 * lam(im) + (ev - od);
    });
  }
  const double bsum = block_sum_128(om_part, sh);
  if (threadIdx.x == 0) {
    const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    omega_acc[b] += bsum;
  }
}

#undef LBM_POP

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
  neighbour_offsets<D, RR>(x, y, z, g.nx, g.ny, g.nz, g.nxy, xo, yo, zo);
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

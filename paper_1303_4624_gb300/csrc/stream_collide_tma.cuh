// stream_collide_tma.cuh - the TMA-staged fused stream-collide (sm_103a).
//
// Same cell update as k_stream_collide (cell_collide: the paper's BGK rule with the
// fourth-order Hermite equilibrium), with the gather of a1 moved off the threads:
//
//   * A CTA of 128 threads owns "chunks" of 128 consecutive cells of one x-row
//     (persistent CTAs, chunk c = blockIdx.x + k gridDim.x).  For chunk
//     (x0, y, z), direction i pulls from the source row (y - e_y, z - e_z) at
//     x0 - e_x ... x0 - e_x + 127 (all periodic).
//   * Warp 0 is also the producer: for each chunk it issues one bulk asynchronous
//     copy (the TMA engine's cp.async.bulk, global -> shared) per direction of the
//     16-byte-aligned row segment that covers those 128 cells (136 elements when
//     e_x != 0, 128 when e_x = 0; two copies where the segment wraps around the
//     row end), into one stage of a ring of STAGES stages.  A stage has a "full"
//     mbarrier (one arrival carrying the expected byte count, completed by the
//     copies) and an "empty" mbarrier (one arrival per warp once its threads have
//     read the stage).  Warp 0 refills a stage as soon as it is empty, STAGES - 1
//     chunks ahead of the one being computed.
//   * Every thread reads its Q populations from the stage at compile-time offsets
//     (row offset + 8 - e_x, or - e_x, plus its lane): no address arithmetic, no
//     periodic wrap in the inner loop.
//   * OUT_SMEM (used for the D2Q33 16-bit forms): the Q results of the chunk go to
//     a shared-memory output tile, and warp 0 writes each direction's 128 results
//     back with one bulk copy (shared -> global), so the stores need no address
//     arithmetic either.  Otherwise each thread stores straight to global memory
//     (measured faster for D3Q95: the tile costs two block barriers per chunk).
//
// Every wait is bounded (limit_ns of wall time): a timeout sets *status (read by
// lbm_synchronize as LBM_EDEVICE), the CTA stops, and warp 0 waits (bounded) for
// the copies it still has in flight before the CTA exits.  The failure is agreed
// on at a CTA-wide barrier (OUT_SMEM), or each warp stops on its own (no barrier
// follows), so no barrier waits on a warp that has left.  TmaTest.stall_chunk
// (tests only) makes the producer skip one chunk's copies so that the consumers'
// wait runs out; nothing else changes.
//
// Needs Nx % 8 == 0 (16-byte copy granularity of FP16 rows).
#pragma once

#include "kernels.cuh"

namespace lbm {

constexpr int kTmaW = 128;     // cells per chunk = threads per CTA
constexpr int kTmaPad = 8;     // x-halo of a shifted row segment (16 bytes of FP16)

struct TmaTest {
  long long stall_chunk;       // -1: none; else the chunk whose copies are skipped
  unsigned long long limit_ns; // bound of every wait
};

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// The single arrival of a phase that also announces the bytes its copies will bring.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of parity `parity` to complete; false after limit_ns of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    for (int k = 0; k < 64; ++k)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
// Bulk copy global -> shared completing on an mbarrier (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// Bulk copy shared -> global, tracked by this thread's bulk async-group.
__device__ __forceinline__ void bulk_s2g(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// This thread's committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// ... and have completed their writes.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// Order this thread's generic-proxy shared-memory writes before later async-proxy
// (bulk copy) reads of them.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <class S>
__device__ __forceinline__ typename Codec<S>::R lds(const S* p) {
  if constexpr (std::is_same<S, __half>::value)
    return __half2float(*p);
  else if constexpr (std::is_same<S, __nv_bfloat16>::value)
    return __bfloat162float(*p);
  else
    return *p;
}

// ---------------------------------------------------------------- stage layout
// Direction i's row segment: 136 elements when e_x != 0 (segment start x0 - 8 for
// e_x > 0, x0 for e_x < 0), 128 when e_x = 0 (start x0); rows packed in direction
// order.  Cell t of the chunk reads element pos(i) + t of its row.
template <int M>
struct TmaRows {
  static constexpr int Q = Model<M>::Q;
  static constexpr int ex(int i) { return Model<M>::vs.e[i][0]; }
  static constexpr int len(int i) { return ex(i) != 0 ? kTmaW + kTmaPad : kTmaW; }
  static constexpr int off(int i) {
    int o = 0;
    for (int j = 0; j < i; ++j) o += len(j);
    return o;
  }
  static constexpr int pos(int i) { return ex(i) > 0 ? kTmaPad - ex(i) : -ex(i); }
  static constexpr int nonzero_ex() {
    int n = 0;
    for (int j = 0; j < Q; ++j) n += ex(j) != 0;
    return n;
  }
  static constexpr int total = off(Q);          // elements per stage
};

template <int M, class S, int STAGES, bool OUT_SMEM>
struct TmaSmem {
  static constexpr size_t kStage = (size_t)TmaRows<M>::total * sizeof(S);
  static constexpr size_t kOut = OUT_SMEM ? (size_t)Model<M>::Q * kTmaW * sizeof(S) : 0;
  static constexpr size_t kBytes = STAGES * kStage + kOut;   // dynamic shared memory
};

// ---------------------------------------------------------------- the kernel
template <int M, class S, int STAGES, int MINB, bool OUT_SMEM>
__global__ void __launch_bounds__(kTmaW, MINB)
    k_stream_collide_tma(const S* __restrict__ src, S* __restrict__ dst, Grid g, double omega,
                         int nchunks, int* __restrict__ status, TmaTest test) {
  using Mo = Model<M>;
  using Rows = TmaRows<M>;
  using Rt = typename Codec<S>::R;
  constexpr int Q = Mo::Q;
  static_assert(Rows::total % 8 == 0, "rows must stay 16-byte aligned");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S* stages = reinterpret_cast<S*>(smem_raw);
  S* obuf = stages + (size_t)STAGES * Rows::total;
  __shared__ __align__(8) unsigned long long full[STAGES], empty[STAGES];
  // per direction: e_x, e_y, e_z and the number of earlier directions with e_x != 0
  // (row offset = 128 i + 8 that number)
  __shared__ char4 sdir[Q];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < Q; i += kTmaW) {
    int before = 0;
    for (int j = 0; j < i; ++j) before += c_mc[M].e[j][0] != 0;
    sdir[i] = make_char4((signed char)c_mc[M].e[i][0], (signed char)c_mc[M].e[i][1],
                         (signed char)c_mc[M].e[i][2], (signed char)before);
  }
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), kTmaW / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  wait_prior_grid();     // the previous step's writes (our src) and reads (our dst) are done
  allow_next_grid();

  const int nxc = (g.nx + kTmaW - 1) / kTmaW;
  const int G = gridDim.x;
  const int my_n = ((int)blockIdx.x < nchunks) ? (nchunks - (int)blockIdx.x + G - 1) / G : 0;
  const uint64_t limit = test.limit_ns;

  // Producer step (all lanes of warp 0): copies of this CTA's k-th chunk into stage
  // k % STAGES, once the chunk that used the stage before has been read.  False if
  // that wait ran out (nothing was issued then).
  int issued = 0;        // chunks issued so far (warp 0)
  auto issue = [&](int k) -> bool {
    const int s = k % STAGES;
    if (k >= STAGES &&
        !mbar_wait_bounded(smem_addr(&empty[s]), (uint32_t)(((k - STAGES) / STAGES) & 1), limit))
      return false;
    issued = k + 1;
    const long long c = (long long)blockIdx.x + (long long)k * G;
    if (c == test.stall_chunk) return true;   // test hook: no copies, no arrival
    const int xc = (int)(c % nxc);
    const int row = (int)(c / nxc);
    const int y = row % g.ny, z = row / g.ny;
    const int x0 = xc * kTmaW;
    const int wc = min(kTmaW, g.nx - x0);
    const uint32_t bar = smem_addr(&full[s]);
    if (lane == 0) {
      constexpr int nz = Rows::nonzero_ex();
      mbar_arrive_expect_tx(bar, (uint32_t)((nz * (wc + kTmaPad) + (Q - nz) * wc) * sizeof(S)));
    }
    __syncwarp();
    S* stage = stages + (size_t)s * Rows::total;
    for (int i = lane; i < Q; i += 32) {
      const char4 d = sdir[i];
      const int ys = wrapi(y - d.y, g.ny);
      const int zs = wrapi(z - d.z, g.nz);
      const S* rowp = src + (size_t)i * (size_t)g.ncell + ((size_t)zs * g.ny + ys) * g.nx;
      const int a = x0 - (d.x > 0 ? kTmaPad : 0);
      const int len = wc + (d.x != 0 ? kTmaPad : 0);
      const uint32_t sd = smem_addr(stage + i * kTmaW + kTmaPad * d.w);
      if (a < 0) {                                   // wraps past x = 0
        bulk_g2s(sd, rowp + (g.nx + a), (uint32_t)(-a * sizeof(S)), bar);
        bulk_g2s(sd + (uint32_t)(-a * sizeof(S)), rowp, (uint32_t)((len + a) * sizeof(S)), bar);
      } else if (a + len > g.nx) {                   // wraps past x = Nx - 1
        const int n1 = g.nx - a;
        bulk_g2s(sd, rowp + a, (uint32_t)(n1 * sizeof(S)), bar);
        bulk_g2s(sd + (uint32_t)(n1 * sizeof(S)), rowp, (uint32_t)((len - n1) * sizeof(S)), bar);
      } else {
        bulk_g2s(sd, rowp + a, (uint32_t)(len * sizeof(S)), bar);
      }
    }
    return true;
  };

  if (warp == 0)
    for (int k = 0; k < STAGES - 1 && k < my_n; ++k) issue(k);   // no wait for the first fills

  bool failed = false;
  int k = 0;
  for (; k < my_n; ++k) {
    const int s = k % STAGES;
    bool ok = true;
    if (warp == 0 && k + STAGES - 1 < my_n) ok = issue(k + STAGES - 1);
    ok = ok && mbar_wait_bounded(smem_addr(&full[s]), (uint32_t)((k / STAGES) & 1), limit);
    const long long c = (long long)blockIdx.x + (long long)k * G;
    const int xc = (int)(c % nxc);
    const int row = (int)(c / nxc);
    const int x0 = xc * kTmaW;
    const int wc = min(kTmaW, g.nx - x0);
    // a1 + a2: the Q gathered populations of cell x0 + tid, at compile-time offsets
    Rt h[Q];
    if (ok && tid < wc) {
      const S* sp = stages + (size_t)s * Rows::total + tid;
      sfor<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        h[i] = lds<S>(sp + (Rows::off(i) + Rows::pos(i)));
      });
    }
    __syncwarp();
    if (ok && lane == 0) mbar_arrive(smem_addr(&empty[s]));   // this warp is done with the stage
    if constexpr (OUT_SMEM) {
      // the output tile is free once warp 0's bulk stores of the previous chunk have read it
      if (warp == 0 && k > 0) bulk_wait_read_all();
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      if (tid < wc)
        cell_collide<M, S>(h, omega, [&](auto I, Rt v) {
          Codec<S>::st(obuf + decltype(I)::value * kTmaW + tid, v);
        });
      fence_proxy_async_smem();
      __syncthreads();
      if (warp == 0) {
        S* drow = dst + (size_t)row * g.nx + x0;
        for (int i = lane; i < Q; i += 32)
          bulk_s2g(drow + (size_t)i * (size_t)g.ncell, smem_addr(obuf + i * kTmaW),
                   (uint32_t)(wc * sizeof(S)));
        bulk_commit();
      }
    } else {
      if (!ok) {
        failed = true;
        break;
      }
      if (tid < wc) {
        const size_t self = (size_t)row * g.nx + x0 + tid;
        cell_collide<M, S>(h, omega, [&](auto I, Rt v) {
          Codec<S>::st(dst + (size_t)decltype(I)::value * (size_t)g.ncell + self, v);
        });
      }
    }
  }
  if (failed) {
    if (lane == 0) atomicExch(status, 1);
    // copies still in flight into this CTA's stages (chunks k .. issued - 1)
    if (warp == 0)
      for (int j = k; j < issued; ++j) {
        const long long c = (long long)blockIdx.x + (long long)j * G;
        if (c != test.stall_chunk)
          mbar_wait_bounded(smem_addr(&full[j % STAGES]), (uint32_t)((j / STAGES) & 1), limit);
      }
  }
  if constexpr (OUT_SMEM)
    if (warp == 0) bulk_wait_all();   // the last chunks' stores are complete
}

}  // namespace lbm

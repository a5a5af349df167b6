// common.h - types shared by the host API and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace lbm {

constexpr int kMaxQc = 95;
constexpr int kMaxGc = 10;

// Per-model constants solved on the host (Formula 5) and kept in constant memory.
struct ModelConst {
  double W[kMaxGc];    // weight of each symmetry group
  double X2[kMaxGc];   // |xi|^2 = a^2 |e|^2 of each group
  float Wf[kMaxGc];
  float X2f[kMaxGc];
  float X2lo[kMaxGc];  // X2 - X2f: with X2f, X2 as a double-float (hi, lo) pair
  double w[kMaxQc];    // weight per direction (storage order)
  double a;            // sqrt(2) c: xi_i = a e_i
  float af, alo;       // a rounded to FP32, and a - af
  double c;
  double T0;           // 1 / (2 c^2), lattice units
  float T0f, iT0f;     // T0 and 1 / T0 rounded to FP32
  float iT0lo;         // 1 / T0 - iT0f
  int e[kMaxQc][3];    // lattice vectors in storage order (zero-padded to 3 components)
  float ef[kMaxQc][3]; // the same as FP32 (loops that index directions at run time)
};

struct Grid {
  int nx, ny, nz, nxy;
  long long ncell;
};

// Failure-detection test of the TMA kernel's bounded waits: the producer skips the
// copies of chunk stall_chunk, so its consumers' wait runs out after limit_ns.
struct StepTest {
  long long stall_chunk;
  unsigned long long limit_ns;
};

// Launchers of one storage form (one translation unit each).  All enqueue on
// `st` and return the launch status.
struct StorageOps {
  int elem_bytes;
  cudaError_t (*upload)(const ModelConst* mc2);
  // The equilibrium of the fields for cells [begin, end) (U strided by g.ncell).
  cudaError_t (*init)(int model, const double* rho, const double* U, const double* T, void* dst,
                      const Grid& g, long long begin, long long end, cudaStream_t st);
  // One stream-collide step.  variant: kVariantDirect, kVariantTma, kVariantSplit or
  // kVariantPair, or-ed with kStepReverse for the direct and pair kernels (the caller
  // checks applicability: Nx % 8 == 0 for TMA, Nx even and 16-bit storage for pair).  status: device int
  // set to 1 if a TMA launch gave up waiting for its copies.  test: NULL, or the
  // failure-detection test setting of a TMA launch (see StepTest).
  cudaError_t (*step)(int model, const void* src, void* dst, const Grid& g, double omega,
                      int variant, int* status, const StepTest* test, cudaStream_t st);
  // One-time per-device launch set-up of the TMA kernels (shared-memory opt-in and
  // occupancy), done before any stream capture.
  cudaError_t (*prepare_tma)(int model);
  // Moments and audit partials of blocks [block0, block0 + nblocks) of kMomentThreads
  // cells (moment_blocks(ncell) blocks cover the grid).
  cudaError_t (*moments)(int model, const void* src, const Grid& g, double* rho, double* U,
                         double* T, double* partials, long long block0, long long nblocks,
                         cudaStream_t st);
  cudaError_t (*get_f)(int model, const void* src, double* f, const Grid& g, cudaStream_t st);
  cudaError_t (*set_f)(int model, const double* f, void* dst, const Grid& g, cudaStream_t st);
  // Overwrite the first / last `width` planes along `axis` (0 x, 1 y, 2 z) with the
  // populations of template cell 0 / 1 (tmpl is [Q][2] in the storage type).
  cudaError_t (*fix_ends)(void* state, const Grid& g, int axis, int width, const void* tmpl, int Q,
                          cudaStream_t st);
  // Halo pack (to_buf = 1: state -> buf) or unpack (0) of the (direction, plane)
  // segments segs[2 j], segs[2 j + 1] (device array), each `plane` elements.
  cudaError_t (*halo_copy)(void* state, void* buf, const int* segs, int nseg, long long plane,
                           long long ncell, int to_buf, cudaStream_t st);
  // Adjoint (lambda type: FP64 for the FP64 form, FP32 otherwise).
  int adj_elem_bytes;
  // One reverse step: nu_out = (collision Jacobian)^T lambda_{n+1} with
  // lambda_{n+1}(x, i) = nu_next(x + e_i, i), or dL/drho_N(x) when dldrho != NULL;
  // adds this step's dL/domega block partials into omega_acc[block].
  cudaError_t (*adjoint_step)(int model, const void* state_n, const void* nu_next,
                              const double* dldrho, void* nu_out, double* omega_acc,
                              const Grid& g, double omega, cudaStream_t st);
  // dL/d(rho0, U0, T0) from lambda_0(x, i) = nu0(x + e_i, i) and the initial fields.
  cudaError_t (*grad_init)(int model, const void* nu0, const double* fields, double* d_rho,
                           double* d_U, double* d_T, const Grid& g, cudaStream_t st);
};

// Blocks of the 3D cell launch shared by stream-collide and the adjoint step.
inline int cell_block_x(int nx) { return nx >= 128 ? 128 : ((nx + 31) / 32) * 32; }
inline long long cell_blocks(const Grid& g) {
  const int bx = cell_block_x(g.nx);
  return (long long)((g.nx + bx - 1) / bx) * g.ny * g.nz;
}
cudaError_t launch_sum_reduce(const double* partials, long long n, double* out, cudaStream_t st);
// Cells [begin, end) of fields with n cells (U strided by n): *first_bad = min over
// bad values of (index << 2 | field) (0 rho, 1 U, 2 T); the caller presets it to all
// ones.
cudaError_t launch_check_fields(const double* rho, const double* U, const double* T, long long n,
                                long long begin, long long end, int D,
                                unsigned long long* first_bad, cudaStream_t st);

extern const StorageOps kOpsFP64, kOpsFP32, kOpsFP16, kOpsBF16;

constexpr int kVariantDirect = 1;
constexpr int kVariantTma = 2;
constexpr int kVariantSplit = 3;
constexpr int kVariantPair = 4;   // two cells per thread, paired FP32 (FP16 / BF16 forms)
// Or-ed into the variant of a direct-kernel step: walk the blocks in reverse order.
// Alternate steps walk opposite ways, so each step starts on the cells its
// predecessor wrote last, which are still in L2.
constexpr int kStepReverse = 0x100;
inline bool tma_applicable(const Grid& g) { return g.nx % 8 == 0; }
inline bool pair_applicable(const Grid& g) { return g.nx % 2 == 0; }

constexpr int kAuditSlots = 8;
constexpr int kMomentThreads = 256;
inline int moment_blocks(long long ncell) {
  return (int)((ncell + kMomentThreads - 1) / kMomentThreads);
}
cudaError_t launch_audit_reduce(const double* partials, int nblocks, double* out, cudaStream_t st);

}  // namespace lbm

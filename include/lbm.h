/*
 * lbm.h - C ABI of the GB300 thermal lattice Boltzmann library (liblbm_gb300.so).
 *
 * The library implements the fused pull stream-and-collide BGK update of
 * J. W. Shim, "Multidimensional On-lattice Higher-order Models in the Thermal
 * Lattice Boltzmann Theory" (arXiv:1303.4624), on the paper's fourth-order
 * on-lattice velocity sets D2Q33 (Table 2) and D3Q95 (Table 3), on one GPU.
 *
 * Conventions shared by every entry point
 *   - Lattice units: V_i = e_i (integer lattice vectors), dx = dt = 1,
 *     k_B/m_g = 1.  The paper's dimensionless variables (text after the
 *     Maxwellian) map to these by v = c V, u = c U and theta = T / T0 with
 *     T0 = 1 / (2 c^2), where c is the model's speed scale of Table 2 / 3.
 *   - Grids are periodic boxes of Nx x Ny x Nz cells (Nz = 1 for D2Q33).
 *     Every field array is x-fastest: index = (z * Ny + y) * Nx + x.
 *     A vector field U is [D][cells] (component-major).  Population arrays
 *     are [Q][cells] in the direction order reported by lbm_model_info.
 *   - Time stepping is the pull form of the paper's update
 *       f_i(x + V_i, t + 1) = (1 - omega) f_i(x, t) + omega f_i^eq(x, t):
 *     each step gathers g_i(x) = f_i(x - e_i) and stores the post-collision
 *     populations at x.  rho, U and T are the same as in the push form.
 *   - f_i^eq is the fourth-order Hermite expansion of the Maxwellian about
 *     (u = 0, theta = 1) on the model's weights (Formula 1 with m = N = 4).
 *   - `where` arguments: LBM_HOST for host pointers, LBM_DEVICE for device
 *     pointers on the context's device.  Caller buffers are borrowed only for
 *     the duration of the call; the library keeps no pointer to them.
 *   - All calls are ordered on the context's CUDA stream.  Calls that take a
 *     host output return after the result is on the host; calls with device
 *     outputs (and lbm_step) return after enqueueing.
 *   - Every call returns LBM_OK (0) or a negative error code; arguments are
 *     validated before any launch that uses them (on the host, except the
 *     initial fields of lbm_init, checked on the device after their upload).  lbm_last_error()
 *     gives a message for the most recent failure on the calling thread.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define LBM_OK         0
#define LBM_EINVAL    -1   /* invalid argument (checked before any launch)          */
#define LBM_ENOMEM    -2   /* device allocation failed                              */
#define LBM_ECUDA     -3   /* a CUDA runtime call or kernel launch failed            */
#define LBM_EUNSTABLE -4   /* the audit found non-finite populations                */
#define LBM_ESTATE    -5   /* call out of order (e.g. lbm_step before lbm_init)      */
#define LBM_EDEVICE   -6   /* a kernel gave up on a bounded wait (reported by sync)  */
#define LBM_EIO       -7   /* a checkpoint file could not be read or written         */

/* ---- models and storage forms ---- */
#define LBM_D2Q33 0        /* Table 2: 33 velocities, 8 groups, reach 4 */
#define LBM_D3Q95 1        /* Table 3: 95 velocities, 10 groups, reach 5 */

#define LBM_FP64    0      /* populations stored in FP64, FP64 arithmetic              */
#define LBM_FP32    1      /* FP32 storage and arithmetic                              */
#define LBM_FP16DEV 2      /* FP16 storage of h_i = f_i / w_i - 1, FP32 arithmetic     */
#define LBM_BF16DEV 3      /* BF16 storage of h_i = f_i / w_i - 1, FP32 arithmetic     */
/* Every form stores the deviation h_i = f_i / w_i - 1 from the rest state
 * (rho0 = 1, U = 0, T = T0, where f_i^eq = w_i exactly), so all directions
 * share one dynamic range.  In the FP32 / FP16 / BF16 forms the moment sums for
 * density and energy are Kahan-compensated FP32, and the temperature
 * theta = (E / rho - |u|^2) / D is recovered in double-float (hi + lo FP32
 * pairs, as accurate as an FP64 recovery rounded to FP32) in all three. */

#define LBM_HOST   0
#define LBM_DEVICE 1

typedef struct lbm_ctx lbm_ctx;     /* opaque; owns the device population buffers */

/*
 * lbm_model_info - the velocity set and weights of a model.
 *   Tables 2 and 3 give one representative velocity per symmetry group; the
 *   set is every signed permutation of each representative (text before
 *   Formula 9).  The weights and c are the FP64 solution of Formula 5 up to
 *   n_max = 8, found by Newton's method from the printed values.
 *   Direction order: 0 is the rest velocity, then opposite pairs
 *   (2p+1, 2p+2) with e_{2p+2} = -e_{2p+1}.
 * Outputs (any may be NULL): Q, D, reach (max |e_i| component), e [Q*D] as
 *   int32 (x fastest within a direction), w [Q], c, T0 (lattice units).
 * Errors: LBM_EINVAL for an unknown model; LBM_ECUDA never.
 */
int lbm_model_info(int model, int* Q, int* D, int* reach, int32_t* e, double* w,
                   double* c, double* T0);

/*
 * lbm_set_allocator - route the library's device allocations through the
 * caller (the Python binding passes PyTorch's caching allocator).  alloc
 * returns a device pointer of at least `bytes` bytes or NULL; free releases it.
 * Both receive the stream of the context that allocates and `user`.  Passing
 * NULL functions restores cudaMalloc / cudaFree.  Affects later allocations
 * only; each buffer is released by the allocator that made it.
 */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*lbm_free_fn)(void* ptr, void* stream, void* user);
int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void* user);

/*
 * lbm_create - allocate a context for one periodic grid on the current device.
 * The model's velocity set and weights are those of Table 2 (D2Q33) or Table 3
 * (D3Q95), the weights re-solved from Formula 5 as lbm_model_info describes;
 * omega is the relaxation frequency of the paper's BGK update (the rule stated
 * before the Maxwellian).
 *   model:   LBM_D2Q33 or LBM_D3Q95
 *   dims:    {Nx, Ny, Nz}, each >= 1, Nz == 1 for D2Q33; Nx*Ny*Nz < 2^31
 *   omega:   BGK relaxation frequency (the paper's omega), 0 <= omega < 2
 *   storage: LBM_FP64 / LBM_FP32 / LBM_FP16DEV / LBM_BF16DEV
 *   stream:  cudaStream_t to order all work on (NULL = legacy default stream)
 * Allocates two population buffers (ping-pong) of Q * cells storage elements.
 * Errors: LBM_EINVAL (bad argument), LBM_ENOMEM, LBM_ECUDA.
 */
int lbm_create(lbm_ctx** out, int model, const int64_t dims[3], double omega,
               int storage, void* stream);

/* lbm_destroy - free every buffer of the context (after its stream drains). */
int lbm_destroy(lbm_ctx* ctx);

/* lbm_set_omega - change the relaxation frequency (0 <= omega < 2) for later
 * steps; invalidates a recorded rollout.  Errors: LBM_EINVAL. */
int lbm_set_omega(lbm_ctx* ctx, double omega);

/*
 * lbm_set_variant - choose the stream-collide kernel (same arithmetic, bitwise
 * identical results):
 *   0 (default) the measured fastest for the context's form (see lbm_step);
 *   1 direct gather: one thread per cell loads its Q populations from HBM;
 *   2 TMA: persistent CTAs of 128 threads; warp 0 streams the Q shifted source row
 *     segments of each 128-cell chunk into a ring of shared-memory stages with bulk
 *     asynchronous copies (full / empty mbarrier pipeline), the threads read their
 *     populations at compile-time offsets, and in the FP16 / BF16 forms the
 *     results leave through a shared-memory tile and bulk stores.  Every wait is
 *     bounded (1 s); a timeout sets the status that lbm_synchronize reports as
 *     LBM_EDEVICE.  Needs Nx % 8 == 0;
 *   3 split: the directions of each cell are divided between two warps that
 *     exchange partial moments through shared memory (half the registers per
 *     thread, twice the resident warps).  FP32 / FP16 / BF16 forms only.
 * Errors: LBM_EINVAL, LBM_ECUDA (set-up of the TMA kernel).
 */
int lbm_set_variant(lbm_ctx* ctx, int variant);

/*
 * lbm_set_graph_steps (execution control; the paper has no counterpart) -
 * lbm_step replays runs of `steps` launches from a CUDA
 * graph (captured on a stream the library owns, by this call for both starting
 * buffers and again on the first lbm_step after a change that invalidates them,
 * and launched on the context's stream) whenever
 * the default direct kernel is in use and at least 2 * steps steps are asked for;
 * the remainder is launched directly.  Results are bitwise those of direct
 * launches.  steps: 0 (launch every step directly) or an even number <= 4096;
 * default 32.  A graph is recaptured after lbm_set_omega, lbm_set_variant or
 * lbm_set_fixed_ends.  Do not call lbm_step while another thread captures the
 * context's stream.  If a capture fails the context falls back to direct launches
 * (this call then returns LBM_ECUDA).  Errors: LBM_EINVAL, LBM_ECUDA.
 */
int lbm_set_graph_steps(lbm_ctx* ctx, int steps);

/*
 * lbm_set_fixed_ends - the end conditions of the paper's shock tube (paragraph
 * before Figure 1: the left and right boundary planes carry the fixed states C_L
 * and C_R).  After every later lbm_step the first and the last `width` planes
 * along `axis` (0 x, 1 y, 2 z) are set to the discrete equilibrium of state `lo`
 * and `hi`; the other axes stay periodic.  States are {rho, U_1..U_D, T} in
 * lattice units (host arrays of D + 2 doubles).  width must be at least the
 * stencil reach (4 for D2Q33, 5 for D3Q95), so that no other cell gathers across
 * the ends, and at most N/2; width 0 switches the ends off.  Not covered by the
 * adjoint: lbm_record / lbm_record_bounded return LBM_EINVAL while active.
 * Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA.
 */
int lbm_set_fixed_ends(lbm_ctx* ctx, int axis, int width, const double* lo, const double* hi);

/* lbm_set_stream - order later calls on another stream of the same device. */
int lbm_set_stream(lbm_ctx* ctx, void* stream);

/*
 * lbm_init - set every cell to the discrete equilibrium f_i^eq(rho, U, T): the
 * fourth-order Hermite expansion of the Maxwellian (the distribution stated after
 * the update rule) on the model's weights, i.e. Formula 1's moment conditions
 * with m = N = 4, in the dimensionless variables theta = T / T0, u = c U
 * defined after the Maxwellian.
 *   rho [cells], U [D][cells] (lattice units), T [cells] (lattice units),
 *   all FP64 in `where` memory.  rho > 0 and T > 0 and all values finite:
 *   LBM_HOST inputs are uploaded in chunks (large grids: 8) on a stream of the
 *   context's own, each chunk checked on the device and turned into its
 *   equilibrium while the next one uploads (pinned host memory lets the copies
 *   overlap); the equilibrium is written to the population buffer that does not
 *   hold the live state, which it replaces only when every value has passed the
 *   check (one blocking read of the check's result).  A refused call leaves the
 *   populations as they were but invalidates a recorded rollout.  LBM_DEVICE
 *   inputs are not inspected (the call stays asynchronous).  The fields are also kept on the device as the
 *   initial state of the differentiable rollout (lbm_record / lbm_backward).
 * Errors: LBM_EINVAL, LBM_ECUDA.
 */
int lbm_init(lbm_ctx* ctx, const double* rho, const double* U, const double* T, int where);

/*
 * lbm_step - advance n >= 0 time steps of the paper's update (the BGK rule stated
 * before the Maxwellian), one fused stream-collide kernel per step, replayed from
 * CUDA graphs in runs of lbm_set_graph_steps steps.  Enqueues and returns, except
 * that with lbm_set_audit_every it blocks at each audit.  Errors: LBM_ESTATE
 * before lbm_init, LBM_EINVAL, LBM_ECUDA, LBM_EUNSTABLE (audit tripped).
 */
int lbm_step(lbm_ctx* ctx, int64_t n);

/* lbm_steps_done - number of steps taken since the last lbm_init / set. */
int64_t lbm_steps_done(const lbm_ctx* ctx);

/*
 * lbm_moments - macroscopic fields of the current state (Formula 1, n <= 2):
 *   rho = sum f_i, rho U = sum f_i e_i, D rho T = sum f_i |e_i - U|^2.
 *   FP64 form: summed in FP64.  FP32 / FP16 / BF16 forms: the collision's own
 *   sums of the deviations (rho - 1 and E - D rho compensated, as double-float),
 *   fields formed in FP32 (relative error ~1e-7 of the stored state's exact
 *   fields).  Outputs rho [cells], U [D][cells], T [cells] as FP64 in `where`
 *   memory; any output may be NULL.  LBM_DEVICE: enqueued on the context's
 *   stream.  LBM_HOST: computed in chunks (large grids: 8), each read back on the
 *   context's copy stream while the next is computed; returns once the host
 *   arrays are filled (pinned host memory lets the copies overlap).
 * Errors: LBM_ESTATE, LBM_EINVAL, LBM_ECUDA.
 */
int lbm_moments(lbm_ctx* ctx, double* rho, double* U, double* T, int where);

/*
 * lbm_set_audit_every (failure detection; the paper has none) - with k > 0, lbm_step
 * runs the conservation audit (lbm_audit) whenever the step count reaches a
 * multiple of k (one blocking read-back each time) and stops with
 * LBM_EUNSTABLE as soon as a population is non-finite; the steps done so far
 * stay done (lbm_steps_done) and the state is kept for inspection.  k = 0 (the
 * default) audits nothing.  Errors: LBM_EINVAL.
 */
int lbm_set_audit_every(lbm_ctx* ctx, int64_t k);

/*
 * lbm_save / lbm_load - checkpoint and resume (the paper has no counterpart).
 * lbm_save writes a header (magic
 * "LBMSTATE", version 1, model, storage, Q, element size, Nx, Ny, Nz, omega, step
 * count; little-endian as the host writes it) followed by the stored deviations
 * exactly as lbm_get_raw returns them.  lbm_load reads such a file into a context
 * of the same model, storage and grid, restores omega and the step count, and
 * continues bit for bit as the saved run would have.  Blocking; the state moves
 * through host memory in 64 MiB pieces.  The initial fields of a recorded rollout
 * are not part of the file (lbm_load invalidates a recording).  lbm_load checks
 * the file's length against the context's state before it uploads anything and
 * uploads into the spare ping-pong buffer, switching to it only after the last
 * piece: a refused or failed load leaves the context's state, omega and step
 * count as they were.
 * Errors: LBM_EINVAL (NULL, foreign or mismatched file), LBM_ESTATE (save before
 * init), LBM_EIO (open, short read or write, wrong file length), LBM_ECUDA.
 */
int lbm_save(lbm_ctx* ctx, const char* path);
int lbm_load(lbm_ctx* ctx, const char* path);

/*
 * lbm_audit - conservation audit of the current state, deterministic (fixed
 * reduction order): per-block sums in FP64 (FP64 form) or double-float (other
 * forms, ~44 significant bits), blocks summed in FP64.  out[8] (host) receives:
 *   [0] mass = sum_x sum_i f_i        [1..3] momentum sum f_i e_i (zero-padded)
 *   [4] energy = sum f_i |e_i|^2 / 2  [5] min over populations of f_i / w_i
 *   [6] number of non-finite populations  [7] number of cells
 * Returns LBM_EUNSTABLE (after filling out) if any population is non-finite.
 */
int lbm_audit(lbm_ctx* ctx, double out[8]);

/*
 * lbm_get_populations / lbm_set_populations - the state as physical FP64
 * populations f [Q][cells] (f_i = w_i (1 + h_i)).  set encodes to the storage
 * form (round to nearest even) and resets the step counter.
 */
int lbm_get_populations(lbm_ctx* ctx, double* f, int where);
int lbm_set_populations(lbm_ctx* ctx, const double* f, int where);

/*
 * lbm_get_raw / lbm_set_raw - the stored deviations h [Q][cells] bit for bit
 * in the storage type (8, 4, 2 or 2 bytes per element); bytes = Q*cells*size.
 * Used for the integer-label streaming check and for saving / restoring state.
 */
int lbm_get_raw(lbm_ctx* ctx, void* h, size_t bytes, int where);
int lbm_set_raw(lbm_ctx* ctx, const void* h, size_t bytes, int where);

/*
 * lbm_record - the forward half of the differentiable rollout
 * (rho0, U0, T0, omega) -> state after nsteps.  Re-initialises from the
 * fields of the last lbm_init, runs nsteps >= 1 steps, and keeps every
 * ckpt_every-th state (1 <= ckpt_every) as a checkpoint for lbm_backward.
 * Checkpoint memory: ceil(nsteps / ckpt_every) states.
 * Errors: LBM_ESTATE (no lbm_init), LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA.
 */
int lbm_record(lbm_ctx* ctx, int64_t nsteps, int64_t ckpt_every);

/*
 * lbm_record_bounded - the same forward as lbm_record, for grids whose uniform
 * checkpoints do not fit: only S_0 is kept.  The reverse sweep of lbm_backward
 * then stores at most max_states >= 1 states (S_0 included), each placed where
 * it minimises the forward steps recomputed (binomial checkpointing: a dynamic
 * programme over the split points, built on the host by this call when
 * nsteps^2 (max_states - 1) <= 2e8, else recursive bisection); ranges deeper
 * than the budget are recomputed from their nearest stored state.  E.g. 7 states
 * (S_0 and 6 more) for 300 steps recompute 1035 forward steps (bisection: 1191).
 * The context's
 * two population buffers serve as work space: after such
 * a backward the context holds S_0 (steps done = 0).  Gradients are bitwise
 * identical to the uniform schedule's.
 * Errors: LBM_ESTATE (no lbm_init), LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA.
 */
int lbm_record_bounded(lbm_ctx* ctx, int64_t nsteps, int64_t max_states);

/*
 * lbm_backward - reverse sweep of the recorded rollout: the exact discrete
 * adjoint of the stream-collide update (transposed collision Jacobian through
 * f^eq, then reverse streaming), recomputing each segment of ckpt_every
 * states from its checkpoint.
 *   dL_drhoN [cells]: gradient of the loss with respect to the final density.
 *   Outputs (any may be NULL): dL_drho0 [cells], dL_dU0 [D][cells],
 *   dL_dT0 [cells] (lattice units), dL_domega (one double, host memory).
 * Arrays are FP64 in `where` memory.  The adjoint runs in FP64 for LBM_FP64
 * contexts and FP32 otherwise.  The recorded trajectory is kept (the call may
 * be repeated with another dL_drhoN); the current state is restored to the
 * final state of the rollout.
 * Errors: LBM_ESTATE (nothing recorded), LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA.
 */
int lbm_backward(lbm_ctx* ctx, const double* dL_drhoN, double* dL_drho0, double* dL_dU0,
                 double* dL_dT0, double* dL_domega, int where);

/* lbm_release_record - free the checkpoints and segment buffers. */
int lbm_release_record(lbm_ctx* ctx);

/* lbm_synchronize - wait for all work on the context's stream; LBM_EDEVICE if
 * a kernel of the context reported a timed-out wait. */
int lbm_synchronize(lbm_ctx* ctx);

/*
 * Domain decomposition (the streaming term of the update couples neighbouring
 * cells, so a grid split into slabs needs their boundary populations every step).
 * A grid is split along its slowest axis (z for D3Q95, y for D2Q33) into slabs
 * of consecutive planes; each slab is a context of its own whose state holds R
 * ghost planes on each side of its interior planes (R = stencil reach, 5 / 4):
 * local plane p in [0, R) is a ghost below, [R, R + n) the interior, and
 * [R + n, n + 2R) a ghost above.  The slab steps as a periodic box over its whole
 * local array: interior cells gather only within [0, n + 2R), never across its
 * ends, so they update exactly as in the undivided grid provided the ghost planes
 * hold the neighbours' populations; ghost planes are recomputed from wrapped data
 * and are overwritten before they are read again.  After every step each slab
 * packs, per face, the populations its neighbour across that face gathers (for
 * every direction with component c > 0 along the axis its top c interior planes
 * go up; c < 0 the bottom |c| planes go down: 102 plane-populations per face for
 * D3Q95, 26 for D2Q33), the message travels by any device-to-device transport
 * (a copy, NCCL send / recv), and the neighbour unpacks it into its ghost planes.
 * The last slab's upper neighbour is the first slab (periodic grid).
 *
 * lbm_create_slab - like lbm_create for a slab whose interior is dims (with
 *   dims[2] (D3Q95) or dims[1] (D2Q33) the slab's own number of planes, at least
 *   R); the context's grid, and every field or population array passed to it
 *   (lbm_init, lbm_moments, lbm_get_raw ...), has R more planes on each side along
 *   the split axis.  lbm_record and lbm_backward refuse slab contexts.
 * lbm_halo_info - ghost planes per side R, interior planes n, segments per
 *   message (one segment = one direction's plane) and bytes per message.
 * lbm_halo_pack(face) - write into the device buffer `buf` (lbm_halo_info's bytes)
 *   the message for the neighbour across `face` (0 below, 1 above), from the
 *   current state; lbm_halo_unpack(face) - store the message received from the
 *   neighbour across `face` into this slab's ghost planes on that side.  Both are
 *   ordered on the context's stream and return after enqueueing.
 * lbm_halo_plan - the message layout (host only, needs no GPU): the `count`
 *   (direction, local plane) pairs a slab with `interior` planes sends across
 *   `face` (send = 1) or receives there (send = 0), in message order; segs may be
 *   NULL to query count.  Segment j occupies elements [j P, (j + 1) P) of the
 *   message, P = Nx Ny (D3Q95) or Nx (D2Q33).
 * Errors: LBM_EINVAL, LBM_ESTATE (not a slab, no state), LBM_ENOMEM, LBM_ECUDA.
 */
int lbm_create_slab(lbm_ctx** out, int model, const int64_t dims[3], double omega, int storage,
                    void* stream);
int lbm_halo_info(const lbm_ctx* ctx, int* ghost, int64_t* interior, int* segments,
                  size_t* face_bytes);
int lbm_halo_pack(lbm_ctx* ctx, int face, void* buf);
int lbm_halo_unpack(lbm_ctx* ctx, int face, const void* buf);
int lbm_halo_plan(int model, int64_t interior, int face, int send, int32_t* segs, int* count);

/*
 * lbm_test_stall (test hook of the failure detection; the paper has no
 * counterpart) - the next TMA stream-collide launch of this context (variant 2
 * must be selected) skips the copies of chunk `chunk` (128 cells of one x-row,
 * chunks numbered x-segment fastest, then y, then z) and bounds every wait by
 * limit_ns nanoseconds (1 us .. 2 s).  The consumers of that chunk wait for
 * copies that never come, give up after limit_ns, set the device status and
 * stop; lbm_synchronize then returns LBM_EDEVICE once (and clears the status).
 * Nothing faults and nothing waits without a bound; the state of that step is
 * incomplete, so reinitialise it afterwards.  That launch is made directly, not
 * from a CUDA graph.  Errors: LBM_EINVAL, LBM_ESTATE (TMA variant not selected).
 */
int lbm_test_stall(lbm_ctx* ctx, int64_t chunk, int64_t limit_ns);

/* lbm_launch_count - kernels this context has launched so far. */
int64_t lbm_launch_count(const lbm_ctx* ctx);

/*
 * lbm_audit_noalloc - the conservation audit of lbm_audit for a caller-owned
 * population array, allocating no device memory.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc, such as
 * code whose device memory belongs in full to another allocator (a framework's
 * pool that has reserved the GPU) or code in a time loop that cannot take the
 * device-wide synchronisation cudaMalloc / cudaFree may cause.
 *   model, storage, dims: as for lbm_create (the layout lbm_get_raw returns);
 *   h:      device pointer (current device) to the stored deviations, Q * cells
 *           elements;
 *   h_bytes: size of the buffer at h; less than Q * cells * element size is
 *           refused;
 *   out:    device pointer (current device) to 8 doubles, filled as lbm_audit's
 *           out (no host copy);
 *   stream: cudaStream_t the work is ordered on (NULL = legacy default stream).
 * h and out are checked with cudaPointerGetAttributes (no allocation): host or
 * another device's memory returns LBM_EINVAL without a launch.
 * The per-block partial sums live in one file-scope device array of 8192 x 8
 * doubles (512 KiB, held by every GPU that loads the library until the process
 * exits), so grids of at most 2,097,152 cells are accepted; larger grids return
 * LBM_EINVAL.  The first call on a device does a set-up with that device
 * current (the array's device address and the constant model tables); make
 * that first call before any stream capture.  A device reset destroys what the
 * set-up made; the first call after it repeats the set-up (it is keyed by the
 * CUDA context's id), so make that call before any capture too.  All calls share the array:
 * calls whose work overlaps on the GPU (other streams, other threads) race.
 * Each call overwrites every partial it reads, so nothing needs clearing.
 * Returns after enqueueing.  Errors: LBM_EINVAL, LBM_ECUDA.
 */
int lbm_audit_noalloc(int model, int storage, const int64_t dims[3], const void* h,
                      size_t h_bytes, double* out, void* stream);

/*
 * lbm_equation_count - Omega(m, D), the number of moment equations of Formula 5
 * up to n_max = 2m for the m-th order Hermite equilibrium (Formulas 6-8, Table 1),
 * from the generating function of partitions into at most D parts (Formula 7).
 *   m in [0, 7], D in [1, 4]; *out receives the count.  Host only.
 * Errors: LBM_EINVAL.
 */
int lbm_equation_count(int m, int D, int64_t* out);

/*
 * lbm_generate_model - an on-lattice isotropic velocity set of order m in D
 * dimensions (Formulas 4, 5, 9, 10): each representative expands into its orbit
 * under coordinate permutations and sign changes (the groups G_k before
 * Formula 9, one weight per orbit), and the group weights and the scale c solve
 * Formula 5 up to n_max = 2m.  Host only; needs no GPU.
 *   D in [1, 4], m in [0, 7];
 *   reps:    [ngroups][D] integers in [-8, 8] (signs and order do not matter),
 *            ngroups = Omega(m, D) - 1 (Formula 10), distinct orbits;
 *   which:   index among the solutions with all weights positive, by increasing c;
 *   qmax:    capacity of e / w in velocities;
 *   Q:       (out) the number of velocities, set even when qmax is too small;
 *   e, w:    (out, may be NULL) velocities [Q][D] (integer lattice vectors, orbit
 *            by orbit in the order of reps, each orbit in decreasing lexicographic
 *            order) and their weights [Q] (sum w = 1);
 *   c:       (out) the lattice scale, v_i = c e_i;
 *   residual:(out, may be NULL) max |Formula 5 residual| (normalised moments);
 *   nsolutions: (out, may be NULL) number of solutions with positive weights.
 * Method: for fixed 1/c^2 the equations are linear in the weights with one
 * equation more than unknowns; the positive roots of the determinant of the
 * augmented system (a polynomial of degree <= m in 1/c^2) are bracketed and
 * bisected, the weights follow by least squares, and Newton's method on the full
 * system polishes (W, c).  Errors: LBM_EINVAL (Formula 10 not met, repeated orbit,
 * entry out of range, qmax too small, no solution with positive weights, which
 * out of range).
 */
int lbm_generate_model(int D, int m, int ngroups, const int* reps, int which, int qmax, int* Q,
                       int* e, double* w, double* c, double* residual, int* nsolutions);

/* lbm_strerror - static text for an error code; lbm_last_error - detail of
 * the last failure on the calling thread (empty string if none). */
const char* lbm_strerror(int code);
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */

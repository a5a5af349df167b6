// lbm_api.cu - host side of the C ABI declared in include/lbm.h.
//
// Holds the model tables (velocity sets expanded at compile time in
// velset.cuh, weights solved here from Formula 5), the context object with its
// ping-pong population buffers, argument validation and the launch sequences.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "common.h"
#include "velset.cuh"
#include "adjoint.h"

using namespace lbm;

// ================================================================ errors
namespace {
thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LBM_CUDA(call)                                     \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
}  // namespace

// ================================================================ model tables (Formula 5)
namespace {

// Printed weights (Tables 2 and 3) and c: the Newton start point.
const double kStartD2Q33[8] = {0.161987, 0.143204, 0.0338840, 0.00556112,
                               8.44799e-5, 0.00113254, 0.0128169, 3.45552e-6};
const double kStartCD2Q33 = 0.819381;
const double kStartD3Q95[10] = {0.206847, 0.00442257, 0.0333341, 0.0128902, 0.0287920,
                                0.00264319, 0.000927908, 0.00106078, 0.000804376, 0.00274697};
const double kStartCD3Q95 = 0.421803;

struct HostModel {
  VelSet vs;
  double W[kMaxG];
  double c;
  double residual;
  double w[kMaxQ];
  ModelConst mc;
};

double dfact_odd(int n) {  // (n-1)!! for even n >= 0
  double r = 1.0;
  for (int k = n - 1; k > 1; k -= 2) r *= k;
  return r;
}

// Normalised Gaussian moment prod_a (a-1)!!/2^(a/2): Formula 4 divided by pi^(D/2).
double gauss_norm(const int a[3]) {
  double r = 1.0;
  for (int k = 0; k < 3; ++k) r *= dfact_odd(a[k]) / std::pow(2.0, a[k] / 2);
  return r;
}

// Exponent classes of Formula 5 up to n_max = 8: doubled partitions of q <= 4
// into at most D parts (Formula 8 counts them: 9 for D = 2, 11 for D = 3).
void partitions_rec(int q, int maxpart, int parts_left, std::vector<int>& cur,
                    std::vector<std::vector<int>>* out) {
  if (q == 0) {
    out->push_back(cur);
    return;
  }
  if (parts_left == 0) return;
  for (int p = (q < maxpart ? q : maxpart); p >= 1; --p) {
    cur.push_back(p);
    partitions_rec(q - p, p, parts_left - 1, cur, out);
    cur.pop_back();
  }
}

bool solve_dense(std::vector<double>& A, std::vector<double>& b, int n) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[r * n + col]) > std::fabs(A[piv * n + col])) piv = r;
    if (A[piv * n + col] == 0.0) return false;
    if (piv != col) {
      for (int k = 0; k < n; ++k) std::swap(A[col * n + k], A[piv * n + k]);
      std::swap(b[col], b[piv]);
    }
    for (int r = col + 1; r < n; ++r) {
      const double f = A[r * n + col] / A[col * n + col];
      for (int k = col; k < n; ++k) A[r * n + k] -= f * A[col * n + k];
      b[r] -= f * b[col];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
  return true;
}

bool build_host_model(int model, HostModel* hm) {
  hm->vs = model == 0 ? make_velset<0>() : make_velset<1>();
  const VelSet& vs = hm->vs;
  const int G = vs.G, D = vs.D, n = G + 1;
  // equations
  std::vector<std::vector<int>> parts;
  for (int q = 0; q <= 4; ++q) {
    std::vector<int> cur;
    partitions_rec(q, q, D, cur, &parts);
  }
  if ((int)parts.size() != n) return false;  // Formula 10: equations == unknowns
  std::vector<double> Mg(parts.size() * G, 0.0), rhs(parts.size()), nn(parts.size());
  for (size_t k = 0; k < parts.size(); ++k) {
    int a[3] = {0, 0, 0};
    for (size_t j = 0; j < parts[k].size(); ++j) a[j] = 2 * parts[k][j];
    rhs[k] = gauss_norm(a);
    nn[k] = a[0] + a[1] + a[2];
    for (int i = 0; i < vs.Q; ++i) {
      double p = 1.0;
      for (int d = 0; d < 3; ++d)
        for (int r = 0; r < a[d]; ++r) p *= vs.e[i][d];
      Mg[k * G + vs.grp[i]] += p;
    }
  }
  std::vector<double> x(n);
  for (int g = 0; g < G; ++g) x[g] = model == 0 ? kStartD2Q33[g] : kStartD3Q95[g];
  x[G] = model == 0 ? kStartCD2Q33 : kStartCD3Q95;
  auto residual = [&](const std::vector<double>& xv, std::vector<double>* F) {
    double mx = 0;
    for (int k = 0; k < n; ++k) {
      double s = 0;
      for (int g = 0; g < G; ++g) s += Mg[k * G + g] * xv[g];
      (*F)[k] = s * std::pow(xv[G], nn[k]) - rhs[k];
      mx = std::fmax(mx, std::fabs((*F)[k]));
    }
    return mx;
  };
  std::vector<double> F(n), J(n * n);
  for (int it = 0; it < 60; ++it) {
    residual(x, &F);
    for (int k = 0; k < n; ++k) {
      double s = 0;
      for (int g = 0; g < G; ++g) {
        J[k * n + g] = Mg[k * G + g] * std::pow(x[G], nn[k]);
        s += Mg[k * G + g] * x[g];
      }
      J[k * n + G] = nn[k] > 0 ? s * nn[k] * std::pow(x[G], nn[k] - 1) : 0.0;
    }
    std::vector<double> dx(n);
    for (int k = 0; k < n; ++k) dx[k] = -F[k];
    if (!solve_dense(J, dx, n)) return false;
    double step = 0;
    for (int k = 0; k < n; ++k) {
      x[k] += dx[k];
      step = std::fmax(step, std::fabs(dx[k]));
    }
    if (step < 1e-17) break;
  }
  hm->residual = residual(x, &F);
  for (int g = 0; g < G; ++g) hm->W[g] = x[g];
  hm->c = x[G];
  for (int i = 0; i < vs.Q; ++i) hm->w[i] = hm->W[vs.grp[i]];

  ModelConst& mc = hm->mc;
  std::memset(&mc, 0, sizeof mc);
  const double a = std::sqrt(2.0) * hm->c;
  for (int g = 0; g < G; ++g) {
    mc.W[g] = hm->W[g];
    mc.X2[g] = a * a * vs.e2[g];
    mc.Wf[g] = (float)mc.W[g];
    mc.X2f[g] = (float)mc.X2[g];
    mc.X2lo[g] = (float)(mc.X2[g] - (double)mc.X2f[g]);
  }
  for (int i = 0; i < vs.Q; ++i) {
    mc.w[i] = hm->w[i];
    for (int d = 0; d < 3; ++d) {
      mc.e[i][d] = vs.e[i][d];
      mc.ef[i][d] = (float)vs.e[i][d];
    }
  }
  mc.a = a;
  mc.af = (float)a;
  mc.alo = (float)(a - (double)mc.af);
  mc.c = hm->c;
  mc.T0 = 1.0 / (2.0 * hm->c * hm->c);
  mc.T0f = (float)mc.T0;
  mc.iT0f = (float)(2.0 * hm->c * hm->c);
  mc.iT0lo = (float)(2.0 * hm->c * hm->c - (double)mc.iT0f);
  return hm->residual < 1e-13;
}

std::mutex g_model_mu;
HostModel g_models[2];
bool g_model_ok[2] = {false, false};
// (device, context id) pairs whose constant tables are current
std::vector<std::pair<int, unsigned long long>> g_uploaded;

const HostModel* host_model(int model) {
  std::lock_guard<std::mutex> lk(g_model_mu);
  if (!g_model_ok[model]) {
    if (!build_host_model(model, &g_models[model])) return nullptr;
    g_model_ok[model] = true;
  }
  return &g_models[model];
}

const StorageOps* ops_for(int storage) {
  switch (storage) {
    case LBM_FP64: return &kOpsFP64;
    case LBM_FP32: return &kOpsFP32;
    case LBM_FP16DEV: return &kOpsFP16;
    case LBM_BF16DEV: return &kOpsBF16;
    default: return nullptr;
  }
}

int ensure_uploaded(int dev) {
  const HostModel* m0 = host_model(0);
  const HostModel* m1 = host_model(1);
  if (!m0 || !m1) return fail(LBM_EINVAL, "model table solve failed");
  std::lock_guard<std::mutex> lk(g_model_mu);
  const unsigned long long id = lbm::current_context_id();
  for (const auto& u : g_uploaded)
    if (u.first == dev && u.second == id && id != 0) return LBM_OK;
  ModelConst both[2] = {m0->mc, m1->mc};
  const StorageOps* all[4] = {&kOpsFP64, &kOpsFP32, &kOpsFP16, &kOpsBF16};
  for (auto* o : all) {
    cudaError_t e = o->upload(both);
    if (e != cudaSuccess) return cuda_fail(e, "constant table upload");
  }
  // the upload made the device's primary context current: record its id
  const unsigned long long now = lbm::current_context_id();
  g_uploaded.erase(std::remove_if(g_uploaded.begin(), g_uploaded.end(),
                                  [dev](const std::pair<int, unsigned long long>& u) {
                                    return u.first == dev;
                                  }),
                   g_uploaded.end());
  g_uploaded.push_back({dev, now});
  return LBM_OK;
}

// ================================================================ slab halo plan
// The (direction, local plane) segments a slab with `nl` interior planes sends
// across `face` (0: towards lower coordinates along the split axis, 1: higher), or
// receives there (send = 0), in direction order and, within a direction, in
// increasing plane order, so that a sender's list and its neighbour's list for the
// same message match entry by entry.  Local planes count from the first ghost
// plane: ghosts [0, R), interior [R, R + nl), ghosts [R + nl, nl + 2R).  A
// direction with component c > 0 along the split axis pulls from c planes below:
// the sender's top c interior planes of it travel across face 1 and fill the
// receiver's ghost planes R - c .. R - 1; c < 0 mirrors that across face 0.
void halo_plan_host(const VelSet& vs, int64_t nl, int face, int send, std::vector<int32_t>* segs) {
  const int axis = vs.D == 3 ? 2 : 1;
  const int R = vs.R;
  // directions crossing this face in this message: upwards (c > 0) for what goes
  // out of face 1 or comes in at face 0, downwards (c < 0) otherwise
  const bool up = (face == 1) == (send != 0);
  segs->clear();
  for (int i = 0; i < vs.Q; ++i) {
    const int c = vs.e[i][axis];
    if (up ? c <= 0 : c >= 0) continue;
    const int a = up ? c : -c;
    for (int m = 0; m < a; ++m) {
      int64_t plane;
      if (face == 1) plane = send ? R + nl - a + m : R + nl + m;
      else plane = send ? R + m : R - a + m;
      segs->push_back(i);
      segs->push_back((int32_t)plane);
    }
  }
}

// ================================================================ allocation
std::mutex g_alloc_mu;
lbm_alloc_fn g_alloc = nullptr;
lbm_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;

}  // namespace

namespace lbm {

DevBuf::~DevBuf() { release(); }

void DevBuf::release() {
  if (!p) return;
  if (free_fn) free_fn(p, stream, user);
  else cudaFree(p);
  p = nullptr;
  bytes = 0;
}

int DevBuf::ensure(size_t nbytes, cudaStream_t st) {
  if (p && bytes >= nbytes) return LBM_OK;
  release();
  if (nbytes == 0) return LBM_OK;
  lbm_alloc_fn a;
  lbm_free_fn f;
  void* u;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
    f = g_free;
    u = g_alloc_user;
  }
  if (a) {
    p = a(nbytes, (void*)st, u);
    if (!p) return fail(LBM_ENOMEM, "allocator returned NULL for %zu bytes", nbytes);
    free_fn = f;
    user = u;
    stream = (void*)st;
  } else {
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return fail(LBM_ENOMEM, "cudaMalloc(%zu): %s", nbytes, cudaGetErrorString(e));
    }
    free_fn = nullptr;
  }
  bytes = nbytes;
  return LBM_OK;
}

}  // namespace lbm

// ================================================================ context
// Steps replayed from a CUDA graph: kGraphSteps launches (an even count, so a replay
// leaves the ping-pong buffers where it found them) captured once per context on a
// library-owned stream and launched on the caller's stream.  One graph per starting
// buffer; recaptured when omega, the kernel variant or the end planes change.
constexpr int kGraphSteps = 32;
struct StepGraph {
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  void reset() {
    for (auto& e : exec)
      if (e) {
        cudaGraphExecDestroy(e);
        e = nullptr;
      }
  }
};

// lbm_init from host fields and lbm_moments to host arrays move their data in chunks
// on a second stream, so that the copy of one chunk overlaps the kernels of the next
// (below this many cells: one chunk).
constexpr int kXferChunks = 8;
constexpr long long kXferMinCells = 1 << 20;

struct lbm_ctx {
  ~lbm_ctx() {
    graph.reset();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (cudaEvent_t& e : xfer_ev)
      if (e) cudaEventDestroy(e);
    if (xfer_stream) cudaStreamDestroy(xfer_stream);
  }
  int model = 0, storage = 0, dev = 0, D = 0, Q = 0;
  const StorageOps* ops = nullptr;
  Grid g{};
  double omega = 1.0;
  cudaStream_t stream = nullptr;
  DevBuf state[2];
  int cur = 0;
  DevBuf fields;      // initial rho | U (D) | T, FP64
  DevBuf mom;         // host-output staging for moments / populations
  DevBuf partials;    // audit block partials
  DevBuf audit_out;   // 8 doubles
  DevBuf status;      // device int: 1 after a kernel gave up on a bounded wait
  DevBuf check;       // device word: first invalid initial field value (lbm_init)
  int variant = 0;    // 0 auto, kVariantDirect, kVariantTma, kVariantSplit
  StepTest test{-1, 0};  // lbm_test_stall: applies to the next TMA launch only
  bool test_pending = false;
  int fix_axis = 0, fix_width = 0;   // fixed-state end planes (width 0: none)
  DevBuf fix_tmpl;    // [Q][2] populations of the two end states
  bool inited = false;
  int64_t steps = 0;
  int64_t launches = 0;
  Record rec;         // checkpointed rollout (adjoint.h)
  int graph_steps = kGraphSteps;   // 0: launch every step directly
  StepGraph graph;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t xfer_stream = nullptr;          // chunked host copies (lbm_init, lbm_moments)
  cudaEvent_t xfer_ev[kXferChunks + 1] = {};   // per chunk, and the start
  int64_t audit_every = 0;         // lbm_step audits after every multiple of this many steps
  double audit_host[kAuditSlots] = {0};
  // slab of a decomposed grid (lbm_create_slab): split axis (2 z, 1 y; -1 none),
  // interior planes, ghost planes per side, and the four segment lists
  // [send low | send high | recv low | recv high] on the device, nseg each
  int slab_axis = -1;
  int64_t slab_interior = 0;
  int slab_ghost = 0;
  int halo_nseg = 0;
  DevBuf halo_segs;
};

namespace {

size_t state_bytes(const lbm_ctx* c) {
  return (size_t)c->Q * (size_t)c->g.ncell * (size_t)c->ops->elem_bytes;
}

bool all_finite(const double* p, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(p[k])) return false;
  return true;
}

// Default kernel (measured on GB300): the two-cell pair kernel for the 16-bit
// D2Q33 forms (+19 % over the direct gather at 4096 x 2048), the one-cell direct
// gather everywhere else (for D3Q95 a two-cell update needs ~255 registers and the
// SM then holds too few warps to cover the gather's latency).
int pick_variant(const lbm_ctx* c) {
  if (c->variant != 0) return c->variant;
  if (c->model == LBM_D2Q33 && c->ops->elem_bytes == 2 && pair_applicable(c->g)) return kVariantPair;
  return kVariantDirect;
}

// n steps enqueued on stream st starting from buffer *cur (which is advanced).
cudaError_t enqueue_steps(lbm_ctx* c, int64_t n, int variant, int* cur, cudaStream_t st) {
  for (int64_t k = 0; k < n; ++k) {
    // steps out of buffer 1 walk the grid backwards (kStepReverse): consecutive steps
    // alternate direction and each starts on its predecessor's L2-resident output.
    // Only for states of at most twice the L2 (129 MB); on large grids the reuse is
    // negligible and the descending walk measured ~1 % slower.
    const bool alt = state_bytes(c) <= ((size_t)256 << 20);
    const bool walks = variant == kVariantDirect || variant == kVariantPair;
    const int v = variant | ((alt && walks && *cur == 1) ? kStepReverse : 0);
    const StepTest* t = nullptr;
    if (c->test_pending && variant == kVariantTma) {
      t = &c->test;
      c->test_pending = false;
    }
    cudaError_t e = c->ops->step(c->model, c->state[*cur].p, c->state[*cur ^ 1].p, c->g, c->omega,
                                 v, static_cast<int*>(c->status.p), t, st);
    if (e != cudaSuccess) return e;
    *cur ^= 1;
    if (c->fix_width > 0) {
      e = c->ops->fix_ends(c->state[*cur].p, c->g, c->fix_axis, c->fix_width, c->fix_tmpl.p, c->Q,
                           st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Capture kGraphSteps steps starting from buffer `parity`.  False (and graphs off for
// this context) if capture or instantiation fails; the caller then launches directly.
bool capture_steps(lbm_ctx* c, int parity, int variant) {
  if (variant == kVariantTma && c->ops->prepare_tma(c->model) != cudaSuccess) {
    cudaGetLastError();
    c->graph_steps = 0;
    return false;
  }
  if (!c->cap_stream &&
      cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->graph_steps = 0;
    return false;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    int cur = parity;
    const cudaError_t le = enqueue_steps(c, c->graph_steps, variant, &cur, c->cap_stream);
    e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph.exec[parity], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->graph.exec[parity] = nullptr;
    c->graph_steps = 0;
    return false;
  }
  return true;
}

int do_steps(lbm_ctx* c, int64_t n) {
  const int variant = pick_variant(c);
  const int64_t per_step = c->fix_width > 0 ? 2 : 1;
  int64_t done = 0;
  if (c->graph_steps > 0 && !c->test_pending && n >= 2 * c->graph_steps &&
      (c->graph.exec[c->cur] || capture_steps(c, c->cur, variant))) {
    for (; n - done >= c->graph_steps; done += c->graph_steps) {
      cudaError_t e = cudaGraphLaunch(c->graph.exec[c->cur], c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "step graph launch");
      c->launches += per_step * c->graph_steps;
    }
  }
  cudaError_t e = enqueue_steps(c, n - done, variant, &c->cur, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream_collide launch");
  c->launches += per_step * (n - done);
  c->steps += n;
  return LBM_OK;
}

}  // namespace

// ---------------------------------------------------------------- internal hooks for adjoint.cu
namespace lbm {
unsigned long long current_context_id() {
  // driver entry points looked up through the runtime once (no link to libcuda)
  using GetCurrentFn = CUresult (*)(CUcontext*);
  using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetIdFn>(f);
    cudaGetLastError();
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int ctx_fail(int code, const char* msg) { return fail(code, "%s", msg); }
int ctx_cuda_fail(cudaError_t e, const char* what) { return cuda_fail(e, what); }
const ModelConst* ctx_model_const(int model) {
  const HostModel* m = host_model(model);
  return m ? &m->mc : nullptr;
}
CtxView ctx_view(lbm_ctx* c) {
  CtxView v;
  v.model = c->model;
  v.storage = c->storage;
  v.D = c->D;
  v.Q = c->Q;
  v.ops = c->ops;
  v.g = c->g;
  v.omega = c->omega;
  v.stream = c->stream;
  v.state[0] = &c->state[0];
  v.state[1] = &c->state[1];
  v.cur = &c->cur;
  v.fields = &c->fields;
  v.inited = c->inited;
  v.steps = &c->steps;
  v.launches = &c->launches;
  v.rec = &c->rec;
  v.variant = pick_variant(c);
  v.fixed_ends = c->fix_width > 0;
  v.slab = c->slab_axis >= 0;
  v.status = static_cast<int*>(c->status.p);
  return v;
}
}  // namespace lbm

// ================================================================ C ABI
extern "C" {

const char* lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of device memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSTABLE: return "non-finite populations";
    case LBM_ESTATE: return "call out of order";
    case LBM_EDEVICE: return "device-side timeout";
    case LBM_EIO: return "file I/O failed";
    default: return "unknown error";
  }
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

int lbm_model_info(int model, int* Q, int* D, int* reach, int32_t* e, double* w, double* c,
                   double* T0) {
  if (model != LBM_D2Q33 && model != LBM_D3Q95) return fail(LBM_EINVAL, "unknown model %d", model);
  const HostModel* hm = host_model(model);
  if (!hm) return fail(LBM_EINVAL, "model table solve failed");
  const VelSet& vs = hm->vs;
  if (Q) *Q = vs.Q;
  if (D) *D = vs.D;
  if (reach) *reach = vs.R;
  if (e)
    for (int i = 0; i < vs.Q; ++i)
      for (int d = 0; d < vs.D; ++d) e[i * vs.D + d] = vs.e[i][d];
  if (w)
    for (int i = 0; i < vs.Q; ++i) w[i] = hm->w[i];
  if (c) *c = hm->c;
  if (T0) *T0 = hm->mc.T0;
  return LBM_OK;
}

int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(LBM_EINVAL, "allocator and free function must both be set or both be NULL");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_user = user;
  return LBM_OK;
}

int lbm_create(lbm_ctx** out, int model, const int64_t dims[3], double omega, int storage,
               void* stream) {
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (model != LBM_D2Q33 && model != LBM_D3Q95) return fail(LBM_EINVAL, "unknown model %d", model);
  const StorageOps* ops = ops_for(storage);
  if (!ops) return fail(LBM_EINVAL, "unknown storage %d", storage);
  if (!dims) return fail(LBM_EINVAL, "dims is NULL");
  for (int k = 0; k < 3; ++k)
    if (dims[k] < 1 || dims[k] > (int64_t)1 << 30) return fail(LBM_EINVAL, "dims[%d] = %lld", k, (long long)dims[k]);
  if (model == LBM_D2Q33 && dims[2] != 1) return fail(LBM_EINVAL, "D2Q33 needs Nz == 1");
  const int64_t ncell = dims[0] * dims[1] * dims[2];
  if (ncell >= ((int64_t)1 << 31)) return fail(LBM_EINVAL, "too many cells (%lld)", (long long)ncell);
  if (dims[1] > 65535 || dims[2] > 65535) return fail(LBM_EINVAL, "Ny and Nz must be <= 65535");
  if (!(omega >= 0.0 && omega < 2.0)) return fail(LBM_EINVAL, "omega = %g outside [0, 2)", omega);
  const HostModel* hm = host_model(model);
  if (!hm) return fail(LBM_EINVAL, "model table solve failed");

  int dev = 0;
  LBM_CUDA(cudaGetDevice(&dev));
  int rc = ensure_uploaded(dev);
  if (rc) return rc;

  lbm_ctx* c = new lbm_ctx();
  c->model = model;
  c->storage = storage;
  c->dev = dev;
  c->D = hm->vs.D;
  c->Q = hm->vs.Q;
  c->ops = ops;
  c->g.nx = (int)dims[0];
  c->g.ny = (int)dims[1];
  c->g.nz = (int)dims[2];
  c->g.nxy = (int)(dims[0] * dims[1]);
  c->g.ncell = ncell;
  c->omega = omega;
  c->stream = (cudaStream_t)stream;
  const size_t sb = state_bytes(c);
  if ((rc = c->state[0].ensure(sb, c->stream)) || (rc = c->state[1].ensure(sb, c->stream)) ||
      (rc = c->partials.ensure((size_t)moment_blocks(ncell) * kAuditSlots * sizeof(double),
                               c->stream)) ||
      (rc = c->audit_out.ensure(kAuditSlots * sizeof(double), c->stream)) ||
      (rc = c->status.ensure(sizeof(int), c->stream))) {
    delete c;
    return rc;
  }
  {
    cudaError_t e = cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "status reset");
    }
  }
  *out = c;
  return LBM_OK;
}

int lbm_destroy(lbm_ctx* c) {
  if (!c) return LBM_OK;
  DeviceGuard dg(c->dev);
  cudaStreamSynchronize(c->stream);
  if (c->xfer_stream) cudaStreamSynchronize(c->xfer_stream);
  delete c;
  return LBM_OK;
}

int lbm_set_omega(lbm_ctx* c, double omega) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (!(omega >= 0.0 && omega < 2.0)) return fail(LBM_EINVAL, "omega = %g outside [0, 2)", omega);
  c->omega = omega;
  c->rec.valid = false;
  c->graph.reset();
  return LBM_OK;
}

int lbm_set_graph_steps(lbm_ctx* c, int steps) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (steps < 0 || steps % 2 || steps > 4096)
    return fail(LBM_EINVAL, "graph steps must be 0 or an even number <= 4096 (got %d)", steps);
  DeviceGuard dg(c->dev);
  c->graph.reset();
  c->graph_steps = steps;
  // capture both starting buffers now, so that no later lbm_step pays for it
  const int variant = pick_variant(c);
  if (steps > 0)
    for (int parity = 0; parity < 2; ++parity)
      if (!capture_steps(c, parity, variant))
        return fail(LBM_ECUDA, "graph capture of the step failed; direct launches stay in use");
  return LBM_OK;
}

int lbm_set_variant(lbm_ctx* c, int variant) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (variant != 0 && variant != kVariantDirect && variant != kVariantTma &&
      variant != kVariantSplit && variant != kVariantPair)
    return fail(LBM_EINVAL, "variant %d", variant);
  if (variant == kVariantPair && c->ops->elem_bytes != 2)
    return fail(LBM_EINVAL, "the pair kernel is for the FP16 / BF16 forms");
  if (variant == kVariantPair && !pair_applicable(c->g))
    return fail(LBM_EINVAL, "the pair kernel needs Nx even");
  if (variant == kVariantSplit && c->storage == LBM_FP64)
    return fail(LBM_EINVAL, "the split kernel is for the FP32-arithmetic forms");
  if (variant == kVariantTma && !tma_applicable(c->g))
    return fail(LBM_EINVAL, "the TMA kernel needs Nx %% 8 == 0");
  if (variant == kVariantTma) {
    DeviceGuard dg(c->dev);
    cudaError_t e = c->ops->prepare_tma(c->model);
    if (e != cudaSuccess) return cuda_fail(e, "TMA kernel set-up");
  }
  c->variant = variant;
  c->graph.reset();
  return LBM_OK;
}

int lbm_set_fixed_ends(lbm_ctx* c, int axis, int width, const double* lo, const double* hi) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (width == 0) {
    c->fix_width = 0;
    c->graph.reset();
    return LBM_OK;
  }
  if (axis < 0 || axis >= c->D) return fail(LBM_EINVAL, "axis %d", axis);
  const int R = c->model == LBM_D2Q33 ? Model<0>::R : Model<1>::R;
  const int n_ax = axis == 0 ? c->g.nx : (axis == 1 ? c->g.ny : c->g.nz);
  if (width < R || 2 * width > n_ax)
    return fail(LBM_EINVAL, "width %d: need reach (%d) <= width <= N/2 (%d)", width, R, n_ax / 2);
  if (!lo || !hi) return fail(LBM_EINVAL, "end states are required");
  const int D = c->D;
  double host[2 * 5];   // rho[2] | U[D][2] | T[2]
  for (int s = 0; s < 2; ++s) {
    const double* st = s == 0 ? lo : hi;
    for (int k = 0; k < D + 2; ++k)
      if (!std::isfinite(st[k])) return fail(LBM_EINVAL, "end state has non-finite values");
    if (!(st[0] > 0.0 && st[D + 1] > 0.0)) return fail(LBM_EINVAL, "end state needs rho > 0, T > 0");
    host[s] = st[0];
    for (int d = 0; d < D; ++d) host[2 + 2 * d + s] = st[1 + d];
    host[2 + 2 * D + s] = st[D + 1];
  }
  DeviceGuard dg(c->dev);
  DevBuf fields;
  int rc;
  if ((rc = fields.ensure(sizeof host, c->stream)) ||
      (rc = c->fix_tmpl.ensure((size_t)c->Q * 2 * c->ops->elem_bytes, c->stream)))
    return rc;
  LBM_CUDA(cudaMemcpyAsync(fields.p, host, (size_t)(D + 2) * 2 * sizeof(double),
                           cudaMemcpyHostToDevice, c->stream));
  Grid t{2, 1, 1, 2, 2};
  const double* f = static_cast<const double*>(fields.p);
  cudaError_t e = c->ops->init(c->model, f, f + 2, f + 2 + 2 * D, c->fix_tmpl.p, t, 0, t.ncell,
                               c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "end-state equilibrium launch");
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  c->launches += 1;
  c->fix_axis = axis;
  c->fix_width = width;
  c->rec.valid = false;
  c->graph.reset();
  return LBM_OK;
}

int lbm_set_stream(lbm_ctx* c, void* stream) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  c->stream = (cudaStream_t)stream;
  return LBM_OK;
}

// The copy stream and its events (created on first use).
static int ensure_xfer(lbm_ctx* c) {
  if (!c->xfer_stream &&
      cudaStreamCreateWithFlags(&c->xfer_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(LBM_ECUDA, "cannot create the copy stream");
  for (cudaEvent_t& ev : c->xfer_ev)
    if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return fail(LBM_ECUDA, "cannot create the copy events");
  return LBM_OK;
}

// lbm_init's chunked upload of host fields (see lbm_init): copies on the copy stream,
// each chunk's field check and equilibrium (into state[spare]) on the context's
// stream after its copies.
static int upload_and_init(lbm_ctx* c, const double* rho, const double* U, const double* T,
                           int spare, unsigned long long* bad_d) {
  const size_t n = (size_t)c->g.ncell;
  double* f = static_cast<double*>(c->fields.p);
  double* fU = f + n;
  double* fT = f + (size_t)(c->D + 1) * n;
  const int nch = (long long)n >= kXferMinCells ? kXferChunks : 1;
  for (int k = 0; k < nch; ++k) {
    const size_t a = n * (size_t)k / (size_t)nch, b = n * (size_t)(k + 1) / (size_t)nch;
    const size_t bytes = (b - a) * sizeof(double);
    LBM_CUDA(cudaMemcpyAsync(f + a, rho + a, bytes, cudaMemcpyHostToDevice, c->xfer_stream));
    for (int d = 0; d < c->D; ++d)
      LBM_CUDA(cudaMemcpyAsync(fU + (size_t)d * n + a, U + (size_t)d * n + a, bytes,
                               cudaMemcpyHostToDevice, c->xfer_stream));
    LBM_CUDA(cudaMemcpyAsync(fT + a, T + a, bytes, cudaMemcpyHostToDevice, c->xfer_stream));
    LBM_CUDA(cudaEventRecord(c->xfer_ev[k], c->xfer_stream));
    LBM_CUDA(cudaStreamWaitEvent(c->stream, c->xfer_ev[k], 0));
    cudaError_t e = launch_check_fields(f, fU, fT, (long long)n, (long long)a, (long long)b, c->D,
                                        bad_d, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "field check launch");
    e = c->ops->init(c->model, f, fU, fT, c->state[spare].p, c->g, (long long)a, (long long)b,
                     c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init launch");
    c->launches += 2;
  }
  return LBM_OK;
}

int lbm_init(lbm_ctx* c, const double* rho, const double* U, const double* T, int where) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (!rho || !U || !T) return fail(LBM_EINVAL, "rho, U and T are required");
  if (where != LBM_HOST && where != LBM_DEVICE) return fail(LBM_EINVAL, "bad where");
  const size_t n = (size_t)c->g.ncell;
  DeviceGuard dg(c->dev);
  int rc = c->fields.ensure((size_t)(c->D + 2) * n * sizeof(double), c->stream);
  if (rc) return rc;
  double* f = static_cast<double*>(c->fields.p);
  double* fU = f + n;
  double* fT = f + (size_t)(c->D + 1) * n;
  if (where == LBM_DEVICE) {
    LBM_CUDA(cudaMemcpyAsync(f, rho, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    LBM_CUDA(cudaMemcpyAsync(fU, U, (size_t)c->D * n * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream));
    LBM_CUDA(cudaMemcpyAsync(fT, T, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    c->cur = 0;
    cudaError_t e = c->ops->init(c->model, f, fU, fT, c->state[0].p, c->g, 0, (long long)n,
                                 c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init launch");
    c->launches += 1;
  } else {
    // Host fields: uploaded in chunks on the copy stream; chunk k's check and
    // equilibrium run on the context's stream once its copies have landed, while the
    // next chunk uploads.  The equilibrium goes to the buffer that does not hold the
    // live state, which becomes live only once every value has passed the check
    // (the fields are validated on the device: a pass over them on the host costs
    // more than the upload).
    if ((rc = c->check.ensure(sizeof(unsigned long long), c->stream))) return rc;
    if ((rc = ensure_xfer(c))) return rc;
    const int spare = c->inited ? (c->cur ^ 1) : 0;
    unsigned long long* bad_d = static_cast<unsigned long long*>(c->check.p);
    LBM_CUDA(cudaMemsetAsync(bad_d, 0xff, sizeof(unsigned long long), c->stream));
    // the copies overwrite the fields buffer only after the work queued before this call
    LBM_CUDA(cudaEventRecord(c->xfer_ev[kXferChunks], c->stream));
    LBM_CUDA(cudaStreamWaitEvent(c->xfer_stream, c->xfer_ev[kXferChunks], 0));
    if ((rc = upload_and_init(c, rho, U, T, spare, bad_d))) {
      // nothing may still read the caller's arrays once the call has returned
      c->rec.valid = false;
      cudaStreamSynchronize(c->xfer_stream);
      cudaStreamSynchronize(c->stream);
      return rc;
    }
    unsigned long long bad = 0;
    LBM_CUDA(cudaMemcpyAsync(&bad, bad_d, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    if (bad != ~0ull) {
      c->rec.valid = false;   // the kept initial fields were overwritten
      const size_t k = (size_t)(bad >> 2);
      switch ((int)(bad & 3)) {
        case 0: return fail(LBM_EINVAL, "rho[%zu] = %g (rho must be finite and > 0)", k, rho[k]);
        case 2: return fail(LBM_EINVAL, "T[%zu] = %g (T must be finite and > 0)", k, T[k]);
        default: return fail(LBM_EINVAL, "U has a non-finite value at cell %zu", k);
      }
    }
    c->cur = spare;
  }
  c->inited = true;
  c->steps = 0;
  c->rec.valid = false;
  return LBM_OK;
}

// The conservation audit of the current state into c->audit_host (blocking).
int run_audit(lbm_ctx* c) {
  cudaError_t e = c->ops->moments(c->model, c->state[c->cur].p, c->g, nullptr, nullptr, nullptr,
                                  static_cast<double*>(c->partials.p), 0,
                                  moment_blocks(c->g.ncell), c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "audit launch");
  e = launch_audit_reduce(static_cast<double*>(c->partials.p), moment_blocks(c->g.ncell),
                          static_cast<double*>(c->audit_out.p), c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "audit reduce launch");
  c->launches += 2;
  LBM_CUDA(cudaMemcpyAsync(c->audit_host, c->audit_out.p, kAuditSlots * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_step(lbm_ctx* c, int64_t n) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (!c->inited) return fail(LBM_ESTATE, "lbm_step before lbm_init");
  if (n < 0) return fail(LBM_EINVAL, "n = %lld", (long long)n);
  DeviceGuard dg(c->dev);
  if (c->audit_every <= 0) return do_steps(c, n);
  for (int64_t left = n; left > 0;) {
    const int64_t m = std::min(left, c->audit_every - c->steps % c->audit_every);
    int rc = do_steps(c, m);
    if (rc) return rc;
    left -= m;
    if (c->steps % c->audit_every == 0) {
      if ((rc = run_audit(c))) return rc;
      if (c->audit_host[6] > 0)   // slot 6: number of non-finite populations
        return fail(LBM_EUNSTABLE, "%g non-finite populations after step %lld; stepping stopped",
                    c->audit_host[6], (long long)c->steps);
    }
  }
  return LBM_OK;
}

int lbm_set_audit_every(lbm_ctx* c, int64_t k) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (k < 0) return fail(LBM_EINVAL, "k = %lld", (long long)k);
  c->audit_every = k;
  return LBM_OK;
}

// ---------------------------------------------------------------- checkpoint files
namespace {
struct StateFileHeader {
  char magic[8];
  int32_t version, model, storage, Q, elem_bytes, reserved;
  int64_t dims[3];
  double omega;
  int64_t steps;
};
constexpr char kStateMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', 'E'};
constexpr size_t kFileChunk = (size_t)64 << 20;
}  // namespace

int lbm_save(lbm_ctx* c, const char* path) {
  if (!c || !path) return fail(LBM_EINVAL, "ctx or path is NULL");
  if (!c->inited) return fail(LBM_ESTATE, "lbm_save before lbm_init");
  DeviceGuard dg(c->dev);
  StateFileHeader h{};
  std::memcpy(h.magic, kStateMagic, sizeof h.magic);
  h.version = 1;
  h.model = c->model;
  h.storage = c->storage;
  h.Q = c->Q;
  h.elem_bytes = c->ops->elem_bytes;
  h.dims[0] = c->g.nx;
  h.dims[1] = c->g.ny;
  h.dims[2] = c->g.nz;
  h.omega = c->omega;
  h.steps = c->steps;
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(LBM_EIO, "cannot open %s for writing", path);
  int rc = LBM_OK;
  if (std::fwrite(&h, sizeof h, 1, f) != 1) rc = fail(LBM_EIO, "write failed: %s", path);
  std::vector<char> buf;
  const size_t total = state_bytes(c);
  const char* src = static_cast<const char*>(c->state[c->cur].p);
  for (size_t off = 0; rc == LBM_OK && off < total; off += kFileChunk) {
    const size_t m = std::min(kFileChunk, total - off);
    buf.resize(m);
    cudaError_t e = cudaMemcpyAsync(buf.data(), src + off, m, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "state read-back");
    else if (std::fwrite(buf.data(), 1, m, f) != m) rc = fail(LBM_EIO, "write failed: %s", path);
  }
  if (std::fclose(f) != 0 && rc == LBM_OK) rc = fail(LBM_EIO, "close failed: %s", path);
  return rc;
}

int lbm_load(lbm_ctx* c, const char* path) {
  if (!c || !path) return fail(LBM_EINVAL, "ctx or path is NULL");
  DeviceGuard dg(c->dev);
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(LBM_EIO, "cannot open %s", path);
  StateFileHeader h{};
  int rc = LBM_OK;
  if (std::fread(&h, sizeof h, 1, f) != 1) rc = fail(LBM_EIO, "%s: short header", path);
  else if (std::memcmp(h.magic, kStateMagic, sizeof h.magic) != 0 || h.version != 1)
    rc = fail(LBM_EINVAL, "%s is not a state file of this library", path);
  else if (h.model != c->model || h.storage != c->storage || h.Q != c->Q ||
           h.elem_bytes != c->ops->elem_bytes || h.dims[0] != c->g.nx || h.dims[1] != c->g.ny ||
           h.dims[2] != c->g.nz)
    rc = fail(LBM_EINVAL, "%s holds model %d storage %d grid %lldx%lldx%lld; the context differs",
              path, h.model, h.storage, (long long)h.dims[0], (long long)h.dims[1],
              (long long)h.dims[2]);
  else if (!(h.omega >= 0.0 && h.omega < 2.0) || h.steps < 0)
    rc = fail(LBM_EINVAL, "%s: bad omega or step count", path);
  const size_t total = state_bytes(c);
  if (rc == LBM_OK) {
    // a file of the wrong length is refused before anything is uploaded
    const long here = std::ftell(f);
    long end = -1;
    if (here >= 0 && std::fseek(f, 0, SEEK_END) == 0) end = std::ftell(f);
    if (end < 0 || std::fseek(f, here, SEEK_SET) != 0)
      rc = fail(LBM_EIO, "%s: cannot determine the file size", path);
    else if ((size_t)(end - here) != total)
      rc = fail(LBM_EIO, "%s: %ld bytes of state, the context needs %zu (truncated or foreign file)",
                path, end - here, total);
  }
  // The state goes into the spare ping-pong buffer; the context switches to it only
  // once every piece has arrived, so a failed load leaves the live state untouched.
  std::vector<char> buf;
  const int spare = c->cur ^ 1;
  char* dst = static_cast<char*>(c->state[spare].p);
  for (size_t off = 0; rc == LBM_OK && off < total; off += kFileChunk) {
    const size_t m = std::min(kFileChunk, total - off);
    buf.resize(m);
    if (std::fread(buf.data(), 1, m, f) != m) {
      rc = fail(LBM_EIO, "%s: truncated state", path);
      break;
    }
    cudaError_t e = cudaMemcpyAsync(dst + off, buf.data(), m, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "state upload");
  }
  std::fclose(f);
  if (rc != LBM_OK) return rc;
  c->cur = spare;
  c->steps = h.steps;
  c->omega = h.omega;
  c->inited = true;
  c->rec.valid = false;
  c->graph.reset();
  return LBM_OK;
}

int64_t lbm_steps_done(const lbm_ctx* c) { return c ? c->steps : -1; }
int64_t lbm_launch_count(const lbm_ctx* c) { return c ? c->launches : -1; }

// lbm_moments' chunked read-back to host arrays (see lbm_moments); dr, du, dt are the
// device staging arrays.
static int moments_to_host(lbm_ctx* c, double* rho, double* U, double* T, double* dr, double* du,
                           double* dt) {
  const size_t n = (size_t)c->g.ncell;
  const long long nb = moment_blocks(c->g.ncell);
  const int nch = (long long)n >= kXferMinCells ? kXferChunks : 1;
  for (int k = 0; k < nch; ++k) {
    const long long b0 = nb * k / nch, b1 = nb * (k + 1) / nch;
    cudaError_t e = c->ops->moments(c->model, c->state[c->cur].p, c->g, dr, du, dt,
                                    static_cast<double*>(c->partials.p), b0, b1 - b0, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "moments launch");
    c->launches += 1;
    LBM_CUDA(cudaEventRecord(c->xfer_ev[k], c->stream));
    LBM_CUDA(cudaStreamWaitEvent(c->xfer_stream, c->xfer_ev[k], 0));
    const size_t a = (size_t)b0 * kMomentThreads;
    const size_t b = std::min(n, (size_t)b1 * kMomentThreads);
    const size_t bytes = (b - a) * sizeof(double);
    if (rho)
      LBM_CUDA(cudaMemcpyAsync(rho + a, dr + a, bytes, cudaMemcpyDeviceToHost, c->xfer_stream));
    if (U)
      for (int d = 0; d < c->D; ++d)
        LBM_CUDA(cudaMemcpyAsync(U + (size_t)d * n + a, du + (size_t)d * n + a, bytes,
                                 cudaMemcpyDeviceToHost, c->xfer_stream));
    if (T) LBM_CUDA(cudaMemcpyAsync(T + a, dt + a, bytes, cudaMemcpyDeviceToHost, c->xfer_stream));
  }
  // the context's stream resumes once the read-back is complete (the staging buffer is
  // free again)
  LBM_CUDA(cudaEventRecord(c->xfer_ev[kXferChunks], c->xfer_stream));
  LBM_CUDA(cudaStreamWaitEvent(c->stream, c->xfer_ev[kXferChunks], 0));
  return LBM_OK;
}

int lbm_moments(lbm_ctx* c, double* rho, double* U, double* T, int where) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (!c->inited) return fail(LBM_ESTATE, "lbm_moments before lbm_init");
  if (where != LBM_HOST && where != LBM_DEVICE) return fail(LBM_EINVAL, "bad where");
  DeviceGuard dg(c->dev);
  const size_t n = (size_t)c->g.ncell;
  double *dr = rho, *du = U, *dt = T;
  int rc = LBM_OK;
  if (where == LBM_HOST) {
    if ((rc = c->mom.ensure((size_t)(c->D + 2) * n * sizeof(double), c->stream))) return rc;
    double* m = static_cast<double*>(c->mom.p);
    dr = rho ? m : nullptr;
    du = U ? m + n : nullptr;
    dt = T ? m + (size_t)(c->D + 1) * n : nullptr;
  }
  if (where == LBM_DEVICE) {
    cudaError_t e = c->ops->moments(c->model, c->state[c->cur].p, c->g, dr, du, dt,
                                    static_cast<double*>(c->partials.p), 0,
                                    moment_blocks(c->g.ncell), c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "moments launch");
    c->launches += 1;
    return LBM_OK;
  }
  // Host outputs: the moments in chunks on the context's stream, each chunk read back
  // on the copy stream while the next one is computed.
  if ((rc = ensure_xfer(c))) return rc;
  rc = moments_to_host(c, rho, U, T, dr, du, dt);
  // returns once the host arrays are filled (or, after an error, no longer written)
  cudaStreamSynchronize(c->xfer_stream);
  return rc;
}

int lbm_audit(lbm_ctx* c, double out[8]) {
  if (!c || !out) return fail(LBM_EINVAL, "ctx or out is NULL");
  if (!c->inited) return fail(LBM_ESTATE, "lbm_audit before lbm_init");
  DeviceGuard dg(c->dev);
  int rc = run_audit(c);
  if (rc) return rc;
  std::memcpy(out, c->audit_host, sizeof c->audit_host);
  return out[6] > 0 ? fail(LBM_EUNSTABLE, "%g non-finite populations", out[6]) : LBM_OK;
}

int lbm_get_populations(lbm_ctx* c, double* f, int where) {
  if (!c || !f) return fail(LBM_EINVAL, "ctx or f is NULL");
  if (!c->inited) return fail(LBM_ESTATE, "no state yet");
  if (where != LBM_HOST && where != LBM_DEVICE) return fail(LBM_EINVAL, "bad where");
  DeviceGuard dg(c->dev);
  const size_t n = (size_t)c->Q * (size_t)c->g.ncell;
  double* dst = f;
  if (where == LBM_HOST) {
    int rc = c->mom.ensure(n * sizeof(double), c->stream);
    if (rc) return rc;
    dst = static_cast<double*>(c->mom.p);
  }
  cudaError_t e = c->ops->get_f(c->model, c->state[c->cur].p, dst, c->g, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_f launch");
  c->launches += 1;
  if (where == LBM_HOST) {
    LBM_CUDA(cudaMemcpyAsync(f, dst, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
  }
  return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const double* f, int where) {
  if (!c || !f) return fail(LBM_EINVAL, "ctx or f is NULL");
  if (where != LBM_HOST && where != LBM_DEVICE) return fail(LBM_EINVAL, "bad where");
  DeviceGuard dg(c->dev);
  const size_t n = (size_t)c->Q * (size_t)c->g.ncell;
  const double* srcp = f;
  if (where == LBM_HOST) {
    if (!all_finite(f, n)) return fail(LBM_EINVAL, "populations have non-finite values");
    int rc = c->mom.ensure(n * sizeof(double), c->stream);
    if (rc) return rc;
    LBM_CUDA(cudaMemcpyAsync(c->mom.p, f, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    srcp = static_cast<const double*>(c->mom.p);
  }
  c->cur = 0;
  cudaError_t e = c->ops->set_f(c->model, srcp, c->state[0].p, c->g, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_f launch");
  c->launches += 1;
  if (where == LBM_HOST) LBM_CUDA(cudaStreamSynchronize(c->stream));
  c->inited = true;
  c->steps = 0;
  c->rec.valid = false;
  return LBM_OK;
}

int lbm_get_raw(lbm_ctx* c, void* h, size_t bytes, int where) {
  if (!c || !h) return fail(LBM_EINVAL, "ctx or h is NULL");
  if (!c->inited) return fail(LBM_ESTATE, "no state yet");
  if (bytes != state_bytes(c)) return fail(LBM_EINVAL, "bytes = %zu, state is %zu", bytes, state_bytes(c));
  if (where != LBM_HOST && where != LBM_DEVICE) return fail(LBM_EINVAL, "bad where");
  DeviceGuard dg(c->dev);
  LBM_CUDA(cudaMemcpyAsync(h, c->state[c->cur].p, bytes,
                           where == LBM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                           c->stream));
  if (where == LBM_HOST) LBM_CUDA(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_set_raw(lbm_ctx* c, const void* h, size_t bytes, int where) {
  if (!c || !h) return fail(LBM_EINVAL, "ctx or h is NULL");
  if (bytes != state_bytes(c)) return fail(LBM_EINVAL, "bytes = %zu, state is %zu", bytes, state_bytes(c));
  if (where != LBM_HOST && where != LBM_DEVICE) return fail(LBM_EINVAL, "bad where");
  DeviceGuard dg(c->dev);
  c->cur = 0;
  LBM_CUDA(cudaMemcpyAsync(c->state[0].p, h, bytes,
                           where == LBM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                           c->stream));
  if (where == LBM_HOST) LBM_CUDA(cudaStreamSynchronize(c->stream));
  c->inited = true;
  c->steps = 0;
  c->rec.valid = false;
  return LBM_OK;
}

int lbm_synchronize(lbm_ctx* c) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  DeviceGuard dg(c->dev);
  int flag = 0;
  LBM_CUDA(cudaMemcpyAsync(&flag, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(cudaStreamSynchronize(c->stream));
  if (flag) {
    // reported once: the flag is cleared for the launches that follow
    LBM_CUDA(cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    return fail(LBM_EDEVICE, "a TMA stream-collide launch timed out waiting for its copies");
  }
  return LBM_OK;
}

// ---------------------------------------------------------------- slabs of a decomposed grid
int lbm_halo_plan(int model, int64_t interior, int face, int send, int32_t* segs, int* count) {
  if (model != LBM_D2Q33 && model != LBM_D3Q95) return fail(LBM_EINVAL, "unknown model %d", model);
  if (face != 0 && face != 1) return fail(LBM_EINVAL, "face must be 0 or 1");
  if (!count) return fail(LBM_EINVAL, "count is NULL");
  const HostModel* hm = host_model(model);
  if (!hm) return fail(LBM_EINVAL, "model table solve failed");
  if (interior < hm->vs.R)
    return fail(LBM_EINVAL, "a slab needs at least the stencil reach (%d) of interior planes", hm->vs.R);
  std::vector<int32_t> v;
  halo_plan_host(hm->vs, interior, face, send, &v);
  const int n = (int)(v.size() / 2);
  if (segs) {
    if (*count < n) {
      *count = n;
      return fail(LBM_EINVAL, "segs holds %d segments, the plan has %d", *count, n);
    }
    std::memcpy(segs, v.data(), v.size() * sizeof(int32_t));
  }
  *count = n;
  return LBM_OK;
}

int lbm_create_slab(lbm_ctx** out, int model, const int64_t dims[3], double omega, int storage,
                    void* stream) {
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!dims) return fail(LBM_EINVAL, "dims is NULL");
  if (model != LBM_D2Q33 && model != LBM_D3Q95) return fail(LBM_EINVAL, "unknown model %d", model);
  const HostModel* hm = host_model(model);
  if (!hm) return fail(LBM_EINVAL, "model table solve failed");
  const int axis = hm->vs.D == 3 ? 2 : 1;
  const int R = hm->vs.R;
  if (dims[axis] < R)
    return fail(LBM_EINVAL, "a slab needs at least the stencil reach (%d) of interior planes", R);
  int64_t full[3] = {dims[0], dims[1], dims[2]};
  full[axis] += 2 * R;
  lbm_ctx* c = nullptr;
  int rc = lbm_create(&c, model, full, omega, storage, stream);
  if (rc) return rc;
  c->slab_axis = axis;
  c->slab_interior = dims[axis];
  c->slab_ghost = R;
  std::vector<int32_t> all, v;
  int nseg = -1;
  for (int list = 0; list < 4; ++list) {   // send low, send high, recv low, recv high
    halo_plan_host(hm->vs, dims[axis], list & 1, list < 2, &v);
    if (nseg < 0) nseg = (int)(v.size() / 2);
    if ((int)(v.size() / 2) != nseg) {
      lbm_destroy(c);
      return fail(LBM_EINVAL, "halo lists differ in length");
    }
    all.insert(all.end(), v.begin(), v.end());
  }
  c->halo_nseg = nseg;
  DeviceGuard dg(c->dev);
  if ((rc = c->halo_segs.ensure(all.size() * sizeof(int32_t), c->stream))) {
    lbm_destroy(c);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(c->halo_segs.p, all.data(), all.size() * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    lbm_destroy(c);
    return cuda_fail(e, "halo plan upload");
  }
  *out = c;
  return LBM_OK;
}

int lbm_halo_info(const lbm_ctx* c, int* ghost, int64_t* interior, int* segments, size_t* face_bytes) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (c->slab_axis < 0) return fail(LBM_ESTATE, "not a slab context (lbm_create_slab)");
  const long long plane = c->slab_axis == 2 ? (long long)c->g.nxy : (long long)c->g.nx;
  if (ghost) *ghost = c->slab_ghost;
  if (interior) *interior = c->slab_interior;
  if (segments) *segments = c->halo_nseg;
  if (face_bytes) *face_bytes = (size_t)c->halo_nseg * (size_t)plane * (size_t)c->ops->elem_bytes;
  return LBM_OK;
}

static int halo_move(lbm_ctx* c, int face, void* buf, int to_buf) {
  if (!c || !buf) return fail(LBM_EINVAL, "ctx or buf is NULL");
  if (c->slab_axis < 0) return fail(LBM_ESTATE, "not a slab context (lbm_create_slab)");
  if (face != 0 && face != 1) return fail(LBM_EINVAL, "face must be 0 or 1");
  if (!c->inited) return fail(LBM_ESTATE, "no state yet");
  DeviceGuard dg(c->dev);
  const long long plane = c->slab_axis == 2 ? (long long)c->g.nxy : (long long)c->g.nx;
  const int list = to_buf ? face : 2 + face;
  const int* segs = static_cast<const int*>(c->halo_segs.p) + (size_t)list * 2 * c->halo_nseg;
  cudaError_t e = c->ops->halo_copy(c->state[c->cur].p, buf, segs, c->halo_nseg, plane, c->g.ncell,
                                    to_buf, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, to_buf ? "halo pack launch" : "halo unpack launch");
  c->launches += 1;
  return LBM_OK;
}

int lbm_halo_pack(lbm_ctx* c, int face, void* buf) { return halo_move(c, face, buf, 1); }
int lbm_halo_unpack(lbm_ctx* c, int face, const void* buf) {
  return halo_move(c, face, const_cast<void*>(buf), 0);
}

int lbm_test_stall(lbm_ctx* c, int64_t chunk, int64_t limit_ns) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (chunk < 0 || limit_ns < 1000 || limit_ns > 2000000000LL)
    return fail(LBM_EINVAL, "chunk >= 0 and 1 us <= limit_ns <= 2 s are required");
  if (pick_variant(c) != kVariantTma) return fail(LBM_ESTATE, "the TMA variant is not selected");
  c->test.stall_chunk = chunk;
  c->test.limit_ns = (unsigned long long)limit_ns;
  c->test_pending = true;
  return LBM_OK;
}

}  // extern "C"

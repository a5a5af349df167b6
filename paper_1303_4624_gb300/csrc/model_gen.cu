// model_gen.cu - host-side generator of on-lattice isotropic velocity sets
// (lbm_equation_count and lbm_generate_model in include/lbm.h).
//
// The construction of the paper's models, for any space dimension D <= 4 and
// order m <= 7:
//   * the moment equations of Formula 5 up to n_max = 2m are indexed by the
//     exponent classes a = 2 p with p a partition of q <= m into at most D parts
//     (Formulas 7 and 8 count them: Omega(m, D), Table 1);
//   * every representative velocity expands into its orbit under coordinate
//     permutations and sign changes (the groups G_k of Formula 9), one weight
//     per orbit;
//   * Formula 10: a model has Omega(m, D) - 1 orbits, so that the weights and
//     the scale c are Omega(m, D) unknowns.
//
// Solution method (this file's own): with y = c^2, Formula 5 reads
//   sum_g S(a, g) W_g = G(a) z^{q(a)},   z = 1 / y,  q(a) = |a| / 2,
// where S(a, g) = sum over the orbit of e^a (integers) and G(a) the normalised
// Gaussian moment (Formula 4 over its n = 0 value).  For fixed z the system is
// linear in W and has one equation more than unknowns, so it is solvable exactly
// when det [S | G z^q] = 0, a polynomial of degree <= m in z whose coefficients
// are minors of S (Laplace expansion along the last column).  Its positive real
// roots are bracketed on a logarithmic grid and bisected; at each root W follows
// from the (consistent) linear system by least squares (Householder QR), and
// (W, c) is polished by Newton's method on the full nonlinear system.  A root
// gives a model when every weight is positive.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <functional>
#include <vector>

#include "../../include/lbm.h"
#include "adjoint.h"

namespace {

using lbm::ctx_fail;

constexpr int kMaxD = 4;
constexpr int kMaxM = 7;
constexpr int kMaxEntry = 8;   // |e_alpha| <= 8 keeps every S(a, g) exact in FP64

using Vec = std::array<int, kMaxD>;

// Formulas 7 and 8: Omega(m, D) = sum_{q <= m} pi(q, D), with pi(q, D) the
// coefficient of x^q in prod_{k=1}^{D} 1 / (1 - x^k).
long long omega_from_generating_function(int m, int D) {
  std::vector<long long> c(m + 1, 0);
  c[0] = 1;
  for (int k = 1; k <= D; ++k)            // multiply by 1 / (1 - x^k) = 1 + x^k + x^2k + ...
    for (int q = k; q <= m; ++q) c[q] += c[q - k];
  long long s = 0;
  for (int q = 0; q <= m; ++q) s += c[q];
  return s;
}

// Exponent classes: a = 2 p for every partition p of q = 0..m into at most D parts
// (parts in non-increasing order, zero-padded).
void enumerate_partitions(int q, int max_parts, int largest, Vec& cur, int depth,
                          std::vector<Vec>& out) {
  if (q == 0) {
    Vec a{};
    for (int k = 0; k < depth; ++k) a[k] = 2 * cur[k];
    out.push_back(a);
    return;
  }
  if (depth == max_parts) return;
  for (int part = std::min(q, largest); part >= 1; --part) {
    cur[depth] = part;
    enumerate_partitions(q - part, max_parts, part, cur, depth + 1, out);
  }
}

std::vector<Vec> exponent_classes(int m, int D) {
  std::vector<Vec> out;
  Vec cur{};
  for (int q = 0; q <= m; ++q) enumerate_partitions(q, D, q, cur, 0, out);
  return out;
}

// Normalised Gaussian moment prod_alpha (a_alpha - 1)!! / 2^{a_alpha / 2} (Formula 4
// divided by pi^{D/2}); every a_alpha is even here.
double gauss_moment(const Vec& a, int D) {
  double r = 1.0;
  for (int k = 0; k < D; ++k) {
    for (int f = a[k] - 1; f > 1; f -= 2) r *= f;
    r /= std::ldexp(1.0, a[k] / 2);
  }
  return r;
}

// Orbit of a representative under the signed permutations (the group G_k of the
// text before Formula 9), duplicates removed, in decreasing lexicographic order.
std::vector<Vec> orbit(const Vec& rep, int D) {
  std::vector<int> idx(D);
  for (int k = 0; k < D; ++k) idx[k] = k;
  std::vector<Vec> out;
  do {
    for (int s = 0; s < (1 << D); ++s) {
      Vec v{};
      for (int k = 0; k < D; ++k) v[k] = ((s >> k) & 1) ? -rep[idx[k]] : rep[idx[k]];
      out.push_back(v);
    }
  } while (std::next_permutation(idx.begin(), idx.end()));
  std::sort(out.begin(), out.end(), [&](const Vec& x, const Vec& y) {
    for (int k = 0; k < D; ++k)
      if (x[k] != y[k]) return x[k] > y[k];
    return false;
  });
  out.erase(std::unique(out.begin(), out.end()), out.end());
  return out;
}

double ipow(int b, int e) {
  double r = 1.0;
  for (int k = 0; k < e; ++k) r *= b;
  return r;
}

// Determinant by LU with partial pivoting (A is n x n, row-major, overwritten).
double det_lu(std::vector<double> A, int n) {
  double d = 1.0;
  for (int j = 0; j < n; ++j) {
    int p = j;
    for (int i = j + 1; i < n; ++i)
      if (std::fabs(A[i * n + j]) > std::fabs(A[p * n + j])) p = i;
    if (A[p * n + j] == 0.0) return 0.0;
    if (p != j) {
      for (int k = 0; k < n; ++k) std::swap(A[j * n + k], A[p * n + k]);
      d = -d;
    }
    d *= A[j * n + j];
    for (int i = j + 1; i < n; ++i) {
      const double f = A[i * n + j] / A[j * n + j];
      for (int k = j; k < n; ++k) A[i * n + k] -= f * A[j * n + k];
    }
  }
  return d;
}

// Solve the square system A x = b (n x n) by LU with partial pivoting; false if singular.
bool solve_lu(std::vector<double> A, std::vector<double> b, int n, std::vector<double>& x) {
  for (int j = 0; j < n; ++j) {
    int p = j;
    for (int i = j + 1; i < n; ++i)
      if (std::fabs(A[i * n + j]) > std::fabs(A[p * n + j])) p = i;
    if (A[p * n + j] == 0.0) return false;
    if (p != j) {
      for (int k = 0; k < n; ++k) std::swap(A[j * n + k], A[p * n + k]);
      std::swap(b[j], b[p]);
    }
    for (int i = j + 1; i < n; ++i) {
      const double f = A[i * n + j] / A[j * n + j];
      for (int k = j; k < n; ++k) A[i * n + k] -= f * A[j * n + k];
      b[i] -= f * b[j];
    }
  }
  x.assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= A[i * n + k] * x[k];
    x[i] = s / A[i * n + i];
  }
  return true;
}

// Least squares min |A x - b| for A r x n (r >= n) by Householder QR.
bool lstsq_qr(std::vector<double> A, std::vector<double> b, int r, int n, std::vector<double>& x) {
  for (int j = 0; j < n; ++j) {
    double norm = 0.0;
    for (int i = j; i < r; ++i) norm += A[i * n + j] * A[i * n + j];
    norm = std::sqrt(norm);
    if (norm == 0.0) return false;
    const double alpha = A[j * n + j] > 0 ? -norm : norm;
    std::vector<double> v(r, 0.0);
    for (int i = j; i < r; ++i) v[i] = A[i * n + j];
    v[j] -= alpha;
    double vv = 0.0;
    for (int i = j; i < r; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int k = j; k < n; ++k) {
      double s = 0.0;
      for (int i = j; i < r; ++i) s += v[i] * A[i * n + k];
      s = 2.0 * s / vv;
      for (int i = j; i < r; ++i) A[i * n + k] -= s * v[i];
    }
    double s = 0.0;
    for (int i = j; i < r; ++i) s += v[i] * b[i];
    s = 2.0 * s / vv;
    for (int i = j; i < r; ++i) b[i] -= s * v[i];
  }
  x.assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= A[i * n + k] * x[k];
    if (A[i * n + i] == 0.0) return false;
    x[i] = s / A[i * n + i];
  }
  return true;
}

struct System {
  int D = 0, neq = 0, G = 0;
  std::vector<double> S;     // [neq][G]
  std::vector<int> q;        // |a| / 2 per equation
  std::vector<double> rhs;   // normalised Gaussian moments
};

// max_a |c^{2q} sum_g S W - G(a)|
double residual(const System& sy, const std::vector<double>& W, double c) {
  double r = 0.0;
  for (int a = 0; a < sy.neq; ++a) {
    double s = 0.0;
    for (int g = 0; g < sy.G; ++g) s += sy.S[a * sy.G + g] * W[g];
    r = std::max(r, std::fabs(s * std::pow(c, 2 * sy.q[a]) - sy.rhs[a]));
  }
  return r;
}

struct Solution {
  double c, res;
  std::vector<double> W;
};

}  // namespace

extern "C" int lbm_equation_count(int m, int D, int64_t* out) {
  if (!out) return ctx_fail(LBM_EINVAL, "out is NULL");
  if (D < 1 || D > kMaxD) return ctx_fail(LBM_EINVAL, "D must be in [1, 4]");
  if (m < 0 || m > kMaxM) return ctx_fail(LBM_EINVAL, "m must be in [0, 7]");
  *out = omega_from_generating_function(m, D);
  return LBM_OK;
}

extern "C" int lbm_generate_model(int D, int m, int ngroups, const int* reps, int which, int qmax,
                                  int* Q, int* e, double* w, double* c_out, double* res_out,
                                  int* nsolutions) {
  if (D < 1 || D > kMaxD) return ctx_fail(LBM_EINVAL, "D must be in [1, 4]");
  if (m < 0 || m > kMaxM) return ctx_fail(LBM_EINVAL, "m must be in [0, 7]");
  if (!reps || !Q || !c_out) return ctx_fail(LBM_EINVAL, "reps, Q and c are required");
  const std::vector<Vec> cls = exponent_classes(m, D);
  const int neq = (int)cls.size();
  if ((long long)neq != omega_from_generating_function(m, D))
    return ctx_fail(LBM_EINVAL, "internal: partition enumeration disagrees with Formula 7");
  if (ngroups + 1 != neq) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "Formula 10: Omega(%d, %d) = %d equations need %d groups, got %d", m, D, neq,
             neq - 1, ngroups);
    return ctx_fail(LBM_EINVAL, msg);
  }
  // orbits
  std::vector<std::vector<Vec>> orbits;
  std::vector<Vec> canon;
  for (int g = 0; g < ngroups; ++g) {
    Vec r{};
    for (int k = 0; k < D; ++k) {
      const int v = reps[g * D + k];
      if (v < -kMaxEntry || v > kMaxEntry)
        return ctx_fail(LBM_EINVAL, "representative entries must be in [-8, 8]");
      r[k] = v < 0 ? -v : v;
    }
    std::sort(r.begin(), r.begin() + D, std::greater<int>());
    if (std::find(canon.begin(), canon.end(), r) != canon.end())
      return ctx_fail(LBM_EINVAL, "two representatives generate the same orbit");
    canon.push_back(r);
    orbits.push_back(orbit(r, D));
  }
  int nq = 0;
  for (const auto& o : orbits) nq += (int)o.size();
  *Q = nq;
  if (qmax < nq) return ctx_fail(LBM_EINVAL, "qmax is smaller than the model's Q (returned in *Q)");
  // the linear structure S W = G z^q
  System sy;
  sy.D = D;
  sy.neq = neq;
  sy.G = ngroups;
  sy.S.assign((size_t)neq * ngroups, 0.0);
  for (int a = 0; a < neq; ++a) {
    int n = 0;
    for (int k = 0; k < D; ++k) n += cls[a][k];
    sy.q.push_back(n / 2);
    sy.rhs.push_back(gauss_moment(cls[a], D));
    for (int g = 0; g < ngroups; ++g) {
      double s = 0.0;
      for (const Vec& v : orbits[g]) {
        double t = 1.0;
        for (int k = 0; k < D; ++k) t *= ipow(v[k], cls[a][k]);
        s += t;
      }
      sy.S[(size_t)a * ngroups + g] = s;
    }
  }
  // det [S | G z^q] as a polynomial in z: coefficient of z^q collects the rows with q(a) = q
  std::vector<double> poly(m + 1, 0.0);
  for (int a = 0; a < neq; ++a) {
    std::vector<double> minor;
    minor.reserve((size_t)ngroups * ngroups);
    for (int i = 0; i < neq; ++i)
      if (i != a)
        for (int g = 0; g < ngroups; ++g) minor.push_back(sy.S[(size_t)i * ngroups + g]);
    const double dm = ngroups ? det_lu(minor, ngroups) : 1.0;
    const double sign = ((a + ngroups) % 2) ? -1.0 : 1.0;
    poly[sy.q[a]] += sign * sy.rhs[a] * dm;
  }
  auto P = [&](double z) {
    double s = 0.0;
    for (int k = m; k >= 0; --k) s = s * z + poly[k];
    return s;
  };
  // positive roots: sign changes on a log grid over z in [1e-8, 1e8], then bisection
  std::vector<double> roots;
  constexpr int kGrid = 4000;
  double z0 = 1e-8, p0 = P(z0);
  for (int k = 1; k <= kGrid; ++k) {
    const double z1 = std::pow(10.0, -8.0 + 16.0 * k / kGrid), p1 = P(z1);
    if (p0 == 0.0) roots.push_back(z0);
    else if ((p0 < 0) != (p1 < 0) && p1 != 0.0) {
      double lo = z0, hi = z1, plo = p0;
      for (int it = 0; it < 200 && hi - lo > 1e-17 * hi; ++it) {
        const double mid = 0.5 * (lo + hi), pm = P(mid);
        if ((pm < 0) == (plo < 0)) { lo = mid; plo = pm; } else hi = mid;
      }
      roots.push_back(0.5 * (lo + hi));
    }
    z0 = z1;
    p0 = p1;
  }
  // weights at each root, then Newton on (W, c) for the full system
  std::vector<Solution> sols;
  for (double z : roots) {
    std::vector<double> b(neq), W;
    for (int a = 0; a < neq; ++a) b[a] = sy.rhs[a] * std::pow(z, sy.q[a]);
    if (!lstsq_qr(sy.S, b, neq, ngroups, W)) continue;
    double c = std::sqrt(1.0 / z);
    double best = residual(sy, W, c);
    for (int it = 0; it < 20; ++it) {
      const int n = ngroups + 1;
      std::vector<double> J((size_t)n * n), F(n), dx;
      for (int a = 0; a < neq; ++a) {
        double s = 0.0;
        for (int g = 0; g < ngroups; ++g) s += sy.S[(size_t)a * ngroups + g] * W[g];
        const double cn = std::pow(c, 2 * sy.q[a]);
        F[a] = -(s * cn - sy.rhs[a]);
        for (int g = 0; g < ngroups; ++g) J[(size_t)a * n + g] = sy.S[(size_t)a * ngroups + g] * cn;
        J[(size_t)a * n + ngroups] = sy.q[a] ? s * 2.0 * sy.q[a] * std::pow(c, 2 * sy.q[a] - 1) : 0.0;
      }
      if (!solve_lu(J, F, n, dx)) break;
      std::vector<double> W2 = W;
      for (int g = 0; g < ngroups; ++g) W2[g] += dx[g];
      const double c2 = c + dx[ngroups];
      const double r2 = residual(sy, W2, c2);
      if (!(r2 < best)) break;
      W = W2;
      c = c2;
      best = r2;
    }
    bool positive = c > 0;
    for (double x : W) positive = positive && x > 0;
    if (positive && best < 1e-9) sols.push_back({c, best, W});
  }
  std::sort(sols.begin(), sols.end(), [](const Solution& x, const Solution& y) { return x.c < y.c; });
  if (nsolutions) *nsolutions = (int)sols.size();
  if (sols.empty()) {
    char msg[160];
    snprintf(msg, sizeof msg,
             "no solution with positive weights (%d positive roots of the determinant)",
             (int)roots.size());
    return ctx_fail(LBM_EINVAL, msg);
  }
  if (which < 0 || which >= (int)sols.size())
    return ctx_fail(LBM_EINVAL, "which is out of range (see *nsolutions)");
  const Solution& s = sols[which];
  *c_out = s.c;
  if (res_out) *res_out = s.res;
  int i = 0;
  for (int g = 0; g < ngroups; ++g)
    for (const Vec& v : orbits[g]) {
      if (e)
        for (int k = 0; k < D; ++k) e[(size_t)i * D + k] = v[k];
      if (w) w[i] = s.W[g];
      ++i;
    }
  return LBM_OK;
}

// velset.cuh - compile-time D2Q33 / D3Q95 velocity sets.
//
// Tables 2 and 3 of the paper give one representative integer velocity per
// symmetry group; the group is the orbit of the representative under all
// coordinate permutations and sign changes (text before Formula 9: G_1, G_4,
// G_8 in 2D and G_1, G_6, G_8, G_12, G_24, G_48 in 3D).  Here each orbit is
// expanded at compile time into the storage order used everywhere in the
// library: direction 0 is the rest velocity, then opposite pairs
// (2p+1, 2p+2) with e_{2p+2} = -e_{2p+1}, pairs in table order, and within a
// group in the order the permutations and signs are enumerated below.
#pragma once

#define LBM_HD __host__ __device__

namespace lbm {

constexpr int kMaxQ = 95;  // == kMaxQc in common.h
constexpr int kMaxG = 10;  // == kMaxGc in common.h

struct VelSet {
  int D, Q, NP, G, R;
  int e[kMaxQ][3];
  int grp[kMaxQ];
  int e2[kMaxG];          // |e|^2 of each group (integer)
};

// Table 2 (D2Q33): representatives c(i, j), groups in table order.
constexpr int kRepsD2Q33[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0},
                                  {2, 2, 0}, {3, 0, 0}, {2, 1, 0}, {4, 4, 0}};
// Table 3 (D3Q95).
constexpr int kRepsD3Q95[10][3] = {{0, 0, 0}, {2, 0, 0}, {2, 2, 0}, {2, 2, 2}, {3, 0, 0},
                                   {3, 3, 0}, {3, 3, 3}, {2, 2, 5}, {4, 4, 0}, {5, 0, 0}};

LBM_HD constexpr int iabs(int v) { return v < 0 ? -v : v; }

template <int G>
LBM_HD constexpr VelSet expand(const int (&reps)[G][3], int D) {
  VelSet v{};
  v.D = D;
  v.G = G;
  constexpr int perm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  constexpr int perm2[2][3] = {{0, 1, 2}, {1, 0, 2}};
  int q = 1;  // slot 0: the rest velocity (group 0 must be (0,0,0))
  for (int k = 0; k < 3; ++k) v.e[0][k] = 0;
  v.grp[0] = 0;
  v.e2[0] = 0;
  for (int g = 1; g < G; ++g) {
    v.e2[g] = reps[g][0] * reps[g][0] + reps[g][1] * reps[g][1] + reps[g][2] * reps[g][2];
    const int np = (D == 3) ? 6 : 2;
    for (int p = 0; p < np; ++p) {
      for (int s = 0; s < (1 << D); ++s) {
        int c[3] = {0, 0, 0};
        for (int k = 0; k < D; ++k) {
          const int src = (D == 3) ? perm3[p][k] : perm2[p][k];
          const int sgn = ((s >> k) & 1) ? -1 : 1;
          c[k] = sgn * reps[g][src];
        }
        // keep the member of each +/- pair whose first nonzero component is positive
        int first = 0;
        for (int k = D - 1; k >= 0; --k)
          if (c[k] != 0) first = c[k];
        if (first <= 0) continue;
        bool dup = false;
        for (int j = 1; j < q; ++j)
          if (v.e[j][0] == c[0] && v.e[j][1] == c[1] && v.e[j][2] == c[2]) dup = true;
        if (dup) continue;
        for (int k = 0; k < 3; ++k) {
          v.e[q][k] = c[k];
          v.e[q + 1][k] = -c[k];
        }
        v.grp[q] = g;
        v.grp[q + 1] = g;
        q += 2;
      }
    }
  }
  v.Q = q;
  v.NP = (q - 1) / 2;
  int r = 0;
  for (int j = 0; j < q; ++j)
    for (int k = 0; k < 3; ++k)
      if (iabs(v.e[j][k]) > r) r = iabs(v.e[j][k]);
  v.R = r;
  return v;
}

template <int MODEL>
LBM_HD constexpr VelSet make_velset() {
  if constexpr (MODEL == 0)
    return expand<8>(kRepsD2Q33, 2);
  else
    return expand<10>(kRepsD3Q95, 3);
}

template <int MODEL>
struct Model {
  static constexpr VelSet vs = make_velset<MODEL>();
  static constexpr int D = vs.D;
  static constexpr int Q = vs.Q;
  static constexpr int NP = vs.NP;
  static constexpr int G = vs.G;
  static constexpr int R = vs.R;
};

static_assert(Model<0>::Q == 33 && Model<0>::R == 4 && Model<0>::NP == 16, "D2Q33 expansion");
static_assert(Model<1>::Q == 95 && Model<1>::R == 5 && Model<1>::NP == 47, "D3Q95 expansion");

}  // namespace lbm

// Kernel instances of the standalone batch for constraint sets other than the box of Sec. 3
// (per-coordinate boxes and Euclidean balls), on the runtime-dimension shapes: one shape per
// dimension range, the one that holds the most points.  d = 49 takes its compiled shapes.
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {

// d = 49 (7x7 patches): the compiled-dimension shapes, in k_sets49.cu
int launch_set_d49(const EmLaunch& L, const CoordBoxes& pj);
int launch_set_d49(const EmLaunch& L, const Ball& pj);

namespace {

template <class PJ>
int launch_set(const EmLaunch& L, const PJ& pj) {
  const int n = L.n, d = L.d, gm = 64;
  if (d == 49) return launch_set_d49(L, pj);
  if (d <= 28) return n <= G28_4::CAP ? launch_em<G28_4>(L, gm, pj) : -1;
  if (d <= 60) return n <= G60_4::CAP ? launch_em<G60_4>(L, gm, pj) : -1;
  if (d <= 120) return n <= G120_4::CAP ? launch_em<G120_4>(L, gm, pj) : -1;
  if (d <= 148) return n <= G148_4::CAP ? launch_em<G148_4>(L, gm, pj) : -1;
  return -1;
}

}  // namespace

int em_set_capacity(int d) {
  if (d == 49) return E49_7W::CAP;
  if (d <= 28) return G28_4::CAP;
  if (d <= 60) return G60_4::CAP;
  if (d <= 120) return G120_4::CAP;
  if (d <= 148) return G148_4::CAP;
  return 0;
}

int launch_em_set(const EmLaunch& L, int kind, const float* a, const float* b, float r) {
  if (kind == 1) return launch_set(L, CoordBoxes{a, b});
  if (kind == 2) return launch_set(L, Ball{a, r});
  return -1;
}

}  // namespace nlemk

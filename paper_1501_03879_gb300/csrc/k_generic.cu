// Kernel instances for any other d <= 148 (runtime dimension, zero-filled layout).
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {
int launch_em_generic(const EmLaunch& L) {
  const int n = L.n, d = L.d, gm = 64;
  if (d <= 28) {
    if (n <= G28_1::CAP) return launch_em<G28_1>(L, gm);
    if (n <= G28_4::CAP) return launch_em<G28_4>(L, gm);
    return -1;
  }
  if (d <= 60) {
    if (n <= G60_1::CAP) return launch_em<G60_1>(L, gm);
    if (n <= G60_4::CAP) return launch_em<G60_4>(L, gm);
    return -1;
  }
  if (d <= 120) {
    if (n <= G120_2::CAP) return launch_em<G120_2>(L, gm);
    if (n <= G120_4::CAP) return launch_em<G120_4>(L, gm);
    return -1;
  }
  if (d <= 148) {
    if (n <= G148_2::CAP) return launch_em<G148_2>(L, gm);
    if (n <= G148_4::CAP) return launch_em<G148_4>(L, gm);
    return -1;
  }
  return -1;
}
}  // namespace nlemk

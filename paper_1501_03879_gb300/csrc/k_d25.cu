// Kernel instances for d = 25 (5x5 patches).
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {
int launch_em_d25(const EmLaunch& L) {
  const int n = L.n, gm = 64;
  if (n <= E25_1::CAP) return launch_em<E25_1>(L, gm);
  if (n <= E25_2::CAP) return launch_em<E25_2>(L, gm);
  if (n <= E25_4::CAP) return launch_em<E25_4>(L, gm);
  if (n <= E25_7::CAP) return launch_em<E25_7>(L, gm);
  return -1;
}
int launch_nlem_k5(const NlemLaunch& L) {
  const int nmax = L.S * L.S, gm = 64;
  if (nmax <= E25_1::CAP) return launch_nlem<E25_1, 5>(L, gm);
  if (nmax <= E25_2::CAP) return launch_nlem<E25_2, 5>(L, gm);
  if (nmax <= E25_4::CAP) return launch_nlem<E25_4, 5>(L, gm);
  if (nmax <= E25_7::CAP) return launch_nlem<E25_7, 5>(L, gm);
  return -1;
}
}  // namespace nlemk

// Kernel instances for d = 81 (9x9 patches).
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {
int launch_em_d81(const EmLaunch& L) {
  const int n = L.n, gm = 64;
  if (n <= E81_2::CAP) return launch_em<E81_2>(L, gm);
  if (n <= E81_4::CAP) return launch_em<E81_4>(L, gm);
  if (n <= E81_7::CAP) return launch_em<E81_7>(L, gm);
  return -1;
}
int launch_nlem_k9(const NlemLaunch& L) {
  const int nmax = L.S * L.S, gm = 64;
  if (nmax <= E81_2::CAP) return launch_nlem<E81_2, 9>(L, gm);
  if (nmax <= E81_4::CAP) return launch_nlem<E81_4, 9>(L, gm);
  if (nmax <= E81_7::CAP) return launch_nlem<E81_7, 9>(L, gm);
  return -1;
}
}  // namespace nlemk

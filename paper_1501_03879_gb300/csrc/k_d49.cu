// Kernel instances for d = 49 (7x7 patches).
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {
int launch_em_d49(const EmLaunch& L) {
  const int n = L.n, gm = 64;
  if (n <= E49_2::CAP) return launch_em<E49_2>(L, gm);
  if (n <= E49_4x3::CAP) return launch_em<E49_4x3>(L, gm);
  if (n <= E49_7::CAP) return launch_em<E49_7>(L, gm);
  if (n <= E49_7W::CAP) return launch_em<E49_7W>(L, gm);
  return -1;
}
int launch_nlem_k7(const NlemLaunch& L) {
  const int nmax = L.S * L.S, gm = 64;
  if (nmax <= E49_2::CAP) return launch_nlem<E49_2, 7>(L, gm);
  if (nmax <= E49_4x3::CAP) return launch_nlem<E49_4x3, 7>(L, gm);
  if (nmax <= E49_7::CAP) return launch_nlem<E49_7, 7>(L, gm);
  if (nmax <= E49_7W::CAP) return launch_nlem<E49_7W, 7>(L, gm);
  return -1;
}
}  // namespace nlemk

// Kernel instances of NLEM-IRLS (the surrogate solver of Eq. 2 inside the one-pixel NLEM kernel).
// Patch 7 takes the same shape ladder as EM-ADMM; patches 5 and 9 take their largest shape.
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {
int launch_nlem_irls(const NlemLaunch& L) {
  const int nmax = L.S * L.S, gm = 64;
  if (L.patch == 7) {
    if (nmax <= E49_2::CAP) return launch_nlem<E49_2, 7, true>(L, gm);
    if (nmax <= E49_4x3::CAP) return launch_nlem<E49_4x3, 7, true>(L, gm);
    if (nmax <= E49_7::CAP) return launch_nlem<E49_7, 7, true>(L, gm);
    if (nmax <= E49_7W::CAP) return launch_nlem<E49_7W, 7, true>(L, gm);
    return -1;
  }
  if (L.patch == 5) return nmax <= E25_7::CAP ? launch_nlem<E25_7, 5, true>(L, gm) : -1;
  if (L.patch == 9) return nmax <= E81_7::CAP ? launch_nlem<E81_7, 9, true>(L, gm) : -1;
  return -1;
}
}  // namespace nlemk

// Kernel instances of EM-ADMM with per-point penalties mu_k = rho w_k (the WPEN variant of
// admm_iterate): standalone problems of d = 49 and NLEM with 7x7 patches, one problem per CTA.
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {
int launch_em_wpen_d49(const EmLaunch& L) {
  const int n = L.n, gm = 64;
  if (n <= E49_2::CAP) return launch_em<E49_2, ScalarBox, true>(L, gm);
  if (n <= E49_4x3::CAP) return launch_em<E49_4x3, ScalarBox, true>(L, gm);
  if (n <= E49_7::CAP) return launch_em<E49_7, ScalarBox, true>(L, gm);
  if (n <= E49_7W::CAP) return launch_em<E49_7W, ScalarBox, true>(L, gm);
  return -1;
}
int launch_nlem_wpen_k7(const NlemLaunch& L) {
  const int nmax = L.S * L.S, gm = 64;
  if (nmax <= E49_2::CAP) return launch_nlem<E49_2, 7, false, true>(L, gm);
  if (nmax <= E49_4x3::CAP) return launch_nlem<E49_4x3, 7, false, true>(L, gm);
  if (nmax <= E49_7::CAP) return launch_nlem<E49_7, 7, false, true>(L, gm);
  if (nmax <= E49_7W::CAP) return launch_nlem<E49_7W, 7, false, true>(L, gm);
  return -1;
}
}  // namespace nlemk

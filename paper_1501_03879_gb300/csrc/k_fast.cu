// Kernel instances of accelerated EM-ADMM (admm_fast_iterate, fast ADMM with restart): standalone
// problems of d = 49 and NLEM with 7x7 patches, one problem per CTA on the two-bank shape F49_7.
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {
int fast_capacity() { return F49_7::CAP; }
int launch_em_fast_d49(const EmLaunch& L) {
  if (L.n > F49_7::CAP) return -1;
  return launch_em<F49_7, ScalarBox, false, true>(L, 16);
}
int launch_nlem_fast_k7(const NlemLaunch& L) {
  if (L.S * L.S > F49_7::CAP) return -1;
  return launch_nlem<F49_7, 7, false, false, true>(L, 16);
}
}  // namespace nlemk

// Shape dispatch: picks the kernel family for (d or patch) and reports capacities.
#include "shapes.h"

namespace nlemk {

int em_capacity(int d) {
  if (d == 49) return E49_7W::CAP;
  if (d == 25) return E25_7::CAP;
  if (d == 81) return E81_7::CAP;
  if (d <= 28) return G28_4::CAP;
  if (d <= 60) return G60_4::CAP;
  if (d <= 120) return G120_4::CAP;
  if (d <= 148) return G148_4::CAP;
  return 0;
}

int nlem_capacity(int patch) {
  if (patch == 7) return E49_7W::CAP;
  if (patch == 5) return E25_7::CAP;
  if (patch == 9) return E81_7::CAP;
  return 0;
}

int launch_em_batch(const EmLaunch& L) {
  if (L.prm.solver == 2) return (L.d == 49 && L.penalty == 0) ? launch_em_fast_d49(L) : -1;
  if (L.penalty == 1) return L.d == 49 ? launch_em_wpen_d49(L) : -1;
  if (L.d == 49) return launch_em_d49(L);
  if (L.d == 25) return launch_em_d25(L);
  if (L.d == 81) return launch_em_d81(L);
  return launch_em_generic(L);
}

int launch_nlem_fp32(const NlemLaunch& L) {
  if (L.prm.solver == 1) return L.layout == 2 ? -1 : launch_nlem_irls(L);   // the pair kernel is ADMM only
  if (L.prm.solver == 2) return (L.patch == 7 && L.layout != 2 && L.penalty == 0) ? launch_nlem_fast_k7(L) : -1;
  if (L.penalty == 1) return (L.patch == 7 && L.layout != 2) ? launch_nlem_wpen_k7(L) : -1;
  if (L.layout == 2) return launch_nlem_pair_k7(L);
  // windows of more than 256 points (17x17 and up): the pixel-pair kernel; smaller windows run
  // the three-CTAs-per-SM pixel shape
  if (L.layout == 0 && nlem_pair_eligible(L) && L.S * L.S > E49_4x3::CAP) return launch_nlem_pair_k7(L);
  if (L.patch == 7) return launch_nlem_k7(L);
  if (L.patch == 5) return launch_nlem_k5(L);
  if (L.patch == 9) return launch_nlem_k9(L);
  return -1;
}

}  // namespace nlemk

// Kernel instances of the standalone batch over constraint sets beyond the box for d = 49: the
// compiled-dimension shapes of the box kernels (up to 896 points).
#include "shapes.h"
#include "solve_kernels.cuh"

namespace nlemk {
namespace {

template <class PJ>
int launch49(const EmLaunch& L, const PJ& pj) {
  const int n = L.n, gm = 64;
  if (n <= E49_4x3::CAP) return launch_em<E49_4x3>(L, gm, pj);
  if (n <= E49_7::CAP) return launch_em<E49_7>(L, gm, pj);
  if (n <= E49_7W::CAP) return launch_em<E49_7W>(L, gm, pj);
  return -1;
}

}  // namespace

int launch_set_d49(const EmLaunch& L, const CoordBoxes& pj) { return launch49(L, pj); }
int launch_set_d49(const EmLaunch& L, const Ball& pj) { return launch49(L, pj); }

}  // namespace nlemk

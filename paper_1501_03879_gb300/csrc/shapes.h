// Compiled kernel shapes.  Cfg<d, G lanes per point, Q slots per lane, P points per lane,
// NW warps>: a CTA holds up to NW*32/G*P points of dimension d.  Within each family the
// dispatcher takes the first shape whose capacity holds the problem.
#pragma once
#include "admm_core.cuh"
#include "kernels.h"

namespace nlemk {
using E49_2 = Cfg<49, 2, 25, 2, 4>;
using E49_4x3 = Cfg<49, 2, 25, 4, 4, 3>;   // three CTAs per SM (168 registers): 5-10% over two
using E49_7 = Cfg<49, 2, 25, 7, 4>;
using E49_7W = Cfg<49, 2, 25, 7, 8>;
using E25_1 = Cfg<25, 1, 25, 1, 4>;
using E25_2 = Cfg<25, 1, 25, 2, 4>;
using E25_4 = Cfg<25, 1, 25, 4, 4>;
using E25_7 = Cfg<25, 1, 25, 7, 4>;
using E81_2 = Cfg<81, 4, 21, 2, 8>;
using E81_4 = Cfg<81, 4, 21, 4, 8>;
using E81_7 = Cfg<81, 4, 21, 7, 8>;
using G28_1 = Cfg<0, 1, 28, 1, 4>;
using G28_4 = Cfg<0, 1, 28, 4, 4>;
using G60_1 = Cfg<0, 2, 30, 1, 4>;
using G60_4 = Cfg<0, 2, 30, 4, 4>;
using G120_2 = Cfg<0, 4, 30, 2, 8>;
using G120_4 = Cfg<0, 4, 30, 4, 8>;
using G148_2 = Cfg<0, 4, 37, 2, 8>;
using G148_4 = Cfg<0, 4, 37, 4, 8, 1>;     // 217 KB of shared memory: one CTA per SM
// accelerated EM-ADMM (two per-point state banks): 4 lanes of 13 slots per point, 7 points per lane,
// 448 point slots; 182 registers of state per thread, one CTA of 256 threads per SM; padded
// reduction rows (4 float4 would put every other lane's row store in the same banks)
using F49_7 = Cfg<49, 4, 13, 7, 8, 0, true>;
// the same for the batched launch: fewer point slots for small windows, and 5x5 patches (2 lanes of 13
// slots per point)
using F49_2 = Cfg<49, 4, 13, 2, 8, 0, true>;
using F49_4 = Cfg<49, 4, 13, 4, 8, 0, true>;
using F25_2 = Cfg<25, 2, 13, 2, 8, 0, true>;
using F25_4 = Cfg<25, 2, 13, 4, 8, 0, true>;

int launch_em_d49(const EmLaunch& L);
int launch_em_d25(const EmLaunch& L);
int launch_em_d81(const EmLaunch& L);
int launch_em_generic(const EmLaunch& L);
int launch_nlem_k7(const NlemLaunch& L);
int launch_nlem_k5(const NlemLaunch& L);
int launch_nlem_k9(const NlemLaunch& L);
}  // namespace nlemk

// Warm-start features of NLEM problems (Sec. 3 problems; the learned start point and penalty):
// for pixel i, with w_j = exp(-||P_i - P_j||^2 / h^2) over its clipped search window and
// p = w / sum w, the row [m (d), q (d), H, pmax] holds
//   m    = sum_j p_j P_j (not projected),
//   q    = the coordinate-wise lower weighted median (per coordinate, the smallest value whose
//          cumulative weight reaches half the total),
//   H    = -sum_j p_j ln p_j,   pmax = max_j p_j.
//
// One CTA of 128 threads per pixel at a time.  Only the pixel's tile, its weights, the weight
// map and the sort keys live on chip (about 22 KB at 7x7 patches and a 21x21 window), so several
// CTAs share an SM and hide each other's latency.
//   - weights: a thread per window point, the squared distance read from the tile;
//   - weighted mean: a thread per coordinate, summed over the window;
//   - medians: coordinate c = (pr, pc) of window point j = (jr, jc) is the tile value at
//     (jr + pr, jc + pc), so every coordinate's values are a shifted copy of one tile.  The tile
//     is sorted once (bitonic, 64-bit keys: order-preserving value bits, then position; each
//     thread holds 8 consecutive ranks, so distances 1-4 are swapped in registers, 8-128 by warp
//     shuffles and 256-512 through shared memory: 3 of the 55 stages need a barrier).  Per
//     coordinate the weights are summed along that order by reading the window's weight map
//     shifted by c; a zero border gives positions outside the shifted window weight 0.  Weights
//     are summed exactly, as 64-bit fixed point with 54 fraction bits (w <= 1 and n <= 1024 keep
//     every sum below 2^63): thread t sums ranks [8t, 8t + 8), a block-wide prefix gives each
//     thread the weight before its run, and the one thread whose run crosses half the total
//     re-walks it.  Coordinates go in chunks of 13, so each thread's sums stay in registers.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kernels.h"

namespace nlemk {
namespace featk {

constexpr int NT = 128, NW = NT / 32;
constexpr int SORT = 1024;                  // sorted entries: the tile has at most 32 x 32 values
constexpr int RPT = SORT / NT;              // ranks per thread
constexpr int CHUNK = 13;                   // coordinates per median pass
constexpr float kFix = 18014398509481984.0f;   // 2^54

__device__ __forceinline__ unsigned long long feat_key(float v, int u) {
  const unsigned int b = __float_as_uint(v);
  const unsigned int o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // ascending float order
  return ((unsigned long long)o << 32) | (unsigned int)u;
}
__device__ __forceinline__ float feat_value(unsigned long long k) {
  const unsigned int o = (unsigned int)(k >> 32);
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}
__device__ __forceinline__ int reflect(int x, int N) { return x < 0 ? -x : (x >= N ? 2 * N - 2 - x : x); }

// Shared-memory carve for window S and patch K (bytes), in this order: sort keys, weight map
// [MAPS][MAPS], median scratch, tile [(S+K-1)^2], weights [S^2].
__host__ __device__ inline int map_side(int S, int K) { return S + 2 * (K - 1); }
__host__ __device__ inline size_t smem_bytes(int S, int K) {
  const size_t m = (size_t)map_side(S, K);
  return 8 * ((size_t)SORT + m * m + (NW + 2) * CHUNK) + 4 * ((size_t)(S + K - 1) * (S + K - 1) + (size_t)S * S);
}

// Bitonic sort, ascending, of the SORT keys held RPT per thread in blocked order (thread t holds
// ranks RPT t .. RPT t + RPT - 1).  On return every thread holds its ranks of the sorted order in
// kv and the whole sorted order is in buf.
__device__ __forceinline__ void sort_keys(unsigned long long (&kv)[RPT], unsigned long long* __restrict__ buf) {
  static_assert(RPT == 8 && SORT == 1024, "the stage split below assumes 8 ranks per thread");
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 2; k <= SORT; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < RPT) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          if ((r & j) == 0) {
            const bool asc = k < RPT ? (r & k) == 0 : ((t * RPT) & k) == 0;
            const unsigned long long a = kv[r], b = kv[r | j];
            const bool sw = (a > b) == asc;
            kv[r] = sw ? b : a;
            kv[r | j] = sw ? a : b;
          }
        }
      } else {
        const bool lower = ((t * RPT) & j) == 0, asc = ((t * RPT) & k) == 0, keep_min = lower == asc;
        if (j < 32 * RPT) {
#pragma unroll
          for (int r = 0; r < RPT; ++r) {
            const unsigned long long o = __shfl_xor_sync(kFull, kv[r], j / RPT);
            kv[r] = keep_min ? (o < kv[r] ? o : kv[r]) : (o > kv[r] ? o : kv[r]);
          }
        } else {
          __syncthreads();
#pragma unroll
          for (int r = 0; r < RPT; ++r) buf[t * RPT + r] = kv[r];
          __syncthreads();
#pragma unroll
          for (int r = 0; r < RPT; ++r) {
            const unsigned long long o = buf[(t * RPT + r) ^ j];
            kv[r] = keep_min ? (o < kv[r] ? o : kv[r]) : (o > kv[r] ? o : kv[r]);
          }
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RPT; ++r) buf[t * RPT + r] = kv[r];
}

// Weighted medians of coordinates [C0, C0 + cn), cn <= CN: per-thread run sums, a block-wide
// prefix of them, and a re-walk of the run that crosses half the total.  off[r] is the
// weight-map offset of this thread's rank RPT t + r (-1 for padding).  Starts and ends with a
// barrier.
template <int D, int K, int CN>
__device__ __forceinline__ void medians(const int (&off)[RPT], const unsigned long long* __restrict__ keys,
                                     const unsigned long long* __restrict__ wmap,
                                     unsigned long long* __restrict__ scratch, int NTILE, int TC, int MC, int C0,
                                     int cn, float* __restrict__ fout) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  __syncthreads();
  // map offset of coordinate C0 + c: coordinate (pr, pc) reads entry (ur - pr + K-1, uc - pc + K-1)
  int coff[CN];
#pragma unroll
  for (int c = 0; c < CN; ++c) coff[c] = c < cn ? ((C0 + c) / K) * MC + (C0 + c) % K : 0;
  unsigned long long acc[CN];
#pragma unroll
  for (int c = 0; c < CN; ++c) acc[c] = 0ull;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    if (off[r] < 0) break;                                  // padding sorts last
    const unsigned long long* base = wmap + off[r];
#pragma unroll
    for (int c = 0; c < CN; ++c) acc[c] += c < cn ? base[-coff[c]] : 0ull;
  }
  unsigned long long incl[CN];
#pragma unroll
  for (int c = 0; c < CN; ++c) incl[c] = acc[c];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int c = 0; c < CN; ++c) {
      const unsigned long long v = __shfl_up_sync(kFull, incl[c], o);
      if (lane >= o) incl[c] += v;
    }
  }
  unsigned long long* wtot = scratch;                       // [NW][CN]
  unsigned long long* xlo = scratch + NW * CN;              // [CN] weight before the crossing run
  int* xrun = reinterpret_cast<int*>(xlo + CN);             // [CN] thread owning that run
  if (lane == 31) {
#pragma unroll
    for (int c = 0; c < CN; ++c) wtot[warp * CN + c] = incl[c];
  }
  __syncthreads();
  // every coordinate sums the same n weights, so one total serves all
  unsigned long long total = 0ull;
  for (int w = 0; w < NW; ++w) total += wtot[w * CN];
#pragma unroll
  for (int c = 0; c < CN; ++c) {
    unsigned long long before = 0ull;
    for (int w = 0; w < warp; ++w) before += wtot[w * CN + c];
    const unsigned long long lo = before + incl[c] - acc[c];   // weight before this run
    const unsigned long long hi = before + incl[c];            // weight through this run
    if (2ull * lo < total && 2ull * hi >= total) {
      xlo[c] = lo;
      xrun[c] = t;
    }
  }
  __syncthreads();
  for (int c = t; c < cn; c += NT) {
    const int pr = (C0 + c) / K, pc = (C0 + c) % K, run = xrun[c];
    unsigned long long cum = xlo[c];
    float med = 0.f;
    for (int r = run * RPT; r < run * RPT + RPT; ++r) {
      const unsigned long long k = keys[r];
      const int u = (int)(unsigned int)k;
      if (u >= NTILE) break;
      const int ur = u / TC, uc = u - ur * TC;
      cum += wmap[(ur - pr + K - 1) * MC + (uc - pc + K - 1)];
      med = feat_value(k);
      if (2ull * cum >= total) break;
    }
    fout[D + C0 + c] = med;
  }
  __syncthreads();
}

template <int D, int K>
__device__ __forceinline__ void all_medians(const int (&off)[RPT], const unsigned long long* keys,
                                            const unsigned long long* wmap, unsigned long long* scratch, int NTILE,
                                            int TC, int MC, float* fout) {
  constexpr int CN = D < CHUNK ? D : CHUNK;
#pragma unroll
  for (int c0 = 0; c0 < D; c0 += CN)
    medians<D, K, CN>(off, keys, wmap, scratch, NTILE, TC, MC, c0, D - c0 < CN ? D - c0 : CN, fout);
}

// CTA-wide sums of a and b and the maximum of m (deterministic order: warp shuffles, then the
// warps in order); every thread gets the results
__device__ __forceinline__ void block_stats(float& a, float& b, float& m) {
  __shared__ float s_part[3][NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(kFull, a, o);
    b += __shfl_xor_sync(kFull, b, o);
    m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
  }
  if (lane == 0) {
    s_part[0][warp] = a;
    s_part[1][warp] = b;
    s_part[2][warp] = m;
  }
  __syncthreads();
  a = b = m = 0.f;
  for (int w = 0; w < NW; ++w) {
    a += s_part[0][w];
    b += s_part[1][w];
    m = fmaxf(m, s_part[2][w]);
  }
}

template <int K>
__global__ void __launch_bounds__(NT, 4)
features_kernel(const float* __restrict__ img, int H, int W, int pitch, int S, float inv_h2,
                const int* __restrict__ pix_list, const long long* __restrict__ n_list, float* __restrict__ feats) {
  constexpr int D = K * K, HK = (K - 1) / 2;
  extern __shared__ unsigned long long fsm[];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int R = (S - 1) / 2, MAPS = map_side(S, K);
  unsigned long long* keys = fsm;
  unsigned long long* wmap = keys + SORT;
  unsigned long long* scratch = wmap + MAPS * MAPS;
  float* tile = reinterpret_cast<float*>(scratch + (NW + 2) * CHUNK);
  float* wv = tile + (S + K - 1) * (S + K - 1);
  const long long items = pix_list ? *n_list : (long long)H * W;
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const long long pix = pix_list ? (long long)pix_list[item] : item;
    float* fout = feats + item * (long long)(2 * D + 2);
    if (pix < 0 || pix >= (long long)H * W) {   // a listed index outside the image: a NaN row
      for (int i = t; i < 2 * D + 2; i += NT) fout[i] = __int_as_float(0x7fc00000);
      continue;
    }
    const int ir = (int)(pix / W), ic = (int)(pix - (long long)ir * W);
    const int r0 = max(ir - R, 0), r1 = min(ir + R, H - 1), c0 = max(ic - R, 0), c1 = min(ic + R, W - 1);
    const int nwr = r1 - r0 + 1, nwc = c1 - c0 + 1, n = nwr * nwc;
    const int TR = nwr + 2 * HK, TC = nwc + 2 * HK, NTILE = TR * TC;
    const int MC = nwc + 2 * (K - 1), MR = nwr + 2 * (K - 1);
    __syncthreads();   // the previous pixel is done with the shared buffers
    // tile rows r0-HK .. r1+HK, cols c0-HK .. c1+HK of the reflect-padded image (a warp per row)
    for (int tr = warp; tr < TR; tr += NW) {
      const float* grow = img + (size_t)reflect(r0 - HK + tr, H) * pitch;
      for (int tc = lane; tc < TC; tc += 32) tile[tr * TC + tc] = __ldg(grow + reflect(c0 - HK + tc, W));
    }
    for (int i = t; i < MR * MC; i += NT) wmap[i] = 0ull;
    __syncthreads();
    // weights, a thread per window point; the statistics for H and pmax on the way
    const float* pcen = tile + (ir - r0) * TC + (ic - c0);
    float sw = 0.f, swl = 0.f, wmax = 0.f;
    for (int j = t; j < n; j += NT) {
      const int jr = j / nwc, jc = j - jr * nwc;
      const float* pj = tile + jr * TC + jc;
      float d0 = 0.f, d1 = 0.f;
#pragma unroll
      for (int qr = 0; qr < K; ++qr) {
#pragma unroll
        for (int qc = 0; qc < K; ++qc) {
          const float e = pcen[qr * TC + qc] - pj[qr * TC + qc];
          if ((qr * K + qc) & 1) d1 = fmaf(e, e, d1); else d0 = fmaf(e, e, d0);
        }
      }
      const float w = expf(-(d0 + d1) * inv_h2);
      wv[j] = w;
      wmap[(jr + K - 1) * MC + jc + K - 1] = __float2ull_rz(w * kFix);
      sw += w;
      swl += w > 0.f ? w * logf(w) : 0.f;
      wmax = fmaxf(wmax, w);
    }
    block_stats(sw, swl, wmax);   // contains the barrier that publishes wv and wmap
    // weighted mean, a thread per coordinate (the window's rows in order, two partial sums)
    const float inv_w = 1.f / sw;
    for (int q = t; q < D; q += NT) {
      const int qr = q / K, qc = q - qr * K;
      float a0 = 0.f, a1 = 0.f;
      for (int jr = 0; jr < nwr; ++jr) {
        const float* trow = tile + (jr + qr) * TC + qc;
        const float* wrow = wv + jr * nwc;
        int jc = 0;
        for (; jc + 1 < nwc; jc += 2) {
          a0 = fmaf(wrow[jc], trow[jc], a0);
          a1 = fmaf(wrow[jc + 1], trow[jc + 1], a1);
        }
        if (jc < nwc) a0 = fmaf(wrow[jc], trow[jc], a0);
      }
      fout[q] = (a0 + a1) * inv_w;
    }
    if (t == 0) {
      fout[2 * D] = logf(sw) - swl * inv_w;
      fout[2 * D + 1] = wmax * inv_w;
    }
    // sort keys of the tile (position u = (ur, uc) row-major in the tile), RPT consecutive
    // positions per thread; padding past the tile sorts last
    unsigned long long kv[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int u = t * RPT + r;
      kv[r] = feat_key(u < NTILE ? tile[u] : __int_as_float(0x7f800000), u);
    }
    sort_keys(kv, keys);
    int off[RPT];   // weight-map offsets of this thread's ranks, decoded once for every chunk
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int u = (int)(unsigned int)kv[r];
      const int ur = u / TC, uc = u - ur * TC;
      off[r] = u < NTILE ? (ur + K - 1) * MC + (uc + K - 1) : -1;
    }
    all_medians<D, K>(off, keys, wmap, scratch, NTILE, TC, MC, fout);
  }
}

template <int K>
int launch(const float* img, int H, int W, int pitch, int S, float inv_h2, const int* pix_list, const long long* n_list,
           long long max_items, float* feats, int sm_count, cudaStream_t stream) {
  const size_t smem = smem_bytes(S, K);
  auto kern = features_kernel<K>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return (int)e;
  if (per_sm < 1) per_sm = 1;
  const long long items = pix_list ? max_items : (long long)H * W;
  long long grid = (long long)sm_count * per_sm * 16;
  if (grid > items) grid = items;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, NT, smem, stream>>>(img, H, W, pitch, S, inv_h2, pix_list, n_list, feats);
  return (int)cudaGetLastError();
}

}  // namespace featk

int launch_features(const float* img, int H, int W, int pitch, int patch, int S, float inv_h2, const int* pix_list,
                    const long long* n_list, long long max_items, float* feats, int sm_count, cudaStream_t stream) {
  if ((S + patch - 1) * (S + patch - 1) > featk::SORT) return -1;   // the tile must fit the sort
  switch (patch) {
    case 5: return featk::launch<5>(img, H, W, pitch, S, inv_h2, pix_list, n_list, max_items, feats, sm_count, stream);
    case 7: return featk::launch<7>(img, H, W, pitch, S, inv_h2, pix_list, n_list, max_items, feats, sm_count, stream);
    case 9: return featk::launch<9>(img, H, W, pitch, S, inv_h2, pix_list, n_list, max_items, feats, sm_count, stream);
    default: return -1;
  }
}

}  // namespace nlemk

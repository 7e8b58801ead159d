// Learned warm start for EM-ADMM: a 3-layer MLP (FP16 weights, FP32 arithmetic) maps the
// features of a problem [weighted mean m (d), coordinate-wise weighted median q (d), weight
// entropy H, largest normalised weight pmax] to a start point and a penalty:
//     x = normalise(f);  h1 = relu(W1 x + b1);  h2 = relu(W2 h1 + b2);  y = W3 h2 + b3
//     x0 = P_C(m + kDeltaScale * y[0:d]),  rho = exp(clamp(y[d], kLogRhoMin, kLogRhoMax))
// normalise: m, q -> (v - 127.5) / 64;  H -> H / log(nref);  pmax unchanged.
// Trained on solves the method itself produces, with hand-written forward, backward and Adam
// kernels; parameters live as an FP32 master copy (updated by Adam) plus the FP16 copy the
// forward pass reads.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "warmstart.h"

namespace nlemk {

namespace {

constexpr int kHid = kWsHidden;
constexpr int kSamples = 32;   // samples per CTA in the batched kernels

__device__ __forceinline__ float normalised(const float* f, int c, int d, float inv_lognref) {
  if (c < 2 * d) return (f[c] - 127.5f) * (1.f / 64.f);
  if (c == 2 * d) return f[c] * inv_lognref;
  return f[c];
}

// Forward pass over kSamples samples per CTA; kHid threads, thread i owns hidden unit i.
// Optionally keeps the normalised inputs and the pre-activations for the backward pass.
__global__ void __launch_bounds__(kHid) mlp_forward_kernel(const __half* __restrict__ w16, const float* __restrict__ feats,
                                                           long long B, int d, float inv_lognref, float* __restrict__ y,
                                                           float* __restrict__ xs, float* __restrict__ a1s,
                                                           float* __restrict__ a2s) {
  const int F = 2 * d + 2, O = d + 1;
  const __half* W1 = w16;
  const __half* b1 = W1 + kHid * F;
  const __half* W2 = b1 + kHid;
  const __half* b2 = W2 + kHid * kHid;
  const __half* W3 = b2 + kHid;
  const __half* b3 = W3 + O * kHid;
  extern __shared__ float sh[];
  float* x = sh;                        // [kSamples][F]
  float* h1 = x + kSamples * F;         // [kSamples][kHid]
  float* h2 = h1 + kSamples * kHid;     // [kSamples][kHid]
  const int t = threadIdx.x;
  const long long s0 = (long long)blockIdx.x * kSamples;
  const int ns = (int)((B - s0) < kSamples ? (B - s0) : kSamples);
  for (int i = t; i < kSamples * F; i += kHid) {
    const int s = i / F, c = i - s * F;
    x[i] = s < ns ? normalised(feats + (s0 + s) * F, c, d, inv_lognref) : 0.f;
  }
  __syncthreads();
  {
    float acc[kSamples];
    const float bb = __half2float(b1[t]);
#pragma unroll
    for (int s = 0; s < kSamples; ++s) acc[s] = bb;
    for (int j = 0; j < F; ++j) {
      const float wv = __half2float(W1[t * F + j]);
#pragma unroll
      for (int s = 0; s < kSamples; ++s) acc[s] = fmaf(wv, x[s * F + j], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < kSamples; ++s) {
      h1[s * kHid + t] = fmaxf(acc[s], 0.f);
      if (a1s && s < ns) a1s[(s0 + s) * kHid + t] = acc[s];
    }
  }
  __syncthreads();
  {
    float acc[kSamples];
    const float bb = __half2float(b2[t]);
#pragma unroll
    for (int s = 0; s < kSamples; ++s) acc[s] = bb;
    for (int j = 0; j < kHid; ++j) {
      const float wv = __half2float(W2[t * kHid + j]);
#pragma unroll
      for (int s = 0; s < kSamples; ++s) acc[s] = fmaf(wv, h1[s * kHid + j], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < kSamples; ++s) {
      h2[s * kHid + t] = fmaxf(acc[s], 0.f);
      if (a2s && s < ns) a2s[(s0 + s) * kHid + t] = acc[s];
    }
  }
  __syncthreads();
  for (int o = t; o < O; o += kHid) {
    float acc[kSamples];
    const float bb = __half2float(b3[o]);
#pragma unroll
    for (int s = 0; s < kSamples; ++s) acc[s] = bb;
    for (int j = 0; j < kHid; ++j) {
      const float wv = __half2float(W3[o * kHid + j]);
#pragma unroll
      for (int s = 0; s < kSamples; ++s) acc[s] = fmaf(wv, h2[s * kHid + j], acc[s]);
    }
    for (int s = 0; s < ns; ++s) y[(s0 + s) * O + o] = acc[s];
  }
  if (xs) {
    for (int i = t; i < ns * F; i += kHid) xs[s0 * F + i] = x[i];
  }
}

// dL/dy of L = (1/B) sum_b [ (1/d) sum_{c<d} (y - t)^2 + (y_d - t_d)^2 ], and the loss.
__global__ void mlp_loss_kernel(const float* __restrict__ y, const float* __restrict__ tgt, long long B, int d,
                                float* __restrict__ dy, float* __restrict__ loss) {
  const int O = d + 1;
  const long long total = B * O;
  float part = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % O);
    const float wgt = c < d ? 1.f / (float)d : 1.f;
    const float e = y[i] - tgt[i];
    part = fmaf(wgt * e, e, part);
    dy[i] = 2.f * wgt * e / (float)B;
  }
  if (loss) {
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part / (float)B);
  }
}

// Back-propagate to the hidden layers, per sample: da2 = (W3^T dy) * [a2 > 0],
// da1 = (W2^T da2) * [a1 > 0].  kHid threads per CTA, thread j owns hidden unit j.
__global__ void __launch_bounds__(kHid) mlp_backprop_kernel(const __half* __restrict__ w16, const float* __restrict__ dy,
                                                            const float* __restrict__ a1s, const float* __restrict__ a2s,
                                                            long long B, int d, float* __restrict__ da1,
                                                            float* __restrict__ da2) {
  const int F = 2 * d + 2, O = d + 1;
  const __half* W2 = w16 + kHid * F + kHid;
  const __half* W3 = W2 + kHid * kHid + kHid;
  __shared__ float sdy[kSamples][96];
  __shared__ float sda2[kSamples][kHid];
  const int t = threadIdx.x;
  const long long s0 = (long long)blockIdx.x * kSamples;
  const int ns = (int)((B - s0) < kSamples ? (B - s0) : kSamples);
  for (int i = t; i < kSamples * O; i += kHid) {
    const int s = i / O, o = i - s * O;
    sdy[s][o] = s < ns ? dy[(s0 + s) * O + o] : 0.f;
  }
  __syncthreads();
  {
    float acc[kSamples];
#pragma unroll
    for (int s = 0; s < kSamples; ++s) acc[s] = 0.f;
    for (int o = 0; o < O; ++o) {
      const float wv = __half2float(W3[o * kHid + t]);
#pragma unroll
      for (int s = 0; s < kSamples; ++s) acc[s] = fmaf(wv, sdy[s][o], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < kSamples; ++s) {
      const float g = (s < ns && a2s[(s0 + s) * kHid + t] > 0.f) ? acc[s] : 0.f;
      sda2[s][t] = g;
      if (s < ns) da2[(s0 + s) * kHid + t] = g;
    }
  }
  __syncthreads();
  {
    float acc[kSamples];
#pragma unroll
    for (int s = 0; s < kSamples; ++s) acc[s] = 0.f;
    for (int i = 0; i < kHid; ++i) {
      const float wv = __half2float(W2[i * kHid + t]);
#pragma unroll
      for (int s = 0; s < kSamples; ++s) acc[s] = fmaf(wv, sda2[s][i], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < kSamples; ++s)
      if (s < ns) da1[(s0 + s) * kHid + t] = a1s[(s0 + s) * kHid + t] > 0.f ? acc[s] : 0.f;
  }
}

// Parameter gradients, one thread per parameter, summed over the batch in sample order:
// gW1 = da1^T x, gb1 = sum da1, gW2 = da2^T relu(a1), gb2, gW3 = dy^T relu(a2), gb3.
__global__ void mlp_param_grad_kernel(const float* __restrict__ xs, const float* __restrict__ a1s,
                                      const float* __restrict__ a2s, const float* __restrict__ da1,
                                      const float* __restrict__ da2, const float* __restrict__ dy, long long B, int d,
                                      float* __restrict__ grad) {
  const int F = 2 * d + 2, O = d + 1;
  const long long nW1 = (long long)kHid * F, nW2 = (long long)kHid * kHid, nW3 = (long long)O * kHid;
  const long long P = nW1 + kHid + nW2 + kHid + nW3 + O;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    long long r = k;
    if (r < nW1) {
      const int i = (int)(r / F), j = (int)(r % F);
      for (long long b = 0; b < B; ++b) s = fmaf(da1[b * kHid + i], xs[b * F + j], s);
    } else if ((r -= nW1) < kHid) {
      for (long long b = 0; b < B; ++b) s += da1[b * kHid + r];
    } else if ((r -= kHid) < nW2) {
      const int i = (int)(r / kHid), j = (int)(r % kHid);
      for (long long b = 0; b < B; ++b) s = fmaf(da2[b * kHid + i], fmaxf(a1s[b * kHid + j], 0.f), s);
    } else if ((r -= nW2) < kHid) {
      for (long long b = 0; b < B; ++b) s += da2[b * kHid + r];
    } else if ((r -= kHid) < nW3) {
      const int i = (int)(r / kHid), j = (int)(r % kHid);
      for (long long b = 0; b < B; ++b) s = fmaf(dy[b * O + i], fmaxf(a2s[b * kHid + j], 0.f), s);
    } else {
      r -= nW3;
      for (long long b = 0; b < B; ++b) s += dy[b * O + r];
    }
    grad[k] = s;
  }
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters, then the FP16 copy.
__global__ void adam_kernel(float* __restrict__ p, __half* __restrict__ p16, float* __restrict__ m,
                            float* __restrict__ v, const float* __restrict__ g, long long P, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += (long long)gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    p[k] = pk;
    p16[k] = __float2half_rn(pk);
  }
}

__global__ void to_half_kernel(const float* __restrict__ p, __half* __restrict__ p16, long long P) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < P; k += (long long)gridDim.x * blockDim.x)
    p16[k] = __float2half_rn(p[k]);
}

// (x0, rho) from the network output and the weighted mean in the features.
__global__ void apply_kernel(const float* __restrict__ feats, const float* __restrict__ y, long long B, int d, float lo,
                             float hi, float* __restrict__ x0, float* __restrict__ rho) {
  const int F = 2 * d + 2, O = d + 1;
  const long long total = B * d;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / d;
    const int c = (int)(i - b * d);
    const float v = feats[b * F + c] + kDeltaScale * y[b * O + c];
    x0[i] = fminf(fmaxf(v, lo), hi);
    if (c == 0) rho[b] = expf(fminf(fmaxf(y[b * O + d], kLogRhoMin), kLogRhoMax));
  }
}

// Compact the pixels that reached the cap without meeting the stopping rule.
__global__ void fallback_list_kernel(const int* __restrict__ iters_used, long long npix, int cap, int* __restrict__ list,
                                     long long* __restrict__ count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
    if (iters_used[i] >= cap) {
      const unsigned long long k = atomicAdd(reinterpret_cast<unsigned long long*>(count), 1ull);
      list[k] = (int)i;
    }
  }
}

// the entries of a caller's pixel list that lie in [0, total), in any order, and their count
// (one atomic per warp: the ballot of valid entries and their ranks within the warp)
__global__ void compact_list_kernel(const int* __restrict__ in, long long n, long long total, int* __restrict__ out,
                                    long long* __restrict__ count) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long i = base + threadIdx.x;
    const int v = i < n ? in[i] : -1;
    const bool ok = i < n && v >= 0 && (long long)v < total;
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    unsigned long long pos = 0;
    if (lane == 0 && m) pos = atomicAdd(reinterpret_cast<unsigned long long*>(count), (unsigned long long)__popc(m));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    if (ok) out[pos + __popc(m & ((1u << lane) - 1u))] = v;
  }
}

__global__ void gather_rows_kernel(const float* __restrict__ src, int cols, const int* __restrict__ rows,
                                   long long nrows, float* __restrict__ dst) {
  const long long total = nrows * cols;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / cols;
    dst[i] = src[(long long)rows[r] * cols + (i - r * cols)];
  }
}

int grid_for(long long n, int threads, int sm_count) {
  long long g = (n + threads - 1) / threads;
  const long long cap = (long long)sm_count * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

long long ws_num_params(int d) {
  const int F = 2 * d + 2, O = d + 1;
  return (long long)kHid * F + kHid + (long long)kHid * kHid + kHid + (long long)O * kHid + O;
}

int ws_forward(const WsModel& m, const float* feats, long long B, float* y, float* xs, float* a1s, float* a2s,
               int sm_count, cudaStream_t s) {
  (void)sm_count;
  if (B <= 0) return 0;
  const int F = 2 * m.d + 2;
  const size_t smem = (size_t)(kSamples * F + 2 * kSamples * kHid) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const long long blocks = (B + kSamples - 1) / kSamples;
  mlp_forward_kernel<<<(unsigned)blocks, kHid, smem, s>>>(m.w16, feats, B, m.d, 1.f / logf(m.nref), y, xs, a1s, a2s);
  return (int)cudaGetLastError();
}

int ws_loss_grad(const WsModel& m, WsScratch& sc, const float* feats, const float* tgt, long long B, float* loss,
                 float* grad, int sm_count, cudaStream_t s) {
  if (B <= 0 || B > sc.cap) return -1;
  const int O = m.d + 1;
  int rc = ws_forward(m, feats, B, sc.y, sc.xs, sc.a1, sc.a2, sm_count, s);
  if (rc) return rc;
  if (loss) cudaMemsetAsync(loss, 0, sizeof(float), s);
  mlp_loss_kernel<<<grid_for(B * O, 256, sm_count), 256, 0, s>>>(sc.y, tgt, B, m.d, sc.dy, loss);
  const long long blocks = (B + kSamples - 1) / kSamples;
  mlp_backprop_kernel<<<(unsigned)blocks, kHid, 0, s>>>(m.w16, sc.dy, sc.a1, sc.a2, B, m.d, sc.da1, sc.da2);
  const long long P = ws_num_params(m.d);
  mlp_param_grad_kernel<<<(unsigned)((P + 127) / 128), 128, 0, s>>>(sc.xs, sc.a1, sc.a2, sc.da1, sc.da2, sc.dy, B,
                                                                    m.d, grad);
  return (int)cudaGetLastError();
}

int ws_adam(WsModel& m, const float* grad, float lr, int sm_count, cudaStream_t s) {
  const long long P = ws_num_params(m.d);
  m.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)m.step), c2 = 1.f - powf(b2, (float)m.step);
  adam_kernel<<<grid_for(P, 256, sm_count), 256, 0, s>>>(m.p32, m.w16, m.adam_m, m.adam_v, grad, P, lr, b1, b2, 1e-8f,
                                                         c1, c2);
  return (int)cudaGetLastError();
}

int ws_sync_half(WsModel& m, int sm_count, cudaStream_t s) {
  const long long P = ws_num_params(m.d);
  to_half_kernel<<<grid_for(P, 256, sm_count), 256, 0, s>>>(m.p32, m.w16, P);
  return (int)cudaGetLastError();
}

int ws_apply(const float* feats, const float* y, long long B, int d, float lo, float hi, float* x0, float* rho,
             int sm_count, cudaStream_t s) {
  if (B <= 0) return 0;
  apply_kernel<<<grid_for(B * d, 256, sm_count), 256, 0, s>>>(feats, y, B, d, lo, hi, x0, rho);
  return (int)cudaGetLastError();
}

int ws_gather_rows(const float* src, int cols, const int* rows, long long nrows, float* dst, int sm_count,
                   cudaStream_t s) {
  gather_rows_kernel<<<grid_for(nrows * cols, 256, sm_count), 256, 0, s>>>(src, cols, rows, nrows, dst);
  return (int)cudaGetLastError();
}

int ws_compact_list(const int* in, long long n, long long total, int* out, long long* count, int sm_count,
                    cudaStream_t s) {
  cudaMemsetAsync(count, 0, sizeof(long long), s);
  if (n > 0) compact_list_kernel<<<grid_for(n, 256, sm_count), 256, 0, s>>>(in, n, total, out, count);
  return (int)cudaGetLastError();
}

int ws_fallback_list(const int* iters_used, long long npix, int cap, int* list, long long* count, int sm_count,
                     cudaStream_t s) {
  cudaMemsetAsync(count, 0, sizeof(long long), s);
  fallback_list_kernel<<<grid_for(npix, 256, sm_count), 256, 0, s>>>(iters_used, npix, cap, list, count);
  return (int)cudaGetLastError();
}


// ------------------------------------------------------------------------------------------
// training labels: the penalty that reached the tolerance first, and the targets
// ------------------------------------------------------------------------------------------
__global__ void label_init_kernel(long long n, int* __restrict__ best_it, float* __restrict__ best_rho) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    best_it[i] = 0x7fffffff;
    best_rho[i] = 1.f;
  }
}

// after the solve with penalty rho: pixels whose iteration count beats the best so far take it
// (strictly fewer iterations, so ties keep the earlier penalty of the grid)
__global__ void label_select_kernel(const int* __restrict__ iters_img, long long total, const int* __restrict__ pix,
                                    long long n, float rho, int* __restrict__ best_it, float* __restrict__ best_rho) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (pix[i] < 0 || pix[i] >= total) continue;   // outside the image: never solved
    const int it = iters_img[pix[i]];
    if (it < best_it[i]) {
      best_it[i] = it;
      best_rho[i] = rho;
    }
  }
}

// rho_map[pix[i]] = best_rho[i] (every other entry 1); counts[j] += #{i : best_rho[i] == grid[j]}
__global__ void label_scatter_kernel(const int* __restrict__ pix, long long n, long long total,
                                     const float* __restrict__ best_rho, float* __restrict__ rho_map,
                                     const float* __restrict__ grid, int n_rho, unsigned long long* __restrict__ counts) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (pix[i] < 0 || pix[i] >= total) continue;
    const float r = best_rho[i];
    rho_map[pix[i]] = r;
    for (int j = 0; j < n_rho; ++j)
      if (grid[j] == r) {
        atomicAdd(counts + j, 1ull);
        break;
      }
  }
}

// targets[i] = [(z[pix[i]] - m_i) / kDeltaScale, ln best_rho[i]] with m_i = feats[i][0:d]; NaN for
// list entries outside the image
__global__ void label_targets_kernel(const float* __restrict__ z_full, long long total, const int* __restrict__ pix,
                                     long long n, int d, const float* __restrict__ feats,
                                     const float* __restrict__ best_rho, float* __restrict__ targets) {
  const long long elems = n * (long long)(d + 1);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < elems;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / (d + 1);
    const int c = (int)(e - i * (d + 1));
    const int p = pix[i];
    if (p < 0 || p >= total) {
      targets[e] = __int_as_float(0x7fc00000);
      continue;
    }
    targets[e] = c < d ? (z_full[(long long)p * d + c] - feats[i * (2 * d + 2) + c]) / kDeltaScale
                       : logf(best_rho[i]);
  }
}

__global__ void fill_f32_kernel(float* __restrict__ p, long long n, float v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

namespace {
inline int grid_for(long long work, int sm_count) {
  long long g = (work + 255) / 256, cap = (long long)sm_count * 8;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}
}  // namespace

int ws_label_init(long long n, int* best_it, float* best_rho, int sm_count, cudaStream_t s) {
  label_init_kernel<<<grid_for(n, sm_count), 256, 0, s>>>(n, best_it, best_rho);
  return (int)cudaGetLastError();
}
int ws_label_select(const int* iters_img, long long total, const int* pix, long long n, float rho, int* best_it,
                    float* best_rho, int sm_count, cudaStream_t s) {
  label_select_kernel<<<grid_for(n, sm_count), 256, 0, s>>>(iters_img, total, pix, n, rho, best_it, best_rho);
  return (int)cudaGetLastError();
}
int ws_label_scatter(const int* pix, long long n, long long total, const float* best_rho, float* rho_map,
                     const float* grid, int n_rho, unsigned long long* counts, int sm_count, cudaStream_t s) {
  label_scatter_kernel<<<grid_for(n, sm_count), 256, 0, s>>>(pix, n, total, best_rho, rho_map, grid, n_rho, counts);
  return (int)cudaGetLastError();
}
int ws_label_targets(const float* z_full, long long total, const int* pix, long long n, int d, const float* feats,
                     const float* best_rho, float* targets, int sm_count, cudaStream_t s) {
  label_targets_kernel<<<grid_for(n * (d + 1), sm_count), 256, 0, s>>>(z_full, total, pix, n, d, feats, best_rho,
                                                                       targets);
  return (int)cudaGetLastError();
}
int ws_fill(float* p, long long n, float v, int sm_count, cudaStream_t s) {
  fill_f32_kernel<<<grid_for(n, sm_count), 256, 0, s>>>(p, n, v);
  return (int)cudaGetLastError();
}

}  // namespace nlemk

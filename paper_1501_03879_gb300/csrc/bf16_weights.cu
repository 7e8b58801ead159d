// Mixed-precision NLEM weights: the patch cross terms <P_i, P_j> of Sec. 3's weights
// w_ij = exp(-||P_i - P_j||^2 / h^2) on the 5th-generation tensor cores (tcgen05.mma,
// kind::f16 with BF16 operands, FP32 accumulation in Tensor Memory), with
// ||P_i - P_j||^2 = ||P_i||^2 + ||P_j||^2 - 2 <P_i, P_j> and the norms in FP32.
//
// One CTA takes a block of 8 x 16 = 128 pixels (M = 128).  Their search windows together
// cover (8 + 2R) x (16 + 2R) window centres (the block's union window), processed in chunks
// of N = 256 centres: A = the block's patches [128 x KP], B = the chunk's patches [256 x KP]
// (bf16, K-major, no swizzle, KP = d rounded up to 16), D = A B^T in TMEM (lane m = pixel m).
// Each thread then reads its pixel's row of D, keeps the centres inside its clipped window
// and writes w_ij into the weight table [pixel][j] (j in the NLEM window order).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "tmem.cuh"

namespace nlemk {

namespace {

constexpr int kBR = 8, kBC = 16, kBM = kBR * kBC;   // pixel block
constexpr int kN = 256;                             // centres per MMA chunk
constexpr uint32_t kTmemCols = 256;                 // FP32 accumulator tile 128 x 256
constexpr uint32_t kWaitTries = 1u << 22;           // bound on mbarrier polls

// tcgen05 shared-memory matrix descriptor for a K-major operand without swizzling: core
// matrices of 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo = byte
// step between 8-row groups.  Fields: start>>4 [0,14), lbo>>4 [16,30), sbo>>4 [32,46),
// descriptor version 1 [46,48), base offset 0, layout type 0 (no swizzle) [61,64).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Arrive on the mbarrier once every MMA this thread issued has completed.
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// Bounded wait for the mbarrier phase with the given parity; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitTries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Make this thread's shared-memory writes visible to the tensor cores' (async proxy) reads.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ int reflect_clamped(int x, int N) {
  x = x < 0 ? -x : (x >= N ? 2 * N - 2 - x : x);
  return x < 0 ? 0 : (x >= N ? N - 1 : x);   // far-outside rows only feed skipped centres
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // round to nearest even
  return *reinterpret_cast<uint32_t*>(&v);
}

template <int K, int KP>
__global__ void __launch_bounds__(kBM, 1)
bf16_weights_kernel(const float* __restrict__ img, int H, int W, int pitch, int S, float inv_h2,
                    float* __restrict__ wtab, int* __restrict__ err) {
  constexpr int D = K * K, HK = (K - 1) / 2, NKC = KP / 8;   // 16-byte K chunks per row
  constexpr uint32_t SBO = NKC * 128, LBO = 128;
  static_assert(KP % 16 == 0 && KP >= D, "K padding");
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Asm = smem;                                  // [128 x KP] bf16
  uint8_t* Bsm = smem + kBM * KP * 2;                   // [256 x KP] bf16
  float* tile = reinterpret_cast<float*>(Bsm + kN * KP * 2);
  __shared__ uint64_t mbar;
  __shared__ uint32_t s_tmem;

  const int t = threadIdx.x, warp = t >> 5;
  const int R = (S - 1) / 2;
  const int r0 = blockIdx.y * kBR, c0 = blockIdx.x * kBC;
  const int UR = kBR + 2 * R, UC = kBC + 2 * R, NU = UR * UC;   // union window centres
  const int TR = UR + 2 * HK, TC = UC + 2 * HK;
  float* unorm = tile + TR * TC;                                // ||P_u||^2 per centre

  if (warp == 0) {
    tmem_alloc(&s_tmem, kTmemCols);
    tmem_relinquish();
  }
  if (t == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // tile of the reflect-padded image: union centre (ur, uc) is image (r0-R+ur, c0-R+uc) and
  // its patch is tile[ur .. ur+K-1][uc .. uc+K-1]
  for (int i = t; i < TR * TC; i += kBM) {
    const int tr = i / TC, tc = i - tr * TC;
    tile[i] = __ldg(img + (size_t)reflect_clamped(r0 - R - HK + tr, H) * pitch + reflect_clamped(c0 - R - HK + tc, W));
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem_d = s_tmem;

  // A: the block's patches; pixel m = (m / 16, m % 16) sits at union centre (mr+R, mc+R)
  for (int idx = t; idx < kBM * NKC; idx += kBM) {
    const int m = idx % kBM, kc = idx / kBM;
    const int mr = m / kBC, mc = m % kBC;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e;
      v[e] = k < D ? tile[(mr + R + k / K) * TC + (mc + R + k % K)] : 0.f;
    }
    uint4 q = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    *reinterpret_cast<uint4*>(Asm + (m / 8) * SBO + kc * 128 + (m % 8) * 16) = q;
  }
  for (int u = t; u < NU; u += kBM) {
    const int ur = u / UC, uc = u - ur * UC;
    float s = 0.f;
    for (int k = 0; k < D; ++k) {
      const float x = tile[(ur + k / K) * TC + (uc + k % K)];
      s = fmaf(x, x, s);
    }
    unorm[u] = s;
  }
  // this thread's pixel
  const int mr = t / kBC, mc = t % kBC;
  const int pr = r0 + mr, pc = c0 + mc;
  const bool pix_ok = pr < H && pc < W;
  float pnorm = 0.f;
  for (int k = 0; k < D; ++k) {
    const float x = tile[(mr + R + k / K) * TC + (mc + R + k % K)];
    pnorm = fmaf(x, x, pnorm);
  }
  const int rw0 = max(pr - R, 0), cw0 = max(pc - R, 0);
  const int nwc = min(pc + R, W - 1) - cw0 + 1;
  float* wrow = wtab + ((size_t)pr * W + pc) * (size_t)(S * S);
  constexpr uint32_t IDESC = idesc_bf16_f32(kBM, kN);
  bool ok = true;
  (void)ok;

  const int nchunks = (NU + kN - 1) / kN;
  for (int ch = 0; ch < nchunks; ++ch) {
    for (int idx = t; idx < kN * NKC; idx += kBM) {   // B: this chunk's centres
      const int nn = idx % kN, kc = idx / kN;
      const int u = ch * kN + nn;
      float v[8];
      if (u < NU) {
        const int ur = u / UC, uc = u - ur * UC;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = kc * 8 + e;
          v[e] = k < D ? tile[(ur + k / K) * TC + (uc + k % K)] : 0.f;
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.f;
      }
      uint4 q = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
      *reinterpret_cast<uint4*>(Bsm + (nn / 8) * SBO + kc * 128 + (nn % 8) * 16) = q;
    }
    fence_proxy_async_smem();
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (t == 0) {
      const uint32_t a0 = smem_u32(Asm), b0 = smem_u32(Bsm);
#pragma unroll
      for (int kk = 0; kk < KP / 16; ++kk)   // K = 16 per MMA = two 16-byte core matrices
        mma_bf16(tmem_d, smem_desc(a0 + kk * 2 * LBO, LBO, SBO), smem_desc(b0 + kk * 2 * LBO, LBO, SBO), IDESC,
                 kk > 0 ? 1u : 0u);
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, (uint32_t)(ch & 1));
    ok = __syncthreads_and(ok);   // one decision for the whole CTA
    if (!ok) {
      if (t == 0) atomicExch(err, 1);
      break;
    }
    tmem_fence_after_sync();
    // row t of D: this pixel against the chunk's 256 centres
    const uint32_t trow = tmem_d + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int cb = 0; cb < kN; cb += 32) {
      uint32_t v[32];
      tmem_ld32(trow + cb, v);
      tmem_wait_ld(v);
      if (!pix_ok) continue;
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int u = ch * kN + cb + e;
        if (u >= NU) break;
        const int ur = u / UC, uc = u - ur * UC;
        const int dr = ur - mr - R, dc = uc - mc - R;
        const int ir = r0 - R + ur, ic = c0 - R + uc;
        if (dr < -R || dr > R || dc < -R || dc > R || ir < 0 || ir >= H || ic < 0 || ic >= W) continue;
        const float D2 = fmaxf(pnorm + unorm[u] - 2.f * __uint_as_float(v[e]), 0.f);
        wrow[(ir - rw0) * nwc + (ic - cw0)] = expf(-D2 * inv_h2);
      }
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  if (warp == 0) tmem_dealloc(tmem_d, kTmemCols);
}

template <int K, int KP>
int launch_weights(const float* img, int H, int W, int pitch, int S, float inv_h2, float* wtab, int* err,
                   cudaStream_t stream) {
  const int R = (S - 1) / 2;
  const int TR = kBR + 2 * R + (K - 1), TC = kBC + 2 * R + (K - 1);
  const size_t smem = (size_t)kBM * KP * 2 + (size_t)kN * KP * 2 + ((size_t)TR * TC + (size_t)(kBR + 2 * R) * (kBC + 2 * R)) * 4;
  if (smem > 200 * 1024) return -1;
  auto kern = bf16_weights_kernel<K, KP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  dim3 grid((W + kBC - 1) / kBC, (H + kBR - 1) / kBR);
  kern<<<grid, kBM, smem, stream>>>(img, H, W, pitch, S, inv_h2, wtab, err);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_bf16_weights(const float* img, int H, int W, int pitch, int patch, int S, float inv_h2, float* wtab,
                        int* err, cudaStream_t stream) {
  switch (patch) {
    case 5: return launch_weights<5, 32>(img, H, W, pitch, S, inv_h2, wtab, err, stream);
    case 7: return launch_weights<7, 64>(img, H, W, pitch, S, inv_h2, wtab, err, stream);
    case 9: return launch_weights<9, 96>(img, H, W, pitch, S, inv_h2, wtab, err, stream);
    default: return -1;
  }
}

}  // namespace nlemk

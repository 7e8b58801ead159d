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
constexpr uint32_t kWaitTries = 1u << 22;           // default bound on mbarrier polls
constexpr int kScrRow = 36;                          // floats per lane of epilogue scratch (16-byte rows,
                                                     // conflict-free 16-byte stores across 8 lanes)

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
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t tries) {
  for (uint32_t i = 0; i < tries; ++i) {
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

// Pack one K x K patch (its top-left corner at src, tile row stride TC) into row n of a
// K-major, non-swizzled operand: element (n, k) at (n / 8) * SBO + (k / 8) * 128 + (n % 8) * 16
// + (k % 8) * 2 bytes.  Returns the FP32 squared norm of the (unrounded) patch, summed in k
// order.  zero: stage a row of zeros (no centre).
template <int K, int KP>
__device__ __forceinline__ float stage_patch(const float* __restrict__ src, int TC, uint8_t* __restrict__ dst, int n,
                                             bool zero) {
  constexpr int D = K * K, NKC = KP / 8;
  constexpr uint32_t SBO = NKC * 128;
  uint8_t* row = dst + (n / 8) * SBO + (n % 8) * 16;
  float norm = 0.f;
#pragma unroll
  for (int kc = 0; kc < NKC; ++kc) {
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e;
      v[e] = (k < D && !zero) ? src[(k / K) * TC + (k % K)] : 0.f;
      if (k < D) norm = fmaf(v[e], v[e], norm);
    }
    *reinterpret_cast<uint4*>(row + kc * 128) =
        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
  }
  return norm;
}

template <int K, int KP>
__global__ void __launch_bounds__(kBM, 1)
bf16_weights_kernel(const float* __restrict__ img, int H, int W, int pitch, int S, float inv_h2,
                    float* __restrict__ wtab, int* __restrict__ err, uint32_t wait_tries, int issue_mma) {
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
  float* scratch = reinterpret_cast<float*>(
      reinterpret_cast<uintptr_t>(unorm + NU + 3) & ~(uintptr_t)15);  // [128][kScrRow], 16-byte aligned

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
  for (int tr = warp; tr < TR; tr += kBM / 32) {   // a warp per tile row, lanes along it
    const float* grow = img + (size_t)reflect_clamped(r0 - R - HK + tr, H) * pitch;
    for (int tc = t & 31; tc < TC; tc += 32) tile[tr * TC + tc] = __ldg(grow + reflect_clamped(c0 - R - HK + tc, W));
  }
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  const uint32_t tmem_d = s_tmem;

  // A: the block's patches, a thread per pixel; pixel m = (m / 16, m % 16) sits at union
  // centre (mr+R, mc+R).  Its FP32 norm comes out of the same pass.
  const int mr = t / kBC, mc = t % kBC;
  const float pnorm = stage_patch<K, KP>(tile + (mr + R) * TC + (mc + R), TC, Asm, t, false);
  const int pr = r0 + mr, pc = c0 + mc;
  const bool pix_ok = pr < H && pc < W;
  // this pixel's search window clipped to the image, in union coordinates
  const int ur_lo = max(pr - R, 0) - r0 + R, ur_hi = min(pr + R, H - 1) - r0 + R;
  const int uc_lo = max(pc - R, 0) - c0 + R, uc_hi = min(pc + R, W - 1) - c0 + R;
  const int nwc = uc_hi - uc_lo + 1;
  float* wrow = wtab + ((size_t)pr * W + pc) * (size_t)(S * S);
  constexpr uint32_t IDESC = idesc_bf16_f32(kBM, kN);
  bool ok = true;
  (void)ok;

  const int nchunks = (NU + kN - 1) / kN;
  for (int ch = 0; ch < nchunks; ++ch) {
    // B: this chunk's centres, a thread per centre (and its FP32 norm)
    for (int nn = t; nn < kN; nn += kBM) {
      const int u = ch * kN + nn;
      const bool live = u < NU;
      const int ur = live ? u / UC : 0, uc = live ? u - ur * UC : 0;
      const float nrm = stage_patch<K, KP>(tile + ur * TC + uc, TC, Bsm, nn, !live);
      if (live) unorm[u] = nrm;
    }
    fence_proxy_async_smem();
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (t == 0 && issue_mma) {   // issue_mma = 0 only in the timeout self-test: nothing commits
      const uint32_t a0 = smem_u32(Asm), b0 = smem_u32(Bsm);
#pragma unroll
      for (int kk = 0; kk < KP / 16; ++kk)   // K = 16 per MMA = two 16-byte core matrices
        mma_bf16(tmem_d, smem_desc(a0 + kk * 2 * LBO, LBO, SBO), smem_desc(b0 + kk * 2 * LBO, LBO, SBO), IDESC,
                 kk > 0 ? 1u : 0u);
      mma_commit(&mbar);
    }
    ok = mbar_wait(&mbar, (uint32_t)(ch & 1), wait_tries);
    ok = __syncthreads_and(ok);   // one decision for the whole CTA
    if (!ok) {
      // flag the timeout, give tensor-core work still in flight one more bounded wait, then
      // leave the chunk loop to free TMEM
      if (t == 0) atomicExch(err, 1);
      if (issue_mma) (void)mbar_wait(&mbar, (uint32_t)(ch & 1), wait_tries);
      __syncthreads();
      break;
    }
    tmem_fence_after_sync();
    // row t of D: this pixel against the chunk's 256 centres, 32 columns at a time.  The 32
    // dot products go to this lane's own scratch row (16-byte stores), and the lane then walks
    // only its own window's columns in the block: a run per union row, at most three rows.
    const uint32_t trow = tmem_d + ((uint32_t)(warp * 32) << 16);
    float* my = scratch + t * kScrRow;
#pragma unroll 1
    for (int cb = 0; cb < kN; cb += 32) {
      const int u0 = ch * kN + cb;
      if (u0 >= NU) break;                       // the same for every thread
      uint32_t v[32];
      tmem_ld32(trow + cb, v);
      tmem_wait_ld(v);
      if (!pix_ok) continue;
#pragma unroll
      for (int e = 0; e < 32; e += 4)
        *reinterpret_cast<float4*>(my + e) = make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]),
                                                         __uint_as_float(v[e + 2]), __uint_as_float(v[e + 3]));
      const int uend = min(u0 + 32, NU);          // exclusive
      for (int ur = max(u0 / UC, ur_lo); ur <= ur_hi && ur * UC < uend; ++ur) {
        const int a = max(ur * UC + uc_lo, u0), b = min(ur * UC + uc_hi + 1, uend);
        float* dst = wrow + (ur - ur_lo) * nwc - (ur * UC + uc_lo);   // indexed by u
        for (int u = a; u < b; ++u) {
          const float D2 = fmaxf(pnorm + unorm[u] - 2.f * my[u - u0], 0.f);
          dst[u] = expf(-D2 * inv_h2);
        }
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
                   cudaStream_t stream, uint32_t wait_tries, int issue_mma) {
  const int R = (S - 1) / 2;
  const int TR = kBR + 2 * R + (K - 1), TC = kBC + 2 * R + (K - 1);
  const size_t smem = (size_t)kBM * KP * 2 + (size_t)kN * KP * 2 +
                      ((size_t)TR * TC + (size_t)(kBR + 2 * R) * (kBC + 2 * R) + 4 + (size_t)kBM * kScrRow) * 4;
  if (smem > 200 * 1024) return -1;
  auto kern = bf16_weights_kernel<K, KP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  dim3 grid((W + kBC - 1) / kBC, (H + kBR - 1) / kBR);
  kern<<<grid, kBM, smem, stream>>>(img, H, W, pitch, S, inv_h2, wtab, err, wait_tries, issue_mma);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_bf16_weights(const float* img, int H, int W, int pitch, int patch, int S, float inv_h2, float* wtab,
                        int* err, cudaStream_t stream, uint32_t wait_tries, int issue_mma) {
  if (wait_tries == 0) wait_tries = kWaitTries;
  if (S < 1 || S > 31) return -1;   // the compiled range (window <= 31)
  switch (patch) {
    case 5: return launch_weights<5, 32>(img, H, W, pitch, S, inv_h2, wtab, err, stream, wait_tries, issue_mma);
    case 7: return launch_weights<7, 64>(img, H, W, pitch, S, inv_h2, wtab, err, stream, wait_tries, issue_mma);
    case 9: return launch_weights<9, 96>(img, H, W, pitch, S, inv_h2, wtab, err, stream, wait_tries, issue_mma);
    default: return -1;
  }
}

}  // namespace nlemk

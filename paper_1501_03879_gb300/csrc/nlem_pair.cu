// NLEM (Sec. 3, Eq. L1regression) with 7x7 patches, two horizontally adjacent pixels per CTA.
//
// Pixels A = (y, x) and B = (y, x+1) search windows that share all but one column each: the
// patch a_j of a shared window position is one and the same vector for both problems.  One CTA
// of 256 threads keeps both problems' ADMM state for every shared point in the same lane, so
// each point quad read from shared memory serves the update of both problems (half the
// shared-memory traffic of one problem per CTA), and one set of CTA barriers per iteration
// serves both problems (twice the work between synchronisations).
//
// Per-point algebra (Algorithm 1 in the reformulation used by the one-problem solver, FP32):
//   e = c + h,  s = min(1, lam / ||e||),  sum_g += s e,  h = s e - a,
// with c = 2 z(t) - z(t-1) per problem and h_k = g_k - a_k started at -a_k.
//
// Layout.  G = 4 lanes share a point slot; lane g owns coordinates [12 g, 12 g + 12) of both
// problems, and the slice-3 lane also owns coordinate 48 (the "tail").  A lane holds P = 7
// slots j = pg + p * 64 (pg = its group).  Slot j holds a window position of A and one of B:
//   - shared positions: the same point for both problems;
//   - the exclusive pair of a window row r (A's leftmost column, B's rightmost column): slot
//     EX0 + r (point index P-1 of group r), whose B point sits in a row array of its own.
// State per slot: hA[6], hB[6] (coordinate pairs, packed FP32) and hT = (hA_48, hB_48).
// Point rows are 52 floats (49 coordinates in order, 3 zeros; 52/4 odd keeps 16-byte loads of
// 8 consecutive rows conflict-free).
//
// The d-vector sums: during the update each lane reduces its 32 partial sums across the 8
// lanes of its slice with shuffles (reduce-scatter), leaving one float4 column per lane; the
// 8 warps' columns are summed by warp 0 after one CTA barrier.  Column c of slice g:
//   c = 0..2  A coordinates 12g + 4c .. +3        c = 4..6  B coordinates 12g + 4(c-4) .. +3
//   c = 3     (A tail sum, A ||dh||^2, A ||g||^2)  c = 7     (B tail sum, B ||dh||^2, B ||g||^2)
// z, c = 2z - z_prev, sum g and the centre patches are kept in the same column layout, each
// slice padded to 9 float4 so that the broadcast loads of the 4 slices hit different banks.
// Warp 0 forms z+ and c+ branch-free and publishes the next iteration's check flag.
//
// The step s of the 14 (point, problem) pairs of a point group: the partial norms are
// reduce-scattered over the group's 4 lanes, each lane turns its own full norms into s (4 rsqrt
// instead of 14), and the s values are gathered back.  The tail coordinate is updated as a
// fourth point quad in the prefetched update loop.
//
// Each problem stops at its own residual check (or the cap): its z is frozen from then on and
// the CTA runs until both are frozen, so the result of each pixel is the iterate at which its
// own stopping rule fired, as for one pixel per CTA.
#include <cuda_runtime.h>
#include <math.h>

#include "debug.h"
#include "kernels.h"
#include "solver_common.cuh"

namespace nlemk {
namespace pairk {

constexpr int K = 7, D = 49, HK = 3;
constexpr int G = 4, QM = 12, NQ = 3;          // slices per point, main slots and quads per slice
constexpr int P = 7, NW = 8, NT = NW * 32;     // slots per lane, warps, threads
constexpr int NG = NT / G, CAP = NG * P;       // 64 point groups, 448 slots
constexpr int DP = 52;                         // point row stride (floats)
constexpr int EX0 = (P - 1) * NG;              // slot of the first exclusive pair
constexpr int RMAX = 21;                       // window rows (window <= 21)
constexpr int NCOL = 32;                       // columns: 4 slices x 8
constexpr int VQ = 9;                          // float4 per slice in the vector layout: 8 columns
                                               // and a pad, so the slices sit in different banks
constexpr int VEC = G * VQ * 4;                // floats per vector (z, c, sum g, centre patches)
constexpr int TILE_MAX = 1024;                 // tile floats ((21 + 6) x (22 + 6) = 756)

constexpr int OFF_PTS = 0;
constexpr int OFF_PTSB = OFF_PTS + CAP * DP;
constexpr int OFF_LAM = OFF_PTSB + RMAX * DP;  // float2 (lam_A, lam_B) per slot, at lam_at(j)
constexpr int SZ_LAM = 2 * (CAP + 2 * P);
constexpr int OFF_FLAG = OFF_LAM + SZ_LAM;     // int per slot: bit 0 A's point, bit 1 B's point
constexpr int OFF_ZV = OFF_FLAG + CAP;
constexpr int OFF_CV = OFF_ZV + VEC;
constexpr int OFF_SGV = OFF_CV + VEC;
constexpr int OFF_PCV = OFF_SGV + VEC;
constexpr int OFF_CRED = OFF_PCV + VEC;        // float4 [NW][NCOL]
constexpr int OFF_TILE = OFF_CRED + 4 * NW * NCOL;   // the tile (setup), FP64 scratch (check)
constexpr int OFF_SCAL = OFF_TILE + TILE_MAX;
constexpr int TOTAL = OFF_SCAL + 32;
constexpr size_t SMEM_BYTES = (size_t)TOTAL * 4;
static_assert(OFF_PTSB % 4 == 0 && OFF_LAM % 4 == 0 && OFF_ZV % 4 == 0 && OFF_CRED % 4 == 0 &&
                  OFF_TILE % 2 == 0,
              "16-byte aligned regions (8-byte for the FP64 scratch)");
static_assert(2 * TILE_MAX >= 4 * (CAP + 64), "FP64 scratch: CAP coefficients + the d-vector");
static_assert(EX0 + RMAX <= CAP && RMAX <= NG, "exclusive slots sit at point index P-1");
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");

// scal: [0] A frozen, [1] B frozen, [2] A iterations, [3] A residual, [4] B iterations,
// [5] B residual; as int: [6] the next iteration checks the residuals, [7] iterations to the
// next periodic check
struct Sm {
  float* pts;
  float* ptsB;
  float2* lam;
  int* flag;
  float* zv;
  float* cv;
  float* sgv;
  float* pcv;
  float4* cred;
  float* tile;
  float* scal;
  __device__ __forceinline__ explicit Sm(float* b)
      : pts(b + OFF_PTS), ptsB(b + OFF_PTSB), lam(reinterpret_cast<float2*>(b + OFF_LAM)),
        flag(reinterpret_cast<int*>(b + OFF_FLAG)), zv(b + OFF_ZV), cv(b + OFF_CV), sgv(b + OFF_SGV),
        pcv(b + OFF_PCV), cred(reinterpret_cast<float4*>(b + OFF_CRED)), tile(b + OFF_TILE), scal(b + OFF_SCAL) {}
};

// float2 index of slot j's (lam_A, lam_B): each block of NG slots (one point index p) is shifted
// by 2 float2, so that the s step's loads of points p and p + 4 fall in different banks
__host__ __device__ __forceinline__ int lam_at(int j) { return j + 2 * (j / NG); }

// index of coordinate q (0..48) of problem X (0 = A, 1 = B) in the column layout
__host__ __device__ __forceinline__ int vidx(int q, int X) {
  if (q < 4 * G * NQ) {
    const int g = q / QM, i = q - g * QM;
    return (g * VQ + 4 * X + i / 4) * 4 + (i % 4);
  }
  return ((G - 1) * VQ + 4 * X + 3) * 4;
}
// float4 index of column col (= slice * 8 + c) in the vector layout
__host__ __device__ __forceinline__ int vcol(int col) { return (col >> 3) * VQ + (col & 7); }

// The check schedule of the stopping rule: iteration `it` evaluates the residuals when it is
// the cap or, with a tolerance, every check_every-th iteration.  One thread keeps a countdown
// in shared memory and publishes the flag of iteration next_it, so the others read a flag
// instead of each computing a remainder.
__device__ __forceinline__ void schedule_check(float* scal, int next_it, const SolveParams& prm) {
  int* si = reinterpret_cast<int*>(scal);
  const int cnt = si[7];
  const bool periodic = cnt == 1;
  si[7] = periodic ? prm.check_every : cnt - 1;
  si[6] = (next_it == prm.iters || (prm.tol > 0.f && periodic)) ? 1 : 0;
}

__device__ __forceinline__ int lane_g() { return (threadIdx.x & 31) >> 3; }
__device__ __forceinline__ int lane_pg() { return (threadIdx.x >> 5) * 8 + (threadIdx.x & 7); }
// sum over the 4 lanes of a point group (8 lanes apart)
__device__ __forceinline__ float gsum(float v) {
  v += __shfl_xor_sync(kFull, v, 8);
  v += __shfl_xor_sync(kFull, v, 16);
  return v;
}
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float4 sel4(bool c, float4 a, float4 b) {
  return make_float4(c ? a.x : b.x, c ? a.y : b.y, c ? a.z : b.z, c ? a.w : b.w);
}
__device__ __forceinline__ float4 shfl4(float4 v, int o) {
  return make_float4(__shfl_xor_sync(kFull, v.x, o), __shfl_xor_sync(kFull, v.y, o),
                     __shfl_xor_sync(kFull, v.z, o), __shfl_xor_sync(kFull, v.w, o));
}
// one step of the reduce-scatter across the lanes of a slice: the lane whose bit `o` is set
// keeps `hi`, its partner keeps `lo`; each returns the pair-sum of the half it keeps
__device__ __forceinline__ float4 rs_step(float4 lo, float4 hi, int o) {
  const bool up = (threadIdx.x & o) != 0;
  const float4 keep = sel4(up, hi, lo), send = sel4(up, lo, hi);
  return f4add(keep, shfl4(send, o));
}

// The B-side row of slot j of this lane's point index p: the exclusive row for the pairs at
// point index P-1, else the slot's own row.
__device__ __forceinline__ const float* brow_of(const Sm& sm, const float* arow, int p, int pg, int nex) {
  return (p == P - 1 && pg < nex) ? sm.ptsB + pg * DP + lane_g() * QM : arow;
}


// Algorithm 1 for both problems from the state the caller set up: point rows (inactive slots
// zero), lam (zero where a problem has no point), zv = cv = z(0) and sgv = 0 per problem, and
// scal[0..1] the initial frozen flags (a missing B starts frozen).  On return zv holds each
// problem's iterate at which its stopping rule fired; scal[2..5] its iterations and residual.
__device__ void pair_iterate(const Sm& sm, int nA, int nB, int nex, const SolveParams& prm) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane_g(), pg = lane_pg();
  const bool tl = (g == G - 1);   // the lane that owns coordinate 48
  const float invnA = nA > 0 ? 1.f / (float)nA : 0.f, invnB = nB > 0 ? 1.f / (float)nB : 0.f;
  const float fnA = (float)nA, fnB = (float)nB;

  float2 hA[P][2 * NQ], hB[P][2 * NQ], hT[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const float* arow = sm.pts + (pg + p * NG) * DP + g * QM;
    const float* brow = brow_of(sm, arow, p, pg, nex);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float4 a4 = reinterpret_cast<const float4*>(arow)[q];
      const float4 b4 = reinterpret_cast<const float4*>(brow)[q];
      hA[p][2 * q] = f2(a4.x, a4.y);
      hA[p][2 * q + 1] = f2(a4.z, a4.w);
      hB[p][2 * q] = f2(b4.x, b4.y);
      hB[p][2 * q + 1] = f2(b4.z, b4.w);
    }
    hT[p] = tl ? f2(arow[QM], brow[QM]) : f2(0.f, 0.f);
  }

  for (int it = 1; it <= prm.iters; ++it) {
    const bool check = reinterpret_cast<const int*>(sm.scal)[6] != 0;
    const float4* cv4 = reinterpret_cast<const float4*>(sm.cv) + g * VQ;
    // phase 1: e = c + h in place and the squared norms, one problem at a time
    float nA[P], nB[P];
    {
      float2 acc[P];
#pragma unroll
      for (int p = 0; p < P; ++p) acc[p] = f2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const float4 c4 = cv4[q];
        const float2 c01 = f2(c4.x, c4.y), c23 = f2(c4.z, c4.w);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          hA[p][2 * q] = __fadd2_rn(hA[p][2 * q], c01);
          acc[p] = __ffma2_rn(hA[p][2 * q], hA[p][2 * q], acc[p]);
          hA[p][2 * q + 1] = __fadd2_rn(hA[p][2 * q + 1], c23);
          acc[p] = __ffma2_rn(hA[p][2 * q + 1], hA[p][2 * q + 1], acc[p]);
        }
      }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        nA[p] = acc[p].x + acc[p].y;
        acc[p] = f2(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const float4 c4 = cv4[4 + q];
        const float2 c01 = f2(c4.x, c4.y), c23 = f2(c4.z, c4.w);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          hB[p][2 * q] = __fadd2_rn(hB[p][2 * q], c01);
          acc[p] = __ffma2_rn(hB[p][2 * q], hB[p][2 * q], acc[p]);
          hB[p][2 * q + 1] = __fadd2_rn(hB[p][2 * q + 1], c23);
          acc[p] = __ffma2_rn(hB[p][2 * q + 1], hB[p][2 * q + 1], acc[p]);
        }
      }
#pragma unroll
      for (int p = 0; p < P; ++p) nB[p] = acc[p].x + acc[p].y;
      const float2 cT = tl ? f2(sm.cv[vidx(48, 0)], sm.cv[vidx(48, 1)]) : f2(0.f, 0.f);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        hT[p] = __fadd2_rn(hT[p], cT);
        const float2 sq = __fmul2_rn(hT[p], hT[p]);
        nA[p] += sq.x;
        nB[p] += sq.y;
      }
    }
    // s = min(1, lam / ||e||) for the 14 (point, problem) pairs of the group.  The partial norms
    // are reduce-scattered over the group's 4 lanes (8 apart): after the xor-16 step the lanes
    // with bit 4 clear hold A's norms, the others B's; after the xor-8 step bit 3 picks points
    // 0..3 or 4..6.  Each lane turns its own full norms into s (4 rsqrt instead of 14), and the
    // s values are gathered back.  r2 = 0 gives s = 1 through fminf, harmless since e = 0 there.
    float sA[P], sB[P];
    float gsA = 0.f, gsB = 0.f;   // sum of ||g||^2 over the pairs this lane owns
    {
      const bool b16 = (lane & 16) != 0, b8 = (lane & 8) != 0;
      float v7[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float keep = b16 ? nB[p] : nA[p], send = b16 ? nA[p] : nB[p];
        v7[p] = keep + __shfl_xor_sync(kFull, send, 16);
      }
      constexpr int PH = (P + 1) / 2;   // 4: points per half
      float s4[PH];
      float gsX = 0.f;
      const float* lamf = reinterpret_cast<const float*>(sm.lam) + (b16 ? 1 : 0);
#pragma unroll
      for (int i = 0; i < PH; ++i) {
        const float lo = v7[i], hi = PH + i < P ? v7[PH + i] : 0.f;
        const float keep = b8 ? hi : lo, send = b8 ? lo : hi;
        const float r2 = keep + __shfl_xor_sync(kFull, send, 8);
        const int p = (b8 ? PH : 0) + i;
        const bool valid = p < P;
        const float l = valid ? lamf[2 * lam_at(pg + p * NG)] : 0.f;
        s4[i] = valid ? fminf(1.f, l * rsqrtf(r2)) : 0.f;
        gsX = fmaf(s4[i] * s4[i], valid ? r2 : 0.f, gsX);
      }
      float s7[P];
#pragma unroll
      for (int i = 0; i < PH; ++i) {
        const float other = __shfl_xor_sync(kFull, s4[i], 8);
        s7[i] = b8 ? other : s4[i];
        if (PH + i < P) s7[PH + i] = b8 ? s4[i] : other;
      }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float other = __shfl_xor_sync(kFull, s7[p], 16);
        sA[p] = b16 ? other : s7[p];
        sB[p] = b16 ? s7[p] : other;
      }
      gsA = b16 ? 0.f : gsX;
      gsB = b16 ? gsX : 0.f;
    }
    // residual pass (check iterations): ||h(t) - h(t+1)||^2 = ||(1-s) e + a - c||^2
    float ddA = 0.f, ddB = 0.f;
    if (check) {
      asm volatile("" ::: "memory");
      const float2 cT = tl ? f2(sm.cv[vidx(48, 0)], sm.cv[vidx(48, 1)]) : f2(0.f, 0.f);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float* arow = sm.pts + (pg + p * NG) * DP + g * QM;
        const float* brow = brow_of(sm, arow, p, pg, nex);
        const float oA = 1.f - sA[p], oB = 1.f - sB[p];
        const float2 oA2 = f2(oA, oA), oB2 = f2(oB, oB);
        float2 dA2 = f2(0.f, 0.f), dB2 = f2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const float4 a4 = reinterpret_cast<const float4*>(arow)[q];
          const float4 b4 = reinterpret_cast<const float4*>(brow)[q];
          const float4 cA = cv4[q], cB = cv4[4 + q];
          float2 x = __ffma2_rn(oA2, hA[p][2 * q], f2(-a4.x - cA.x, -a4.y - cA.y));
          dA2 = __ffma2_rn(x, x, dA2);
          x = __ffma2_rn(oA2, hA[p][2 * q + 1], f2(-a4.z - cA.z, -a4.w - cA.w));
          dA2 = __ffma2_rn(x, x, dA2);
          x = __ffma2_rn(oB2, hB[p][2 * q], f2(-b4.x - cB.x, -b4.y - cB.y));
          dB2 = __ffma2_rn(x, x, dB2);
          x = __ffma2_rn(oB2, hB[p][2 * q + 1], f2(-b4.z - cB.z, -b4.w - cB.w));
          dB2 = __ffma2_rn(x, x, dB2);
        }
        const float2 tv = tl ? f2(-arow[QM], -brow[QM]) : f2(0.f, 0.f);
        const float2 x = __ffma2_rn(f2(oA, oB), hT[p], f2(tv.x - cT.x, tv.y - cT.y));
        ddA += dA2.x + dA2.y + x.x * x.x;
        ddB += dB2.x + dB2.y + x.y * x.y;
        asm volatile("" ::: "memory");
      }
    }
    // phase 2: sum g and h = s e - a, quad by quad; each quad's A and B sums go straight into
    // the first reduce-scatter step (A columns to the lanes with bit 2 clear, B to the others)
    float4 u[4];
    {
      const float* abase = sm.pts + pg * DP + g * QM;
      float4 a_n1 = reinterpret_cast<const float4*>(abase)[0];
      float4 a_n2 = reinterpret_cast<const float4*>(abase + NG * DP)[0];
      float4 a_n3 = reinterpret_cast<const float4*>(abase + 2 * NG * DP)[0];
      float2 aT = f2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q <= NQ; ++q) {   // q = NQ: the tail quad (coordinate 48 and three zeros)
        float2 aA0 = f2(0.f, 0.f), aA1 = aA0, aB0 = aA0, aB1 = aA0;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const float4 a4 = a_n1;
          a_n1 = a_n2;
          a_n2 = a_n3;
          {
            const int lin = q * P + p + 3;   // the quad three steps ahead
            const int nq = lin / P, np = lin % P;
            if (nq < NQ) a_n3 = reinterpret_cast<const float4*>(abase + np * NG * DP)[nq];
            else if (nq == NQ) a_n3 = tl ? reinterpret_cast<const float4*>(abase + np * NG * DP)[nq]
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          float4 b4 = a4;
          if (p == P - 1 && pg < nex && (q < NQ || tl))
            b4 = reinterpret_cast<const float4*>(sm.ptsB + pg * DP + g * QM)[q];
          if (q == NQ) {
            const float2 sT = f2(sA[p], sB[p]);
            aT = __ffma2_rn(sT, hT[p], aT);
            hT[p] = __ffma2_rn(sT, hT[p], f2(a4.x, b4.x));
            continue;
          }
          const float2 sA2 = f2(sA[p], sA[p]), sB2 = f2(sB[p], sB[p]);
          aA0 = __ffma2_rn(sA2, hA[p][2 * q], aA0);
          hA[p][2 * q] = __ffma2_rn(sA2, hA[p][2 * q], f2(a4.x, a4.y));
          aA1 = __ffma2_rn(sA2, hA[p][2 * q + 1], aA1);
          hA[p][2 * q + 1] = __ffma2_rn(sA2, hA[p][2 * q + 1], f2(a4.z, a4.w));
          aB0 = __ffma2_rn(sB2, hB[p][2 * q], aB0);
          hB[p][2 * q] = __ffma2_rn(sB2, hB[p][2 * q], f2(b4.x, b4.y));
          aB1 = __ffma2_rn(sB2, hB[p][2 * q + 1], aB1);
          hB[p][2 * q + 1] = __ffma2_rn(sB2, hB[p][2 * q + 1], f2(b4.z, b4.w));
        }
        if (q < NQ)
          u[q] = rs_step(make_float4(aA0.x, aA0.y, aA1.x, aA1.y), make_float4(aB0.x, aB0.y, aB1.x, aB1.y), 4);
      }
      u[3] = rs_step(make_float4(aT.x, ddA, gsA, 0.f), make_float4(aT.y, ddB, gsB, 0.f), 4);
    }
    {
      const float4 v0 = rs_step(u[0], u[2], 2), v1 = rs_step(u[1], u[3], 2);
      sm.cred[warp * NCOL + lane] = rs_step(v0, v1, 1);   // column lane: slice lane/8, c = lane%8
    }
    __syncthreads();
    // finalize (warp 0, lane = column): z+ = P_C(z - sum g / n), c+ = 2 z+ - z, residuals
    if (warp == 0) {
      float4 tot = sm.cred[lane], tb = sm.cred[NCOL + lane];
#pragma unroll
      for (int w = 2; w < NW; w += 2) {
        tot = f4add(tot, sm.cred[w * NCOL + lane]);
        tb = f4add(tb, sm.cred[(w + 1) * NCOL + lane]);
      }
      tot = f4add(tot, tb);
      const int c = lane & 7, X = c >> 2, cc = c & 3;
      const bool frozen = sm.scal[X] != 0.f;
      if (lane == 0) schedule_check(sm.scal, it + 1, prm);
      const float invn = X ? invnB : invnA, fn = X ? fnB : fnA;
      const int nreal = cc < 3 ? 4 : ((lane >> 3) == G - 1 ? 1 : 0);
      float4* zv4 = reinterpret_cast<float4*>(sm.zv);
      float4* cvw = reinterpret_cast<float4*>(sm.cv);
      float4* sgv4 = reinterpret_cast<float4*>(sm.sgv);
      const int vc = vcol(lane);
      const float4 z4 = zv4[vc];
      float4 c4o = make_float4(0.f, 0.f, 0.f, 0.f), s4o = c4o;
      if (check) {
        c4o = cvw[vc];
        s4o = sgv4[vc];
      }
      float p_dd = 0.f, p_dS = 0.f, p_zz = 0.f, p_zx = 0.f, p_dz = 0.f, p_dzA = 0.f, p_E = 0.f, p_G = 0.f;
      float zn[4], cn[4], sn[4];
      // branch-free: slots that hold no coordinate (z = c = sum g = 0 there) are masked to zero
      // by selects, which keeps the lane-dependent slot count from splitting the warp
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool real = i < nreal;
        const float A = real ? f4get(tot, i) : 0.f, z = f4get(z4, i);
        const float zc = frozen ? z : clampf(fmaf(-A, invn, z), prm.lo, prm.hi);
        const float znew = real ? zc : 0.f;
        if (check) {
          const float del = f4get(c4o, i) - znew;   // c(t) - z(t+1)
          const float SD = f4get(s4o, i) - A;       // sum_k (g_k(t) - g_k(t+1))
          const float dz = z - znew;
          p_dd = fmaf(del, del, p_dd);
          p_dS = fmaf(del, SD, p_dS);
          p_zz = fmaf(znew, znew, p_zz);
          p_zx = fmaf(znew, fmaf(fn, del, SD), p_zx);
          p_dz = fmaf(dz, dz, p_dz);
          p_dzA = fmaf(dz, A, p_dzA);
        }
        zn[i] = znew;
        cn[i] = real ? (frozen ? z : 2.f * znew - z) : 0.f;
        sn[i] = A;
      }
      if (cc == 3) {
        p_E = tot.y;
        p_G = tot.z;
      }
      zv4[vc] = make_float4(zn[0], zn[1], zn[2], zn[3]);
      cvw[vc] = make_float4(cn[0], cn[1], cn[2], cn[3]);
      sgv4[vc] = make_float4(sn[0], sn[1], sn[2], sn[3]);
      if (check) {
        // sums over the 16 lanes of the same problem (lane bit 2 = X)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          if (o == 4) continue;
          p_dd += __shfl_xor_sync(kFull, p_dd, o);
          p_dS += __shfl_xor_sync(kFull, p_dS, o);
          p_zz += __shfl_xor_sync(kFull, p_zz, o);
          p_zx += __shfl_xor_sync(kFull, p_zx, o);
          p_dz += __shfl_xor_sync(kFull, p_dz, o);
          p_dzA += __shfl_xor_sync(kFull, p_dzA, o);
          p_E += __shfl_xor_sync(kFull, p_E, o);
          p_G += __shfl_xor_sync(kFull, p_G, o);
        }
        if ((lane & ~4) == 0 && !frozen) {
          const float spr = fmaxf(fn * p_dd + 2.f * p_dS + p_E, 0.f);
          const float sx = fmaxf(spr + 2.f * p_zx + fn * p_zz, 0.f);
          const float su = fmaxf(fn * p_dz - 2.f * p_dzA + p_G, 0.f);
          const float den_p = fmaxf(fmaxf(sqrtf(sx), sqrtf(fn * p_zz)), 1e-30f);
          const float den_d = fmaxf(sqrtf(su), 1e-30f);
          const float rp = sqrtf(spr) / den_p, rd = sqrtf(fn * p_dz) / den_d;
          const bool conv = prm.tol > 0.f && rp < prm.tol && rd < prm.tol;
          if (conv || it == prm.iters) {
            sm.scal[X] = 1.f;
            sm.scal[2 + 2 * X] = (float)it;
            sm.scal[3 + 2 * X] = fmaxf(rp, rd);
          }
        }
      }
    }
    __syncthreads();
    if (check && sm.scal[0] != 0.f && sm.scal[1] != 0.f) break;
  }
  __syncthreads();
}

// FP64 objective of problem (1) and projected-gradient optimality residual of problem X at its
// z (zv), with the weights exp(-||P_X - P_j||^2 / h^2) recomputed in double.  Same formulas as
// fp64_check in admm_core.cuh; the tile region is the scratch.
__device__ void pair_fp64(const Sm& sm, int X, int nex, const SolveParams& prm, double ih2, double& F, double& R) {
  const int t = threadIdx.x;
  double* coef = reinterpret_cast<double*>(sm.tile);
  double* gvec = coef + CAP;
  __shared__ double s_F[NW], s_wb[NW], s_ws[NW], s_g2[NW];
  __shared__ double s_R, s_Fo;
  const double tau = 1e-9 * fmax(1.0, (double)prm.hi - (double)prm.lo);
  auto row_of = [&](int j) -> const float* {
    return (X == 1 && j >= EX0 && j < EX0 + nex) ? sm.ptsB + (j - EX0) * DP : sm.pts + j * DP;
  };
  double f = 0.0, wb = 0.0, ws = 0.0;
  for (int j = t; j < CAP; j += NT) {
    if (!((sm.flag[j] >> X) & 1)) {
      coef[j] = 0.0;
      continue;
    }
    const float* row = row_of(j);
    double r2 = 0.0, dw = 0.0;
    for (int q = 0; q < D; ++q) {
      const double a = -(double)row[q];
      const double e = (double)sm.zv[vidx(q, X)] - a;
      const double u = (double)sm.pcv[vidx(q, X)] - a;
      r2 += e * e;
      dw += u * u;
    }
    const double r = sqrt(r2), w = exp(-dw * ih2);
    f += w * r;
    ws += w;
    if (r <= tau) {
      wb += w;
      coef[j] = 0.0;
    } else {
      coef[j] = w / r;
    }
  }
  __syncthreads();
  double g2 = 0.0;
  for (int q = t; q < D; q += NT) {
    const double z = (double)sm.zv[vidx(q, X)];
    double gq = 0.0;
    for (int j = 0; j < CAP; ++j)
      if (coef[j] != 0.0) gq += coef[j] * (z + (double)row_of(j)[q]);
    gvec[q] = gq;
    g2 += gq * gq;
  }
  for (int o = 16; o > 0; o >>= 1) {
    f += __shfl_xor_sync(kFull, f, o);
    wb += __shfl_xor_sync(kFull, wb, o);
    ws += __shfl_xor_sync(kFull, ws, o);
    g2 += __shfl_xor_sync(kFull, g2, o);
  }
  if ((t & 31) == 0) {
    s_F[t >> 5] = f;
    s_wb[t >> 5] = wb;
    s_ws[t >> 5] = ws;
    s_g2[t >> 5] = g2;
  }
  __syncthreads();
  if (t == 0) {
    double FF = 0, WB = 0, WS = 0, G2 = 0;
    for (int w = 0; w < NW; ++w) {
      FF += s_F[w];
      WB += s_wb[w];
      WS += s_ws[w];
      G2 += s_g2[w];
    }
    const double gn = sqrt(G2);
    const double scale = gn > 0.0 ? fmax(gn - WB, 0.0) / gn : 0.0;
    double RR = 0.0;
    if (WS > 0.0) {
      for (int q = 0; q < D; ++q) {
        const double z = (double)sm.zv[vidx(q, X)];
        double tq = z - scale * gvec[q] / WS;
        tq = fmin(fmax(tq, (double)prm.lo), (double)prm.hi);
        RR += (z - tq) * (z - tq);
      }
    }
    s_R = sqrt(RR);
    s_Fo = FF;
  }
  __syncthreads();
  F = s_Fo;
  R = s_R;
}

__device__ __forceinline__ int reflect(int x, int N) { return x < 0 ? -x : (x >= N ? 2 * N - 2 - x : x); }

// One pixel pair: tile of the reflect-padded image around the union of the two clipped search
// windows -> point rows -> weights of both problems -> start points -> Algorithm 1 -> the
// centre coordinates.  EX: the caller's per-pixel start points, penalties and solution patches
// (ex) are taken; the plain instance compiles without them.  Ends with a barrier.
template <bool EX>
__device__ void pair_pixel(const Sm& sm, const float* __restrict__ img, int H, int W, int pitch, int S,
                           float inv_h2, double ih2, const SolveParams& prm, int init_mode, long long item,
                           float* __restrict__ out, int* __restrict__ iters_used, float* __restrict__ resid,
                           double* __restrict__ obj64, double* __restrict__ kkt64, const PixelExtra& ex) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane_g(), pg = lane_pg();
  const bool tl = (g == G - 1);
  const int WP = (W + 1) / 2, R = (S - 1) / 2;
  const int y = (int)(item / WP), x = 2 * (int)(item - (long long)y * WP);
  const bool hasB = x + 1 < W;
  const int r0 = max(y - R, 0), r1 = min(y + R, H - 1), nwr = r1 - r0 + 1;
  const int a0 = max(x - R, 0), a1 = min(x + R, W - 1);
  const int b0 = hasB ? max(x + 1 - R, 0) : a0, b1 = hasB ? min(x + 1 + R, W - 1) : a1;
  const bool exA = b0 > a0, exB = b1 > a1;        // one exclusive column each at most
  const int nex = (exA || exB) ? nwr : 0;
  const int nsc = a1 - b0 + 1, nsh = nwr * nsc;   // shared columns and positions
  const int nA = nwr * (a1 - a0 + 1), nB = hasB ? nwr * (b1 - b0 + 1) : 0;
  const int TC = (b1 - a0 + 1) + 2 * HK, TR = nwr + 2 * HK;
  for (int tr = warp; tr < TR; tr += NW) {
    const long long gr = (long long)reflect(r0 - HK + tr, H) * pitch;
    for (int tc = lane; tc < TC; tc += 32) {
      const long long gi = gr + reflect(a0 - HK + tc, W);
      const float v = NLEM_DBG_OK(gi, (long long)H * pitch, kDbgImageRead) ? __ldg(img + gi) : 0.f;
      if (NLEM_DBG_OK(tr * TC + tc, TILE_MAX, kDbgPairTile)) sm.tile[tr * TC + tc] = v;
    }
  }
  if (t == 0) {
    sm.scal[0] = 0.f;
    sm.scal[1] = hasB ? 0.f : 1.f;
    for (int i = 2; i < 6; ++i) sm.scal[i] = 0.f;
    reinterpret_cast<int*>(sm.scal)[7] = prm.check_every;
    schedule_check(sm.scal, 1, prm);
  }
  __syncthreads();
  // point rows: shared positions fill the slots in row-major order, skipping the exclusive
  // slots EX0 .. EX0 + nex - 1 (A's column a0 and, in ptsB, B's column b1 of window row r)
  for (int jj = t; jj < CAP + RMAX; jj += NT) {
    int r = 0, u = -1;
    float* dst;
    if (jj < CAP) {
      const int j = jj;
      int fl = 0;
      dst = sm.pts + j * DP;
      if (j >= EX0 && j < EX0 + nex) {
        r = j - EX0;
        if (exA) u = a0;
        fl = (exA ? 1 : 0) | (exB ? 2 : 0);
      } else {
        const int m = j < EX0 ? j : j - nex;
        if (m < nsh) {
          r = m / nsc;
          u = b0 + (m - r * nsc);
          fl = 1 | (hasB ? 2 : 0);
        }
      }
      sm.flag[j] = fl;
    } else {
      r = jj - CAP;
      dst = sm.ptsB + r * DP;
      if (r < nex && exB) u = b1;
    }
    float4* row4 = reinterpret_cast<float4*>(dst);
    const float* tp = sm.tile + r * TC + (u - a0);
#pragma unroll
    for (int i4 = 0; i4 < DP / 4; ++i4) {
      float v[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int q = 4 * i4 + c;
        const int ti = r * TC + (u - a0) + (q / K) * TC + (q % K);
        v[c] = (u >= 0 && q < D && NLEM_DBG_OK(ti, TR * TC, kDbgPairTile)) ? -tp[(q / K) * TC + (q % K)] : 0.f;
      }
      if (NLEM_DBG_OK(dst - sm.pts + 4 * i4 + 3, OFF_LAM - OFF_PTS, kDbgPairRow))
        row4[i4] = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
  // centre patches in the column layout (slots that hold no coordinate are zero)
  for (int i = t; i < 4 * NCOL; i += NT) {
    const int col = i >> 2, slot = i & 3, sg = col >> 3, c = col & 7, X = c >> 2, cc = c & 3;
    const int q = cc < 3 ? sg * QM + 4 * cc + slot : ((sg == G - 1 && slot == 0) ? 4 * G * NQ : -1);
    float v = 0.f;
    const int ti = (y - r0 + q / K) * TC + (x + X - a0 + q % K);
    if (q >= 0 && (X == 0 || hasB) && NLEM_DBG_OK(ti, TR * TC, kDbgPairTile)) v = sm.tile[ti];
    sm.pcv[vcol(col) * 4 + slot] = v;
  }
  __syncthreads();
  // each pixel's penalty: the caller's per-pixel one, else the launch's
  const long long pix0 = (long long)y * W + x;
  const float imuA = (EX && ex.rho) ? 1.f / __ldg(ex.rho + pix0) : prm.inv_mu;
  const float imuB = (EX && ex.rho && hasB) ? 1.f / __ldg(ex.rho + pix0 + 1) : prm.inv_mu;
  // weights w_j = exp(-||P_X - P_j||^2 / h^2) of both problems (zero where X has no point j)
  float wA[P], wB[P];
  {
    const float4* pc4 = reinterpret_cast<const float4*>(sm.pcv) + g * VQ;
    const float2 pT = tl ? f2(sm.pcv[vidx(48, 0)], sm.pcv[vidx(48, 1)]) : f2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int j = pg + p * NG;
      const float* arow = sm.pts + j * DP + g * QM;
      const float* brow = brow_of(sm, arow, p, pg, nex);
      float dA = 0.f, dB = 0.f;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const float4 a4 = reinterpret_cast<const float4*>(arow)[q];
        const float4 b4 = reinterpret_cast<const float4*>(brow)[q];
        const float4 pa = pc4[q], pb = pc4[4 + q];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float ea = f4get(pa, c) + f4get(a4, c), eb = f4get(pb, c) + f4get(b4, c);
          dA = fmaf(ea, ea, dA);
          dB = fmaf(eb, eb, dB);
        }
      }
      if (tl) {
        const float ea = pT.x + arow[QM], eb = pT.y + brow[QM];
        dA = fmaf(ea, ea, dA);
        dB = fmaf(eb, eb, dB);
      }
      dA = gsum(dA);
      dB = gsum(dB);
      const int fl = sm.flag[j];
      wA[p] = (fl & 1) ? expf(-dA * inv_h2) : 0.f;
      wB[p] = (fl & 2) ? expf(-dB * inv_h2) : 0.f;
      if (g == 0) sm.lam[lam_at(j)] = f2(wA[p] * imuA, wB[p] * imuB);
    }
  }
  float4* zv4 = reinterpret_cast<float4*>(sm.zv);
  float4* cvw = reinterpret_cast<float4*>(sm.cv);
  float4* sgv4 = reinterpret_cast<float4*>(sm.sgv);
  if (EX && ex.x0) {   // the caller's start points of both pixels, projected onto C
    if (t < NCOL) {
      const int sg = t >> 3, c = t & 7, X = c >> 2, cc = c & 3;
      const long long pixX = (long long)y * W + x + X;
      float zz[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int q = cc < 3 ? sg * QM + 4 * cc + i : ((sg == G - 1 && i == 0) ? 4 * G * NQ : -1);
        zz[i] = (q >= 0 && (X == 0 || hasB)) ? clampf(__ldg(ex.x0 + pixX * D + q), prm.lo, prm.hi) : 0.f;
      }
      zv4[vcol(t)] = cvw[vcol(t)] = make_float4(zz[0], zz[1], zz[2], zz[3]);
      sgv4[vcol(t)] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
  } else if (init_mode == 1) {   // the noisy patches, projected onto C
    if (t < NCOL) {
      const float4 pc = reinterpret_cast<const float4*>(sm.pcv)[vcol(t)];
      const int cc = t & 3, nreal = cc < 3 ? 4 : ((t >> 3) == G - 1 ? 1 : 0);
      float zz[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) zz[i] = i < nreal ? clampf(f4get(pc, i), prm.lo, prm.hi) : 0.f;
      zv4[vcol(t)] = cvw[vcol(t)] = make_float4(zz[0], zz[1], zz[2], zz[3]);
      sgv4[vcol(t)] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
  } else {   // P_C(weighted mean) of each problem (sum w >= 1: the centre point weighs 1)
    float4 u[4];
    {
      float4 accA[NQ], accB[NQ];
      float2 accT = f2(0.f, 0.f);
      float swA = 0.f, swB = 0.f;
#pragma unroll
      for (int q = 0; q < NQ; ++q) accA[q] = accB[q] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float* arow = sm.pts + (pg + p * NG) * DP + g * QM;
        const float* brow = brow_of(sm, arow, p, pg, nex);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const float4 a4 = reinterpret_cast<const float4*>(arow)[q];
          const float4 b4 = reinterpret_cast<const float4*>(brow)[q];
          accA[q] = make_float4(fmaf(-wA[p], a4.x, accA[q].x), fmaf(-wA[p], a4.y, accA[q].y),
                                fmaf(-wA[p], a4.z, accA[q].z), fmaf(-wA[p], a4.w, accA[q].w));
          accB[q] = make_float4(fmaf(-wB[p], b4.x, accB[q].x), fmaf(-wB[p], b4.y, accB[q].y),
                                fmaf(-wB[p], b4.z, accB[q].z), fmaf(-wB[p], b4.w, accB[q].w));
        }
        if (tl) {
          accT.x = fmaf(-wA[p], arow[QM], accT.x);
          accT.y = fmaf(-wB[p], brow[QM], accT.y);
        }
        swA += wA[p];
        swB += wB[p];
      }
      if (g != 0) swA = swB = 0.f;
#pragma unroll
      for (int q = 0; q < NQ; ++q) u[q] = rs_step(accA[q], accB[q], 4);
      u[3] = rs_step(make_float4(accT.x, swA, 0.f, 0.f), make_float4(accT.y, swB, 0.f, 0.f), 4);
    }
    {
      const float4 v0 = rs_step(u[0], u[2], 2), v1 = rs_step(u[1], u[3], 2);
      sm.cred[warp * NCOL + lane] = rs_step(v0, v1, 1);
    }
    __syncthreads();
    if (warp == 0) {
      float4 tot = sm.cred[lane];
      for (int w = 1; w < NW; ++w) tot = f4add(tot, sm.cred[w * NCOL + lane]);
      const float swA = __shfl_sync(kFull, tot.y, 3), swB = __shfl_sync(kFull, tot.y, 7);
      const int c = lane & 7, X = c >> 2, cc = c & 3, nreal = cc < 3 ? 4 : ((lane >> 3) == G - 1 ? 1 : 0);
      const float sw = X ? swB : swA;
      const float inv = sw > 0.f ? 1.f / sw : 0.f;
      float zz[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) zz[i] = i < nreal ? clampf(f4get(tot, i) * inv, prm.lo, prm.hi) : 0.f;
      zv4[vcol(lane)] = cvw[vcol(lane)] = make_float4(zz[0], zz[1], zz[2], zz[3]);
      sgv4[vcol(lane)] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
  }
  pair_iterate(sm, nA, nB, nex, prm);
  const long long pixA = (long long)y * W + x;
  if (EX && ex.z_out) {   // the whole solution patch of each pixel
    for (int i = t; i < 2 * D; i += NT) {
      const int X = i / D, q = i - X * D;
      if (X == 0 || hasB) ex.z_out[(pixA + X) * D + q] = sm.zv[vidx(q, X)];
    }
  }
  if (t == 0) {
    out[pixA] = sm.zv[vidx(D / 2, 0)];
    if (iters_used) iters_used[pixA] = (int)sm.scal[2];
    if (resid) resid[pixA] = sm.scal[3];
  } else if (t == 1 && hasB) {
    out[pixA + 1] = sm.zv[vidx(D / 2, 1)];
    if (iters_used) iters_used[pixA + 1] = (int)sm.scal[4];
    if (resid) resid[pixA + 1] = sm.scal[5];
  }
  if (obj64 || kkt64) {
    for (int X = 0; X < (hasB ? 2 : 1); ++X) {
      double F, Rk;
      pair_fp64(sm, X, nex, prm, ih2, F, Rk);
      if (t == 0) {
        if (obj64) obj64[pixA + X] = F;
        if (kkt64) kkt64[pixA + X] = Rk;
      }
      __syncthreads();
    }
  }
  __syncthreads();
}

template <bool EX>
__global__ void __launch_bounds__(NT, 1)
nlem_pair_kernel(const float* __restrict__ img, int H, int W, int pitch, int S, float inv_h2, double ih2,
                 SolveParams prm, int init_mode, float* __restrict__ out, int* __restrict__ iters_used,
                 float* __restrict__ resid, double* __restrict__ obj64, double* __restrict__ kkt64, PixelExtra ex) {
  extern __shared__ float4 smem_raw[];
  const Sm sm(reinterpret_cast<float*>(smem_raw));
  const long long items = (long long)H * ((W + 1) / 2);
  for (long long it = blockIdx.x; it < items; it += gridDim.x)
    pair_pixel<EX>(sm, img, H, W, pitch, S, inv_h2, ih2, prm, init_mode, it, out, iters_used, resid, obj64, kkt64, ex);
}

}  // namespace pairk

bool nlem_pair_eligible(const NlemLaunch& L) {
  return L.patch == pairk::K && L.S >= 1 && L.S <= 2 * ((pairk::RMAX - 1) / 2) + 1 && !L.wtab && !L.pix_list;
}

int launch_nlem_pair_k7(const NlemLaunch& L) {
  if (!nlem_pair_eligible(L)) return -1;
  const bool ex = L.ex.x0 || L.ex.rho || L.ex.z_out;
  auto kern = ex ? pairk::nlem_pair_kernel<true> : pairk::nlem_pair_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pairk::SMEM_BYTES);
  if (e != cudaSuccess) return (int)e;
  const long long items = (long long)L.H * ((L.W + 1) / 2);
  long long grid = items, cap = (long long)L.sm_count * 64;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, pairk::NT, pairk::SMEM_BYTES, L.stream>>>(L.img, L.H, L.W, L.pitch, L.S, L.inv_h2,
                                                                   L.inv_h2_exact, L.prm, L.init_mode, L.out,
                                                                   L.iters_used, L.resid, L.obj64, L.kkt64, L.ex);
  return (int)cudaGetLastError();
}

}  // namespace nlemk

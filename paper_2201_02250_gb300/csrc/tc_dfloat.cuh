// Double-float tile products on the tensor cores: C(128 x 64) -= A(128 x 64) B(64 x 64), where A, B
// and C hold double-float values, computed with BF16 x BF16 -> FP32 tcgen05 MMAs.
//
// Method (an error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 2012): every row of A is scaled by a power of two 2^eA_r >= its
// largest magnitude, every column of B by 2^eB_c, and each scaled value y in [-1, 1] is written as seven
// base-256 digits, y = sum_s t_s 256^-(s+1) with integers |t_0| <= 256, |t_s| <= 128 (s > 0), obtained by
// repeated rounding to the nearest integer (each step is exact in double-float arithmetic).  Digit s
// is stored as the BF16 value t_s 2^(-8 s), which is exact (at most 8 significant bits).  The product
// of digit i of A and digit j of B then has the natural weight 2^(-8 (i + j)), and the 28 digit pairs
// with i + j <= 6 are accumulated by the tensor cores in seven FP32 accumulator blocks, one per weight.
// Block d sums d + 1 pairs over 64 terms, at most 9 x 2^20 units of its weight, below 2^24, so FP32
// accumulates every block exactly whatever the order.  The result, 2^(eA_r + eB_c - 16) times the sum
// of the blocks, is formed in double-float.  Its error is about 2^-52 of max_k |A_rk| max_k |B_kc|
// (seven digits: the dropped pairs weigh 2^-56 and less), which stays below the double-float product's
// error bound of a few 2^-47 (|A| |B|)_rc unless the largest entries of the row and of the column sit
// at different k and exceed their partners by more than about 2^5.
//
// Shared memory: A digits 7 x 16 KiB, B digits 7 x 8 KiB (168 KiB), K-major canonical layout
// (tc_sm100.cuh).  TMEM: 7 accumulator blocks x 64 columns (512 columns allocated: one CTA per SM).
#pragma once

#include <cuda_bf16.h>

#include "dfloat.cuh"
#include "tc_sm100.cuh"

namespace a2ls {
namespace tcdf {

constexpr int TM = 128, TN = 64, TK = 64;   // tile shape
constexpr int NDIG = 7;                      // base-256 digits per value
constexpr int NBLK = NDIG;                   // exact accumulator blocks, one per digit weight 0 .. 6
constexpr uint32_t A_DIGIT_BYTES = TM * TK * 2;
constexpr uint32_t B_DIGIT_BYTES = TN * TK * 2;
constexpr size_t SMEM_BYTES = (size_t)NDIG * (A_DIGIT_BYTES + B_DIGIT_BYTES);   // 172032
constexpr uint32_t TMEM_COLS = 512;
constexpr long WAIT_LIMIT = 1L << 26;        // polls of the completion barrier before giving up

// the NDIG digits of y = x / 2^e (|y| <= 1), as BF16 values t_s 2^(-8 s)
__device__ __forceinline__ void df_digits(dfloat x, int e, __nv_bfloat16 (&d)[NDIG]) {
  float yh = ldexpf(x.hi, -e), yl = ldexpf(x.lo, -e);
#pragma unroll
  for (int s = 0; s < NDIG; ++s) {
    const float t = rintf(__fmul_rn(yh, 256.f));
    d[s] = __float2bfloat16_rn(ldexpf(t, -8 * s));
    // y <- 256 y - t: exact (256 y is exact and t is within one half of it)
    yh = __fsub_rn(__fmul_rn(yh, 256.f), t);
    yl = __fmul_rn(yl, 256.f);
    const dfloat r = df_two_sum(yh, yl);
    yh = r.hi;
    yl = r.lo;
  }
}

// exponent e with |v| < 2^e (0 for v = 0)
__device__ __forceinline__ int scale_exponent(float maxabs) {
  int e = 0;
  if (maxabs > 0.f) frexpf(maxabs, &e);
  return e;
}

struct Ctx {
  unsigned char* smem;   // SMEM_BYTES, 16-byte aligned
  uint64_t* bar;         // completion mbarrier (initialised with count 1)
  uint32_t tmem;         // TMEM base address (TMEM_COLS columns)
  uint32_t phase;        // parity of the next completion
  int* eA;               // shared, TM row exponents
  int* eB;               // shared, TN column exponents
};

// A digits: rows [0, TM) x k [0, TK) of A(m, k) = fa(m, k) (zero outside), 256 threads: two per row.
template <class FA>
__device__ __forceinline__ void split_a(Ctx& c, FA fa) {
  const int tid = threadIdx.x, r = tid >> 1, h = tid & 1;
  dfloat v[32];
  float mx = 0.f;
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    v[q] = fa(r, h * 32 + q);
    mx = fmaxf(mx, fabsf(v[q].hi));
  }
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  const int e = scale_exponent(mx);
  if (h == 0) c.eA[r] = e;
#pragma unroll
  for (int q8 = 0; q8 < 4; ++q8) {
    __nv_bfloat16 dg[8][NDIG];
#pragma unroll
    for (int q = 0; q < 8; ++q) df_digits(v[q8 * 8 + q], e, dg[q]);
    const uint32_t off = tc::operand_offset(r, h * 32 + q8 * 8, TK);
#pragma unroll
    for (int s = 0; s < NDIG; ++s) {
      __nv_bfloat162 p0 = __halves2bfloat162(dg[0][s], dg[1][s]), p1 = __halves2bfloat162(dg[2][s], dg[3][s]),
                     p2 = __halves2bfloat162(dg[4][s], dg[5][s]), p3 = __halves2bfloat162(dg[6][s], dg[7][s]);
      uint4 w;
      w.x = *reinterpret_cast<uint32_t*>(&p0);
      w.y = *reinterpret_cast<uint32_t*>(&p1);
      w.z = *reinterpret_cast<uint32_t*>(&p2);
      w.w = *reinterpret_cast<uint32_t*>(&p3);
      *reinterpret_cast<uint4*>(c.smem + s * A_DIGIT_BYTES + off) = w;
    }
  }
}

// B digits: k [0, TK) x columns [0, TN) of B(k, n) = fb(k, n), stored as the K-major operand (n, k);
// 256 threads: column n = tid % 64, k quarter tid / 64.  red: shared scratch of 4 x TN floats.
template <class FB>
__device__ __forceinline__ void split_b(Ctx& c, FB fb, float* red) {
  const int tid = threadIdx.x, n = tid & (TN - 1), qk = tid >> 6;
  dfloat v[16];
  float mx = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    v[q] = fb(qk * 16 + q, n);
    mx = fmaxf(mx, fabsf(v[q].hi));
  }
  red[qk * TN + n] = mx;
  __syncthreads();
  mx = fmaxf(fmaxf(red[n], red[TN + n]), fmaxf(red[2 * TN + n], red[3 * TN + n]));
  const int e = scale_exponent(mx);
  if (qk == 0) c.eB[n] = e;
#pragma unroll
  for (int q8 = 0; q8 < 2; ++q8) {
    __nv_bfloat16 dg[8][NDIG];
#pragma unroll
    for (int q = 0; q < 8; ++q) df_digits(v[q8 * 8 + q], e, dg[q]);
    const uint32_t off = tc::operand_offset(n, qk * 16 + q8 * 8, TK);
#pragma unroll
    for (int s = 0; s < NDIG; ++s) {
      __nv_bfloat162 p0 = __halves2bfloat162(dg[0][s], dg[1][s]), p1 = __halves2bfloat162(dg[2][s], dg[3][s]),
                     p2 = __halves2bfloat162(dg[4][s], dg[5][s]), p3 = __halves2bfloat162(dg[6][s], dg[7][s]);
      uint4 w;
      w.x = *reinterpret_cast<uint32_t*>(&p0);
      w.y = *reinterpret_cast<uint32_t*>(&p1);
      w.z = *reinterpret_cast<uint32_t*>(&p2);
      w.w = *reinterpret_cast<uint32_t*>(&p3);
      *reinterpret_cast<uint4*>(c.smem + NDIG * A_DIGIT_BYTES + s * B_DIGIT_BYTES + off) = w;
    }
  }
}

// After split_a / split_b by all threads: the 40 MMAs of the 28 digit pairs, issued by thread 0, then
// a bounded wait by every thread.  Returns false (on every thread) if the products did not complete.
__device__ __forceinline__ bool multiply(Ctx& c) {
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0) {
    const uint32_t a0 = tc::smem_u32(c.smem), b0 = a0 + NDIG * A_DIGIT_BYTES;
    // descriptors of the first K-chunk of digit plane 0; the others differ only in the start address
    // field (address / 16, low bits), which no offset here carries out of
    const uint64_t ad0 = tc::smem_desc(a0, 128, TK * 16), bd0 = tc::smem_desc(b0, 128, TK * 16);
    // The B digit planes are consecutive 64-row groups of one K-major operand, so an MMA with A digit i
    // and B digits j0 .. j0 + nj - 1 (N = 64 nj <= 256) writes pair (i, j) into block i + j, the
    // block of its weight.  The two MMAs of digit 0 write all seven blocks first; the others add.
#pragma unroll
    for (int i = 0; i < NDIG; ++i)
#pragma unroll
      for (int j0 = 0; j0 < NDIG - i; j0 += 4) {
        const int nj = (NDIG - i - j0) < 4 ? (NDIG - i - j0) : 4;
        const uint32_t idesc = tc::idesc_bf16_f32(TM, TN * nj);
#pragma unroll
        for (int kk = 0; kk < TK / 16; ++kk)
          tc::mma_bf16(c.tmem + (i + j0) * TN, ad0 + ((i * A_DIGIT_BYTES + kk * 256) >> 4),
                       bd0 + ((j0 * B_DIGIT_BYTES + kk * 256) >> 4), idesc, (i == 0 && kk == 0) ? 0u : 1u);
      }
    tc::commit(c.bar);
  }
  __syncwarp();
  const bool ok = tc::mbar_wait_bounded(c.bar, c.phase, WAIT_LIMIT);
  c.phase ^= 1u;
  tc::fence_after_sync();
  return __syncthreads_and(ok) != 0;
}

// L2 prefetch of rows [0, rows) x bytes [0, row_bytes) starting at base with the given row pitch,
// spread over the CTA (one 128-byte line per request)
__device__ __forceinline__ void prefetch_rows_l2(const void* base, int64_t pitch_bytes, int rows, int row_bytes) {
  // one request per 128-byte line the row's bytes touch, at the line's aligned start (a row may start
  // anywhere in a line; no request reaches past the row's last byte's line)
  if (row_bytes <= 0) return;
  const int lines = (row_bytes + 127) / 128 + 1;
  for (int e = threadIdx.x; e < rows * lines; e += blockDim.x) {
    const uintptr_t first = reinterpret_cast<uintptr_t>(base) + (uintptr_t)((e / lines) * pitch_bytes);
    const uintptr_t line = (first & ~(uintptr_t)127) + (uintptr_t)(e % lines) * 128;
    if (line <= first + row_bytes - 1) asm volatile("prefetch.global.L2 [%0];" ::"l"(line));
  }
}

// C(rows x cols) -= the tile product, for C in global memory (double-float, row pitch ldc elements),
// coalesced: in two halves of 32 columns, the old values are read row-contiguously into shared memory
// (the B digits' region, free once the MMAs have completed), each thread subtracts the product for 16
// outputs of its TMEM lane (warp w: rows 32 (w % 4) .., columns 16 (w / 4) .. of the half), and the
// half is written back row-contiguously.  Ends with the fences and barrier that let the next tile reuse
// TMEM and shared memory.
constexpr int SUB_LD = 33;   // staging row stride in double-float values (odd: spreads the banks)
__device__ __forceinline__ void epilogue_subtract(Ctx& c, dfloat* C, int64_t ldc, int rows, int cols) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = (warp & 3) * 32 + lane, nq = (warp >> 2) * 16;
  const uint32_t lane_addr = c.tmem + ((uint32_t)((warp & 3) * 32) << 16);
  dfloat* S = reinterpret_cast<dfloat*>(c.smem + NDIG * A_DIGIT_BYTES);   // TM x SUB_LD
  const int em = c.eA[m];
#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    const int cbase = half * 32;
    // old values: one warp per row, one 8-byte value per thread (C's column offset can be odd: the
    // overlap phase of the factorisation starts at column n_I, so wider accesses could be misaligned)
    for (int e = tid; e < TM * 32; e += 256) {
      const int r = e >> 5, cc = e & 31, col = cbase + cc;
      S[r * SUB_LD + cc] = (r < rows && col < cols) ? C[(int64_t)r * ldc + col] : dfloat(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int cb = 0; cb < 16; cb += 8) {
      float acc[NBLK][8];
#pragma unroll
      for (int g = 0; g < NBLK; ++g) tc::tmem_ld8(lane_addr + g * TN + cbase + nq + cb, acc[g]);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        dfloat sum = df_two_sum(acc[0][q], acc[1][q]);
#pragma unroll
        for (int g = 2; g < NBLK; ++g) sum = sum + dfloat(acc[g][q], 0.f);
        const int e = em + c.eB[cbase + nq + cb + q] - 16;
        dfloat& o = S[m * SUB_LD + nq + cb + q];
        o = o - dfloat(ldexpf(sum.hi, e), ldexpf(sum.lo, e));
      }
    }
    __syncthreads();
    for (int e = tid; e < TM * 32; e += 256) {
      const int r = e >> 5, cc = e & 31, col = cbase + cc;
      if (r < rows && col < cols) C[(int64_t)r * ldc + col] = S[r * SUB_LD + cc];
    }
    __syncthreads();
  }
  tc::fence_before_sync();
  __syncthreads();
}

}  // namespace tcdf
}  // namespace a2ls

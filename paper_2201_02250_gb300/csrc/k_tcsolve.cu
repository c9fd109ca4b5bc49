// Double-float block triangular solves of the local eigensolves on the tensor cores.
//
// The operator of the local eigenproblem (Eq. 3.1) is applied through the double-float LU of the
// splitting A~_ii: X <- inv(U) inv(L) X for a block of p <= 32 columns.  In the block-inverted storage
// both sweeps are sequences of 64 x 64 tile products (k_dense.cu).  Here each product runs as
// BF16 x BF16 -> FP32 tcgen05 MMAs on base-256 digit expansions (the scheme of tc_dfloat.cuh):
//   * after the factorisation every 64 x 64 factor tile a sweep reads (the off-diagonal tiles inside
//     the envelope of L and U, and the two inverted triangles of each diagonal tile) is split once
//     into seven BF16 digit planes with one power-of-two scale per row (k_factor_digits);
//   * a sweep keeps, for every finished 64-row block of X, its seven digit planes with one scale per
//     column in a scratch array, so that each later block reads digits instead of splitting again;
//   * per 64-row block, the tiles of its panel stream through two shared-memory stages by cp.async,
//     their 112 M=64 x N=32 x K=16 MMAs (28 digit pairs) fill one of two TMEM buffers while the CTA
//     folds the previous tile's five accumulator blocks into double-float registers; then the diagonal
//     tile product X_b = inv(T_bb) (X_b - panel) runs the same way and X_b's digits are stored.
// One CTA of 256 threads per subdomain (largest first); 173 KB of shared memory and 512 TMEM columns.
#include "a2ls_internal.cuh"
#include "tc_dfloat.cuh"

#include <algorithm>

namespace a2ls {
namespace tcs {

constexpr int M = 64, NC = 32, K = 64, NDIG = tcdf::NDIG;
// FP32 accumulator blocks of NC columns: digit weights 0, 1, 2, 3 (exact) and 4-6 together
constexpr int NBLK = 5;
constexpr uint32_t A_PLANE = M * K * 2;            // 8 KiB
constexpr uint32_t B_PLANE = NC * K * 2;           // 4 KiB
constexpr uint32_t A_TILE = NDIG * A_PLANE + M * 4;   // digit planes, then int32 row exponents
constexpr uint32_t B_TILE = NDIG * B_PLANE + NC * 4;  // digit planes, then int32 column exponents
constexpr uint32_t STAGE = A_TILE + B_TILE;
constexpr size_t SMEM = 2 * (size_t)STAGE;
constexpr uint32_t BUF_COLS = NBLK * NC;           // TMEM columns of one accumulator buffer
constexpr uint32_t TMEM_COLS = 512;
constexpr int THREADS = 256;
static_assert(A_TILE % 16 == 0 && B_TILE % 16 == 0, "16-byte copies");
static_assert(2 * BUF_COLS <= TMEM_COLS, "two accumulator buffers");

// kinds of digit tiles
enum { KIND_OFF = 0, KIND_DIAG_LOWER = 1, KIND_DIAG_UPPER = 2 };

// ---------------------------------------------------------------------------------------------
// digits of the factor tiles: one CTA per tile (i, b, c, kind) -> fdig + index * A_TILE
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS) k_factor_digits(const int4* __restrict__ jobs, const int* ni,
                                                           const int* ld, const int64_t* foff,
                                                           const dfloat* __restrict__ fac,
                                                           unsigned char* __restrict__ fdig) {
  const int4 jb = jobs[blockIdx.x];
  const int i = jb.x, b = jb.y, c = jb.z, kind = jb.w;
  const int n = ni[i];
  const int64_t L = ld[i];
  const dfloat* A = fac + foff[i];
  unsigned char* out = fdig + (size_t)blockIdx.x * A_TILE;
  const int t = threadIdx.x, r = t >> 2, q = t & 3;   // row r, k-quarter q (16 columns)
  const int gr = b * M + r;
  dfloat v[16];
  float mx = 0.f;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int k = q * 16 + u, gc = c * K + k;
    dfloat x(0.f, 0.f);
    if (gr < n && gc < n) {
      if (kind == KIND_OFF) x = A[(int64_t)gr * L + gc];
      else if (kind == KIND_DIAG_LOWER) x = (k < r) ? A[(int64_t)gr * L + gc] : (k == r ? dfloat(1.f, 0.f) : x);
      else x = (k >= r) ? A[(int64_t)gr * L + gc] : x;
    }
    v[u] = x;
    mx = fmaxf(mx, fabsf(x.hi));
  }
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  const int e = tcdf::scale_exponent(mx);
  if (q == 0) reinterpret_cast<int*>(out + NDIG * A_PLANE)[r] = e;
#pragma unroll
  for (int h8 = 0; h8 < 2; ++h8) {
    __nv_bfloat16 dg[8][NDIG];
#pragma unroll
    for (int u = 0; u < 8; ++u) tcdf::df_digits(v[h8 * 8 + u], e, dg[u]);
    const uint32_t off = tc::operand_offset(r, q * 16 + h8 * 8, K);
#pragma unroll
    for (int s = 0; s < NDIG; ++s) {
      __nv_bfloat162 p0 = __halves2bfloat162(dg[0][s], dg[1][s]), p1 = __halves2bfloat162(dg[2][s], dg[3][s]),
                     p2 = __halves2bfloat162(dg[4][s], dg[5][s]), p3 = __halves2bfloat162(dg[6][s], dg[7][s]);
      uint4 w;
      w.x = *reinterpret_cast<uint32_t*>(&p0);
      w.y = *reinterpret_cast<uint32_t*>(&p1);
      w.z = *reinterpret_cast<uint32_t*>(&p2);
      w.w = *reinterpret_cast<uint32_t*>(&p3);
      *reinterpret_cast<uint4*>(out + s * A_PLANE + off) = w;
    }
  }
}

// 16-byte asynchronous copy with an L2 eviction-priority policy
__device__ __forceinline__ void cp16(void* smem, const void* gmem, uint64_t policy) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(smem)), "l"(gmem),
               "l"(policy)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// the factor digits stream through L2 once per sweep (evicted first); the digits of X's finished
// blocks are read again by every later block of the sweep (kept)
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// bytes [0, nbytes) from src to dst in 16-byte copies by the whole CTA (one commit group)
__device__ __forceinline__ void copy_async(unsigned char* dst, const unsigned char* src, uint32_t nbytes,
                                           uint64_t policy) {
  for (uint32_t o = threadIdx.x * 16; o < nbytes; o += THREADS * 16) cp16(dst + o, src + o, policy);
  cp_commit();
}

// digits of S (64 rows x 32 columns of double-float in shared memory) as the N x K operand (column j
// is operand row j, S's row index is K), one scale per column; red: 8 x 32 floats of scratch
__device__ __forceinline__ void split_columns(const dfloat* S, unsigned char* dst, float* red) {
  const int t = threadIdx.x, j = t & 31, g = t >> 5;   // column j, rows 8g .. 8g + 7
  dfloat v[8];
  float mx = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = S[(g * 8 + k) * NC + j];
    mx = fmaxf(mx, fabsf(v[k].hi));
  }
  red[g * NC + j] = mx;
  __syncthreads();
  mx = 0.f;
#pragma unroll
  for (int u = 0; u < 8; ++u) mx = fmaxf(mx, red[u * NC + j]);
  const int e = tcdf::scale_exponent(mx);
  if (g == 0) reinterpret_cast<int*>(dst + NDIG * B_PLANE)[j] = e;
  __nv_bfloat16 dg[8][NDIG];
#pragma unroll
  for (int k = 0; k < 8; ++k) tcdf::df_digits(v[k], e, dg[k]);
  const uint32_t off = tc::operand_offset(j, g * 8, K);
#pragma unroll
  for (int s = 0; s < NDIG; ++s) {
    __nv_bfloat162 p0 = __halves2bfloat162(dg[0][s], dg[1][s]), p1 = __halves2bfloat162(dg[2][s], dg[3][s]),
                   p2 = __halves2bfloat162(dg[4][s], dg[5][s]), p3 = __halves2bfloat162(dg[6][s], dg[7][s]);
    uint4 w;
    w.x = *reinterpret_cast<uint32_t*>(&p0);
    w.y = *reinterpret_cast<uint32_t*>(&p1);
    w.z = *reinterpret_cast<uint32_t*>(&p2);
    w.w = *reinterpret_cast<uint32_t*>(&p3);
    *reinterpret_cast<uint4*>(dst + s * B_PLANE + off) = w;
  }
}

// The 112 MMAs of one tile product (A digits at a, B digits at b) into TMEM buffer `buf`: pair (i, j) of
// digits, M = 64, N = 32, into the block of its weight i + j (weights 4 to 6 share the last block).  The
// blocks of weight 0 to 3 stay below 2^24 units of their weight over 64 terms and are exact; the shared
// last block rounds at 2^-56 of the result.  Two threads of different warps issue in parallel, each for
// its own blocks (part 0: weights 0-3, 40 MMAs; part 1: weights 4-6, 72 MMAs), then each commits to the
// barrier (initialised for two arrivals).  The first product into a block, pair (0, j) with j its
// first weight, overwrites it; the MMAs of one issuing thread run in order.
__device__ __forceinline__ void issue_mmas(uint32_t tmem, int buf, const unsigned char* a, const unsigned char* bsm,
                                           uint64_t* bar, int part) {
  constexpr uint32_t idesc = tc::idesc_bf16_f32(M, NC);
  const uint32_t a0 = tc::smem_u32(a), b0 = tc::smem_u32(bsm);
  // descriptors of the first K-chunk of plane 0; the others differ only in the start address field
  const uint64_t ad0 = tc::smem_desc(a0, 128, K * 16), bd0 = tc::smem_desc(b0, 128, K * 16);
#pragma unroll
  for (int i = 0; i < NDIG; ++i)
#pragma unroll
    for (int j = 0; j < NDIG - i; ++j) {
      if ((i + j >= NBLK - 1) != (part == 1)) continue;
#pragma unroll
      for (int kk = 0; kk < K / 16; ++kk)
        tc::mma_bf16(tmem + buf * BUF_COLS + (i + j < NBLK ? i + j : NBLK - 1) * NC,
                     ad0 + ((i * A_PLANE + kk * 256) >> 4), bd0 + ((j * B_PLANE + kk * 256) >> 4), idesc,
                     (i == 0 && j < NBLK && kk == 0) ? 0u : 1u);
    }
  tc::commit(bar);
}

template <class F>
__device__ __forceinline__ void fold(uint32_t tmem, int buf, const int* eA, const int* eB, F f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qd = warp & 3, h = warp >> 2;
  const int row = qd * 16 + (lane & 15);
  const uint32_t base = tmem + ((uint32_t)(qd * 32) << 16) + buf * BUF_COLS + h * 16;
  const int er = eA[row];
#pragma unroll
  for (int c8 = 0; c8 < 16; c8 += 8) {
    float acc[NBLK][8];
#pragma unroll
    for (int g = 0; g < NBLK; ++g) tc::tmem_ld8(base + g * NC + c8, acc[g]);
    tc::tmem_wait_ld();
    if (lane < 16) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        // exact sum of the two leading blocks, then the smaller ones in decreasing weight
        dfloat s = df_two_sum(acc[0][q], acc[1][q]);
#pragma unroll
        for (int g = 2; g < NBLK; ++g) s = s + dfloat(acc[g][q], 0.f);
        const int col = h * 16 + c8 + q;
        const int e = er + eB[col] - 16;
        f(col, dfloat(ldexpf(s.hi, e), ldexpf(s.lo, e)));
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// one sweep (forward with L, or backward with U) over the subdomains with 1 <= p <= 32
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS, 1) k_block_solve_tc(
    const int* ni, const int* sched, const int* active, const int* pvec, dfloat* X, const int64_t* xoff, int col0,
    int ldx, const int64_t* ftoff, const int64_t* ftab, const unsigned char* __restrict__ fdig,
    unsigned char* __restrict__ xdig, const int64_t* xdoff, int forward, int* st) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tbase;
  __shared__ float red[8 * NC];
  __shared__ int tiles[MAXN_LOCAL / M + 1];
  __shared__ int sexpA[2][M], sexpB[2][NC];   // scale exponents of the tiles in flight
  const int i = sched[blockIdx.x];
  if (active && !active[i]) return;
  const int p = pvec[i];
  if (p < 1 || p > NC) return;
  const int n = ni[i], nb = (n + M - 1) / M;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {   // two arrivals per phase: the two MMA-issuing threads commit separately
    tc::mbar_init(&bar[0], 2);
    tc::mbar_init(&bar[1], 2);
  }
  if (warp == 0) {
    tc::tmem_alloc(&tbase, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;
  dfloat* Xi = X + xoff[i] + col0;
  const int64_t* tab = ftab + ftoff[i];   // nb x (nb + 1): (b, c) tile, (b, nb) the upper diagonal inverse
  unsigned char* xd = xdig + xdoff[i];
  unsigned char* stage[2] = {sm, sm + STAGE};
  const int qd = warp & 3, h = warp >> 2, row = qd * 16 + (lane & 15);

  const uint64_t pol_stream = policy_evict_first(), pol_keep = policy_evict_last();
  auto wait_mma = [&](int u) -> bool {
    const bool done = tc::mbar_wait_bounded(&bar[u], phase[u], tcdf::WAIT_LIMIT);
    phase[u] ^= 1u;
    tc::fence_after_sync();
    return done;
  };

  for (int bb = 0; bb < nb && ok; ++bb) {
    const int b = forward ? bb : nb - 1 - bb;
    const int r0 = b * M, tb = min(M, n - r0);
    // tiles of the block's panel (the list is built by thread 0 and read by all after a barrier)
    const int c_lo = forward ? 0 : b + 1, c_hi = forward ? b : nb;
    __shared__ int ntiles;
    if (tid == 0) {
      int T0 = 0;
      for (int c = c_lo; c < c_hi; ++c)
        if (tab[(int64_t)b * (nb + 1) + c] >= 0) tiles[T0++] = c;
      ntiles = T0;
    }
    __syncthreads();
    const int T = ntiles;
    dfloat acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = dfloat(0.f, 0.f);
    auto load = [&](int tt) {
      const int c = tiles[tt];
      unsigned char* sgt = stage[tt & 1];
      copy_async(sgt, fdig + tab[(int64_t)b * (nb + 1) + c], A_TILE, pol_stream);
      copy_async(sgt + A_TILE, xd + (size_t)c * B_TILE, B_TILE, pol_keep);
    };
    // Pipeline per tile tt: wait for its operands, save its scale exponents (the stage is refilled
    // before the fold reads them), issue its MMAs into TMEM buffer tt & 1, wait for tile tt - 1's MMAs,
    // start loading tile tt + 1 into the stage tile tt - 1 used, then fold tile tt - 1.  The copies of
    // tile tt + 1 thus overlap tile tt's MMAs and tile tt - 1's fold.
    if (T > 0) load(0);
    for (int tt = 0; tt < T && ok; ++tt) {
      cp_wait_all();
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();   // every thread's copies of tile tt have landed
      tc::fence_after_sync();
      {
        const unsigned char* sp = stage[tt & 1];
        if (tid < M) sexpA[tt & 1][tid] = reinterpret_cast<const int*>(sp + NDIG * A_PLANE)[tid];
        else if (tid < M + NC) sexpB[tt & 1][tid - M] = reinterpret_cast<const int*>(sp + A_TILE + NDIG * B_PLANE)[tid - M];
      }
      if (tid == 0 || tid == 32) issue_mmas(tmem, tt & 1, stage[tt & 1], stage[tt & 1] + A_TILE, &bar[tt & 1], tid >> 5);
      __syncwarp();
      if (tt > 0) {
        const int u = (tt - 1) & 1;
        ok = __syncthreads_and(wait_mma(u)) != 0;
        if (!ok) break;
        if (tt + 1 < T) load(tt + 1);   // stage u is free: tile tt - 1's MMAs have completed
        fold(tmem, u, sexpA[u], sexpB[u], [&](int col, dfloat v) { acc[col - h * 16] += v; });
        tc::fence_before_sync();
        __syncthreads();   // TMEM buffer u is read before tile tt + 1's MMAs overwrite it
      } else {
        if (tt + 1 < T) load(tt + 1);   // stage 1 has not been used yet
        __syncthreads();   // the saved exponents of tile 0 are visible before its fold
      }
    }
    if (T > 0 && ok) {
      const int u = (T - 1) & 1;
      ok = __syncthreads_and(wait_mma(u)) != 0;
      if (ok) fold(tmem, u, sexpA[u], sexpB[u], [&](int col, dfloat v) { acc[col - h * 16] += v; });
      tc::fence_before_sync();
      __syncthreads();
    }
    if (!ok) break;
    // S = X_b - panel (64 x 32, zero outside the block and the columns) in stage 1, the inverted
    // diagonal tile's digits into stage 0
    dfloat* S = reinterpret_cast<dfloat*>(stage[1]);
    copy_async(stage[0], fdig + tab[(int64_t)b * (nb + 1) + (forward ? b : nb)], A_TILE, pol_stream);
    if (lane < 16) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int col = h * 16 + u;
        dfloat x(0.f, 0.f);
        if (row < tb && col < p) x = Xi[(int64_t)(r0 + row) * ldx + col] - acc[u];
        S[row * NC + col] = x;
      }
    }
    __syncthreads();
    split_columns(S, stage[0] + A_TILE, red);
    cp_wait_all();
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0 || tid == 32) issue_mmas(tmem, 0, stage[0], stage[0] + A_TILE, &bar[0], tid >> 5);
    __syncwarp();
    ok = __syncthreads_and(wait_mma(0)) != 0;
    if (!ok) break;
    // X_b = inv(T_bb) S: written to X and, for the later blocks of the sweep, as digits
    fold(tmem, 0, reinterpret_cast<const int*>(stage[0] + NDIG * A_PLANE),
         reinterpret_cast<const int*>(stage[0] + A_TILE + NDIG * B_PLANE), [&](int col, dfloat v) {
           if (row < tb && col < p) Xi[(int64_t)(r0 + row) * ldx + col] = v;
           S[row * NC + col] = (row < tb && col < p) ? v : dfloat(0.f, 0.f);
         });
    tc::fence_before_sync();
    __syncthreads();
    split_columns(S, stage[1] + sizeof(dfloat) * M * NC, red);
    __syncthreads();
    {
      const uint4* src = reinterpret_cast<const uint4*>(stage[1] + sizeof(dfloat) * M * NC);
      uint4* dst = reinterpret_cast<uint4*>(xd + (size_t)b * B_TILE);
      for (uint32_t o = tid; o < B_TILE / 16; o += THREADS) dst[o] = src[o];
    }
    __threadfence();   // the digits are read back through L2 by this CTA's later asynchronous copies
    __syncthreads();
  }
  if (!ok && tid == 0) raise_status(st, A2LS_ERR_TIMEOUT, i, forward);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace tcs

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
void tc_solve_prepare(a2ls_handle* h, const dfloat* fac, TcSolve& ts) {
  using namespace tcs;
  cudaStream_t st = h->st;
  const int N = h->N;
  const int T = h->h_toff[N];
  std::vector<int> tf(T), tg(T);
  A2LS_CUDA(cudaMemcpyAsync(tf.data(), h->d_tf, sizeof(int) * T, cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaMemcpyAsync(tg.data(), h->d_tg, sizeof(int) * T, cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  std::vector<int64_t> ftoff(N + 1, 0), xdoff(N + 1, 0);
  for (int i = 0; i < N; ++i) {
    const int nb = (h->h_n[i] + M - 1) / M;
    ftoff[i + 1] = ftoff[i] + (int64_t)nb * (nb + 1);
    xdoff[i + 1] = xdoff[i] + (int64_t)nb * B_TILE;
  }
  std::vector<int64_t> tab(ftoff[N], -1);
  std::vector<int4> jobs;
  for (int i = 0; i < N; ++i) {
    const int nb = (h->h_n[i] + M - 1) / M;
    const int* tfi = tf.data() + h->h_toff[i];
    const int* tgi = tg.data() + h->h_toff[i];
    int64_t* ti = tab.data() + ftoff[i];
    auto add = [&](int b, int c, int slot, int kind) {
      ti[(int64_t)b * (nb + 1) + slot] = (int64_t)jobs.size() * A_TILE;
      jobs.push_back(make_int4(i, b, c, kind));
    };
    for (int b = 0; b < nb; ++b) {
      for (int c = 0; c < b; ++c)
        if (tfi[b] <= c * M + M - 1) add(b, c, c, KIND_OFF);        // L: row block b reaches column tile c
      add(b, b, b, KIND_DIAG_LOWER);
      for (int c = b + 1; c < nb; ++c)
        if (tgi[c] <= b * M + M - 1) add(b, c, c, KIND_OFF);        // U: column tile c reaches row block b
      add(b, b, nb, KIND_DIAG_UPPER);
    }
  }
  ts.ntiles = (int64_t)jobs.size();
  ts.d_ftoff = dalloc<int64_t>(h, N + 1);
  ts.d_ftab = dalloc<int64_t>(h, ftoff[N]);
  ts.d_xdoff = dalloc<int64_t>(h, N + 1);
  ts.d_fdig = dalloc<unsigned char>(h, (size_t)ts.ntiles * A_TILE);
  ts.d_xdig = dalloc<unsigned char>(h, (size_t)xdoff[N]);
  int4* d_jobs = dalloc<int4>(h, jobs.size());
  A2LS_CUDA(cudaMemcpyAsync(ts.d_ftoff, ftoff.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(ts.d_ftab, tab.data(), sizeof(int64_t) * tab.size(), cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(ts.d_xdoff, xdoff.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(int4) * jobs.size(), cudaMemcpyHostToDevice, st));
  // the grid dimension limit (2^31 - 1) is far above any tile count the 8192-row subdomains allow
  k_factor_digits<<<(unsigned)jobs.size(), THREADS, 0, st>>>(d_jobs, h->d_ni, h->d_ld, h->d_foff, fac, ts.d_fdig);
  A2LS_LAUNCH();
  A2LS_CUDA(cudaFuncSetAttribute(k_block_solve_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
  A2LS_CUDA(cudaStreamSynchronize(st));   // the job list is freed below
  dfree(h, d_jobs);
  ts.ready = true;
}

void tc_solve_release(a2ls_handle* h, TcSolve& ts) {
  if (!ts.ready) return;
  dfree(h, ts.d_ftoff);
  dfree(h, ts.d_ftab);
  dfree(h, ts.d_xdoff);
  dfree(h, ts.d_fdig);
  dfree(h, ts.d_xdig);
  ts = TcSolve{};
}

void tc_block_solve(a2ls_handle* h, const TcSolve& ts, dfloat* X, const int64_t* xoff, int col0, int ldx,
                    const int* pvec, const int* active, int forward, unsigned char* xdig) {
  using namespace tcs;
  tcs::k_block_solve_tc<<<h->N, THREADS, SMEM, h->st>>>(h->d_ni, h->d_sched, active, pvec, X, xoff, col0, ldx,
                                                        ts.d_ftoff, ts.d_ftab, ts.d_fdig, xdig ? xdig : ts.d_xdig,
                                                        ts.d_xdoff, forward, h->d_status);
  A2LS_LAUNCH();
}

}  // namespace a2ls

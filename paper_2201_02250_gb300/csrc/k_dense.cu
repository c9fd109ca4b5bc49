// Batched dense kernels over the subdomains: LU without pivoting (exact local
// LU of Section 4; no pivoting is needed for the diagonally dominant local
// matrices of the target problems and a pivot check reports A2LS_ERR_SINGULAR
// otherwise), inversion of the 64x64 diagonal tiles, and the triangular
// solves of the apply (single right-hand side) and of the eigensolver
// (p right-hand sides).
//
// Storage of one factored subdomain (n x n, row-major, leading dimension ld):
// unit-lower L strictly below the diagonal, U on and above it, except inside
// the 64x64 diagonal tiles, which hold inv(L_bb) strictly below their
// diagonal and inv(U_bb) on and above it.  A triangular solve is then a
// sequence of dense matrix-vector products (no sequential substitution).
#include "a2ls_internal.cuh"
#include "tc_dfloat.cuh"

#include <algorithm>
#include <type_traits>

namespace a2ls {

template <class T> struct AccOf;
template <> struct AccOf<__nv_bfloat16> { using type = float; };
template <> struct AccOf<float> { using type = float; };
template <> struct AccOf<double> { using type = double; };
template <> struct AccOf<dfloat> { using type = dfloat; };

// depth of the operand chunks staged by the tile products
constexpr int GK = 32;

// ---------------------------------------------------------------------------
// Narrowest tile product for the column chunks of the eigen solves: M <= 64 rows, Nc <= 8
// columns; 256 threads, thread (ty, tx) owns row ty and columns 2tx, 2tx+1.
// ---------------------------------------------------------------------------
template <class T, class Acc>
__device__ __forceinline__ void cta_gemm_n8(const T* __restrict__ A, int64_t lda, const T* __restrict__ B,
                                            int64_t ldb, int M, int Nc, int K, int amask, Acc (&acc)[2], Acc* sA,
                                            Acc* sB) {
  const int tid = threadIdx.x, tx = tid & 3, ty = tid >> 2;
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = tid; e < 64 * GK; e += 256) {
      const int m = e / GK, k = e % GK;
      Acc v = 0;
      const int kk = k0 + k;
      if (m < M && kk < K) {
        if (amask == 0) v = (Acc)A[m * lda + kk];
        else if (amask == 1) v = (kk < m) ? (Acc)A[m * lda + kk] : (kk == m ? (Acc)1 : (Acc)0);
        else v = (kk >= m) ? (Acc)A[m * lda + kk] : (Acc)0;
      }
      sA[k * 65 + m] = v;
    }
    {
      const int e = tid;  // GK * 8 == 256
      const int k = e / 8, c = e % 8;
      const int kk = k0 + k;
      sB[k * 9 + c] = (c < Nc && kk < K) ? (Acc)B[kk * ldb + c] : (Acc)0;
    }
    __syncthreads();
    // a triangular A has no entries of row ty in this chunk when the chunk lies wholly right of the
    // diagonal (unit lower) or wholly left of it (upper); whole warps skip together
    const bool zero_chunk = (amask == 1 && k0 > ty) || (amask == 2 && k0 + GK - 1 < ty);
    if (tx * 2 < Nc && !zero_chunk) {
#pragma unroll 8
      for (int k = 0; k < GK; ++k) {
        const Acc a = sA[k * 65 + ty];
        mac(acc[0], a, sB[k * 9 + tx * 2]);
        mac(acc[1], a, sB[k * 9 + tx * 2 + 1]);
      }
    }
    __syncthreads();
  }
}

// Inverses of the triangles of a factored tb x tb block t (unit lower L strictly below the diagonal,
// U on and above it) into s, given rp[c] = 1 / U_cc.  256 threads, two per column: each sums every
// other term of the column's dot products with two accumulators (a quarter of the serial chain);
// threads 0-127 form inv(L), 128-255 inv(U).  The pair sums are full-warp shuffles, so every thread
// of the block must call this.
template <class R>
__device__ void tile_inverses(const R (*t)[TB + 1], R (*s)[TB + 1], const R* rp, int tb) {
  const int tid = threadIdx.x;
  const int col = (tid & 127) >> 1, h = tid & 1;
  const bool active_col = col < tb;
  if (tid < 128) {
    // inv(L), column col: x_r = -(L[r][col] + sum_{q=col+1}^{r-1} L[r][q] x_q); this thread sums the q
    // with (q - col - 1) % 2 == h and writes the rows r with (r - col - 1) % 2 == h, so it reads only
    // entries that it wrote itself
    for (int r = 1; r < TB; ++r) {  // uniform across the warp
      R a0 = R(0.0), a1 = R(0.0);
      const bool act = active_col && r > col && r < tb;
      if (act) {
        int q = col + 1 + h;
        for (; q + 2 < r; q += 4) {
          mac(a0, t[r][q], s[q][col]);
          mac(a1, t[r][q + 2], s[q + 2][col]);
        }
        if (q < r) mac(a0, t[r][q], s[q][col]);
      }
      R v = finish(a0) + finish(a1);
      v += warp_xor(v, 1);
      if (act && ((r - col - 1) & 1) == h) s[r][col] = -(t[r][col] + v);
    }
  } else {
    // inv(U), column col: x_col = 1 / U_col,col, x_r = -(sum_{q=r+1}^{col} U[r][q] x_q) / U_rr; this
    // thread sums the q with (col - q) % 2 == h and writes the rows with (col - r) % 2 == h
    if (active_col && h == 0) s[col][col] = rp[col];
    for (int r = TB - 2; r >= 0; --r) {
      R a0 = R(0.0), a1 = R(0.0);
      const bool act = active_col && r < col;
      if (act) {
        int q = col - h;
        for (; q - 2 > r; q -= 4) {
          mac(a0, t[r][q], s[q][col]);
          mac(a1, t[r][q - 2], s[q - 2][col]);
        }
        if (q > r) mac(a0, t[r][q], s[q][col]);
      }
      R v = finish(a0) + finish(a1);
      v += warp_xor(v, 1);
      if (act && ((col - r) & 1) == h) s[r][col] = -(v * rp[r]);
    }
  }
}

// ---------------------------------------------------------------------------
// batched LU without pivoting
// ---------------------------------------------------------------------------
// Four consecutive shared-memory values as vector loads (the address is 16-byte aligned: rows of the
// staged tiles are TS = 68 elements long and the column offset is a multiple of 4).
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4(const dfloat* p, dfloat (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 2);
  v[0] = dfloat(a.x, a.y); v[1] = dfloat(a.z, a.w); v[2] = dfloat(b.x, b.y); v[3] = dfloat(b.z, b.w);
}

// Tile product with register prefetch: acc(64 x 64) += A(0:64, 0:K) B(0:K, 0:64), 256 threads,
// thread (ty, tx) owns rows ty*4.. and columns tx*4..; fa(m, k) and fb(k, c) fetch operand elements
// (zero outside the operands).  The next TGK-deep slab is loaded into registers while the current
// one is multiplied from shared memory, where each k holds a row of TS elements so that a thread's
// four operands are one or two vector loads and the 16 threads of a row group read disjoint banks.
constexpr int TGK = 16;
constexpr int TS = 68;
template <class Acc, class FA, class FB>
__device__ __forceinline__ void tile_gemm(FA fa, FB fb, int K, Acc (&acc)[4][4], Acc* sA, Acc* sB) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  Acc ra[4], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * 256;
      ra[u] = fa(e / TGK, k0 + e % TGK);   // A(m, k0 + k): consecutive threads walk k
      rb[u] = fb(k0 + e / 64, e % 64);     // B(k0 + k, c): consecutive threads walk c
    }
  };
  if (K > 0) fetch(0);
  for (int k0 = 0; k0 < K; k0 += TGK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * 256;
      sA[(e % TGK) * TS + e / TGK] = ra[u];
      sB[(e / 64) * TS + e % 64] = rb[u];
    }
    __syncthreads();
    if (k0 + TGK < K) fetch(k0 + TGK);
    const int kk = min(TGK, K - k0);
#pragma unroll 8
    for (int k = 0; k < kk; ++k) {
      Acc a[4], b[4];
      load4(sA + k * TS + ty * 4, a);
      load4(sB + k * TS + tx * 4, b);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) mac(acc[u][v], a[u], b[v]);
    }
    __syncthreads();
  }
}

// Blocked right-looking LU without pivoting, one CTA per subdomain (largest first).  Each step
// factors a diagonal block of up to 64 columns in shared memory and inverts its triangles there;
// the block column below it (L21 = A21 inv(U11)), the block row to its right (U12 = inv(L11) A12)
// and the trailing matrix (A22 -= L21 U12) are then tile products.  The factors are the unique
// unpivoted L and U, whatever the blocking, so the phase split below may leave blocks that are not
// aligned to the 64-grid of the block-inverted storage (whose diagonal tiles are inverted afterwards).
// phase: -1 all columns; 0 the interior columns [0, n_I) (the trailing Schur complement on the
// overlap rows is left in place); 1 the remaining columns [n_I, n).
constexpr size_t lu_smem_elems() { return 2 * (size_t)TB * 65 + 2 * (size_t)TGK * TS; }

// TC (double-float only): the trailing update A22 -= L21 U12 runs on the tensor cores as digit-split
// BF16 products (tc_dfloat.cuh) in 128 x 64 tiles; its operand digits reuse the shared memory of the
// other steps, so one CTA runs per SM, holding all of that SM's TMEM.
template <class T, bool TC>
__global__ void __launch_bounds__(256, TC ? 1 : 2) k_lu(int N, const int* ni, const int* ld, const int64_t* foff,
                                            T* fac, int allow_last_zero, double* last_pivot,
                                            const double* dscale, int* st, const int* sched, const int* nI,
                                            int phase, const int* off, const int* pf, const int* pg, int boost) {
  using Acc = typename AccOf<T>::type;
  static_assert(!TC || std::is_same<T, dfloat>::value, "tensor-core trailing update is for double-float");
  extern __shared__ __align__(16) unsigned char lu_smem_raw[];
  __shared__ unsigned char lnz[MAXN_LOCAL / TB + 1], unz[MAXN_LOCAL / TB + 1];
  __shared__ __align__(8) uint64_t tc_bar;
  __shared__ uint32_t tc_base;
  __shared__ int tc_eA[TC ? tcdf::TM : 1], tc_eB[TC ? tcdf::TN : 1];
  __shared__ float tc_red[TC ? 4 * tcdf::TN : 1];
  tcdf::Ctx ctx{lu_smem_raw, &tc_bar, 0u, 0u, tc_eA, tc_eB};
  bool tc_fail = false;
  if constexpr (TC) {
    if (threadIdx.x == 0) tc::mbar_init(&tc_bar, 1);
    if (threadIdx.x < 32) {
      tc::tmem_alloc(&tc_base, tcdf::TMEM_COLS);
      tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    ctx.tmem = tc_base;
  }
  __shared__ Acc rdiag[TB];                       // reciprocals of the diagonal block's pivots
  Acc* Dm = reinterpret_cast<Acc*>(lu_smem_raw);  // 64 x 65: the diagonal block, factored in place
  Acc* Iv = Dm + TB * 65;                         // 64 x 65: inv(L11) strictly below, inv(U11) on/above
  Acc* sA = Iv + TB * 65;                         // TGK x TS (16-byte aligned: 2 * 64 * 65 is even)
  Acc* sB = sA + TGK * TS;                        // TGK x TS
  const int i = sched ? sched[blockIdx.x] : blockIdx.x;
  const int n = ni[i];
  const int64_t L = ld[i];
  T* A = fac + foff[i];
  const double scale = dscale[i] > 0 ? dscale[i] : 1.0;
  const double tiny = (Unit<T>::u < 1e-15 ? 1e-14 : 1e-12) * scale;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int kbeg = (phase == 1) ? nI[i] : 0;
  const int kend = (phase == 0) ? nI[i] : n;
  for (int k0 = kbeg; k0 < kend; k0 += TB) {
    const int w = min(TB, kend - k0);
    // 1. the diagonal block: LU in shared memory
    for (int e = tid; e < w * w; e += 256) Dm[(e / w) * 65 + e % w] = (Acc)A[(int64_t)(k0 + e / w) * L + k0 + e % w];
    __syncthreads();
    // Thread (ty, tx) = (tid / 64, tid % 64) owns column tx and the rows ty, ty + 4, ...; step c subtracts
    // a21 (a12 / pivot)^T from the trailing block, and the multipliers of L are formed after the loop.
    // The owner of entry (c+1, c+1) checks the next pivot right after its own update and forms its
    // reciprocal in the working arithmetic, so each step needs one barrier.
    auto pivot = [&](int c) {
      if (allow_last_zero && k0 + c == n - 1) {
        // record the last pivot of A~_ii and replace it by the scale; the eigensolver decides from it
        // whether A~_ii is singular
        last_pivot[i] = (double)Dm[c * 65 + c];
        Dm[c * 65 + c] = (Acc)scale;
      } else if (fabs((double)Dm[c * 65 + c]) <= tiny) {
        // static pivoting: counted and replaced; otherwise an error (the replacement keeps the
        // remaining steps finite until the host reads the status)
        if (boost)
          atomicAdd(st + ST_BOOSTS, 1);
        else
          raise_status(st, A2LS_ERR_SINGULAR, i, k0 + c);
        Dm[c * 65 + c] = (Acc)scale;
      }
      rdiag[c] = Acc(1.0) / Dm[c * 65 + c];
    };
    if (tid == 0) pivot(0);
    __syncthreads();
    {
      const int cx = tid & (TB - 1), ry = tid >> 6;
      for (int c = 0; c + 1 < w; ++c) {
        if (cx > c && cx < w) {
          const Acc u = Dm[c * 65 + cx] * rdiag[c];
          for (int r = c + 1 + ((ry - c - 1) & 3); r < w; r += 4) Dm[r * 65 + cx] -= Dm[r * 65 + c] * u;
          if (cx == c + 1 && ry == ((c + 1) & 3)) pivot(c + 1);
        }
        __syncthreads();
      }
    }
    for (int e = tid; e < w * w; e += 256) {
      const int r = e / w, c = e % w;
      if (r > c) Dm[r * 65 + c] *= rdiag[c];
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += 256) A[(int64_t)(k0 + e / w) * L + k0 + e % w] = (T)Dm[(e / w) * 65 + e % w];
    const int c0 = k0 + w;
    if (c0 >= n) break;
    // inverses of the triangles: inv(L11) strictly below the diagonal, inv(U11) on and above
    tile_inverses<Acc>(reinterpret_cast<const Acc(*)[TB + 1]>(Dm), reinterpret_cast<Acc(*)[TB + 1]>(Iv), rdiag, w);
    const int tiles = (n - c0 + TB - 1) / TB;
    // envelope: a row tile of L21 is nonzero only if one of its rows starts left of c0, a column tile
    // of U12 only if one of its columns starts above c0
    {
      const int lane = tid & 31, warp = tid >> 5, o = off[i];
      for (int t = warp; t < tiles; t += 8) {
        const int a0 = c0 + t * TB, a1 = min(n, a0 + TB);
        int fm = n, gm = n;
        for (int r = a0 + lane; r < a1; r += 32) {
          fm = min(fm, pf[o + r]);
          gm = min(gm, pg[o + r]);
        }
        for (int q = 16; q > 0; q >>= 1) {
          fm = min(fm, __shfl_xor_sync(0xffffffffu, fm, q));
          gm = min(gm, __shfl_xor_sync(0xffffffffu, gm, q));
        }
        if (lane == 0) {
          lnz[t] = fm < c0;
          unz[t] = gm < c0;
        }
      }
    }
    __syncthreads();
    // 2. L21 = A21 inv(U11), 64-row tiles
    for (int t = 0; t < tiles; ++t) {
      if (!lnz[t]) continue;
      const int r0 = c0 + t * TB, rows = min(TB, n - r0);
      Acc acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0;
      tile_gemm<Acc>([&](int m, int k) -> Acc { return (m < rows && k < w) ? (Acc)A[(int64_t)(r0 + m) * L + k0 + k] : (Acc)0; },
                     [&](int k, int c) -> Acc { return (k < w && c < w && c >= k) ? Iv[k * 65 + c] : (Acc)0; },
                     w, acc, sA, sB);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int r = ty * 4 + u, c = tx * 4 + v;
          if (r < rows && c < w) A[(int64_t)(r0 + r) * L + k0 + c] = (T)finish(acc[u][v]);
        }
    }
    // 3. U12 = inv(L11) A12, 64-column tiles
    for (int t = 0; t < tiles; ++t) {
      if (!unz[t]) continue;
      const int cs = c0 + t * TB, cols = min(TB, n - cs);
      Acc acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0;
      tile_gemm<Acc>([&](int m, int k) -> Acc { return (m < w && k < w) ? (k < m ? Iv[m * 65 + k] : (k == m ? (Acc)1 : (Acc)0)) : (Acc)0; },
                     [&](int k, int c) -> Acc { return (k < w && c < cols) ? (Acc)A[(int64_t)(k0 + k) * L + cs + c] : (Acc)0; },
                     w, acc, sA, sB);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int r = ty * 4 + u, c = tx * 4 + v;
          if (r < w && c < cols) A[(int64_t)(k0 + r) * L + cs + c] = (T)finish(acc[u][v]);
        }
    }
    __syncthreads();  // L21 and U12 complete before the trailing update reads them
    // 4. A22 -= L21 U12
    if constexpr (TC) {
      const int rtiles = (n - c0 + tcdf::TM - 1) / tcdf::TM;
      for (int rt = 0; rt < rtiles && !tc_fail; ++rt) {
        const int ta = 2 * rt, tb2 = 2 * rt + 1;   // the two 64-row tiles of this 128-row tile
        if (!lnz[ta] && !(tb2 < tiles && lnz[tb2])) continue;
        const int r0 = c0 + rt * tcdf::TM, rows = min(tcdf::TM, n - r0);
        tcdf::split_a(ctx, [&](int m, int k) -> dfloat {
          return (m < rows && k < w) ? (dfloat)A[(int64_t)(r0 + m) * L + k0 + k] : dfloat(0.f, 0.f);
        });
        for (int ct = 0; ct < tiles; ++ct) {
          if (!unz[ct]) continue;
          const int cs = c0 + ct * TB, cols = min(TB, n - cs);
          tcdf::split_b(ctx, [&](int k, int c) -> dfloat {
            return (k < w && c < cols) ? (dfloat)A[(int64_t)(k0 + k) * L + cs + c] : dfloat(0.f, 0.f);
          }, tc_red);
          // while the MMAs run: this tile's A22 rows (read by the epilogue) and the next column tile of
          // U12 (read by the next split) into L2
          tcdf::prefetch_rows_l2(A + (int64_t)r0 * L + cs, L * (int64_t)sizeof(T), rows, cols * (int)sizeof(T));
          {
            int nt = ct + 1;
            while (nt < tiles && !unz[nt]) ++nt;
            if (nt < tiles) {
              const int cs2 = c0 + nt * TB;
              tcdf::prefetch_rows_l2(A + (int64_t)k0 * L + cs2, L * (int64_t)sizeof(T), w,
                                     min(TB, n - cs2) * (int)sizeof(T));
            }
          }
          if (!tcdf::multiply(ctx)) {
            if (threadIdx.x == 0) raise_status(st, A2LS_ERR_TIMEOUT, i, k0);
            tc_fail = true;
            break;
          }
          tcdf::epilogue_subtract(ctx, reinterpret_cast<dfloat*>(A) + (int64_t)r0 * L + cs, L, rows, cols);
        }
      }
      __syncthreads();
      if (tc_fail) break;
    } else {
    for (int t = 0; t < tiles * tiles; ++t) {
      if (!lnz[t / tiles] || !unz[t % tiles]) continue;
      const int r0 = c0 + (t / tiles) * TB, cs = c0 + (t % tiles) * TB;
      const int rows = min(TB, n - r0), cols = min(TB, n - cs);
      Acc acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0;
      tile_gemm<Acc>([&](int m, int k) -> Acc { return (m < rows && k < w) ? (Acc)A[(int64_t)(r0 + m) * L + k0 + k] : (Acc)0; },
                     [&](int k, int c) -> Acc { return (k < w && c < cols) ? (Acc)A[(int64_t)(k0 + k) * L + cs + c] : (Acc)0; },
                     w, acc, sA, sB);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int r = ty * 4 + u, c = tx * 4 + v;
          if (r < rows && c < cols) {
            T* p = A + (int64_t)(r0 + r) * L + cs + c;
            *p = (T)((Acc)*p - acc[u][v]);
          }
        }
    }
    __syncthreads();
    }
  }
  if constexpr (TC) {
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(ctx.tmem, tcdf::TMEM_COLS);
  }
}

template <class T>
void lu_batched(a2ls_handle* h, T* fac, int allow_last_zero, double* last_pivot, double* diag_scale, int phase) {
  using Acc = typename AccOf<T>::type;
  if constexpr (std::is_same<T, dfloat>::value) {
    if (h->opt.tensor_cores) {
      const size_t smem = std::max(lu_smem_elems() * sizeof(Acc), tcdf::SMEM_BYTES);
      A2LS_CUDA(cudaFuncSetAttribute(k_lu<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_lu<T, true><<<h->N, 256, smem, h->st>>>(h->N, h->d_ni, h->d_ld, h->d_foff, fac, allow_last_zero, last_pivot,
                                                diag_scale, h->d_status, h->d_sched, h->d_nI, phase, h->d_off,
                                                h->d_pf, h->d_pg, h->opt.static_pivoting);
      A2LS_LAUNCH();
      return;
    }
  }
  const size_t smem = lu_smem_elems() * sizeof(Acc);
  A2LS_CUDA(cudaFuncSetAttribute(k_lu<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_lu<T, false><<<h->N, 256, smem, h->st>>>(h->N, h->d_ni, h->d_ld, h->d_foff, fac, allow_last_zero, last_pivot,
                                             diag_scale, h->d_status, h->d_sched, h->d_nI, phase, h->d_off, h->d_pf,
                                             h->d_pg, h->opt.static_pivoting);
  A2LS_LAUNCH();
}

// A_ii from the splitting's partial factorisation.  A~_ii differs from A_ii only on the diagonal of the
// overlap rows (Definition 3.1: A~ = A_ii - diag(s_i) there), so after the interior columns are
// eliminated both share every factor entry and their Schur complements on the overlap differ by
// diag(s_i): dst = src + diag(s_i) on the overlap block, converted to the precision of the A_ii
// factors.  When the subdomain has no overlap rows the splitting's replaced last pivot is restored.
// Only the entries inside the envelope are copied (dst is zero elsewhere): row r from its first
// envelope column pf_r, skipping the 64-column tiles of U whose columns all start below row r.
template <class TS, class TD>
__global__ void k_schur_copy(const int* ni, const int* nI, const int* ld, const int64_t* foff, const int* off,
                             const TS* __restrict__ src, TD* __restrict__ dst, const double* lump,
                             const double* last_pivot, const int* __restrict__ pf, const int* __restrict__ toff,
                             const int* __restrict__ tg) {
  const int i = blockIdx.x;
  const int n = ni[i], n_I = nI[i];
  const int64_t L = ld[i];
  const TS* S = src + foff[i];
  TD* D = dst + foff[i];
  const int* tgi = tg + toff[i];
  for (int r = blockIdx.y; r < n; r += gridDim.y) {
    const TS* Sr = S + (int64_t)r * L;
    TD* Dr = D + (int64_t)r * L;
    // off-diagonal entries convert directly (a double-float pair rounds to FP32 as hi + lo)
    for (int c = pf[off[i] + r] + threadIdx.x; c < n; c += blockDim.x)
      if (c != r && (c < r || tgi[c / TB] <= r)) Dr[c] = (TD)Sr[c];
    if (threadIdx.x == 0) {
      double v = (double)Sr[r];
      if (r >= n_I) v += lump[off[i] + r];
      if (r == n - 1 && n_I == n && last_pivot) v = last_pivot[i];
      Dr[r] = (TD)v;
    }
  }
}

template <class TS, class TD>
void schur_copy(a2ls_handle* h, const TS* src, TD* dst, const double* last_pivot) {
  dim3 grid(h->N, 32);
  k_schur_copy<TS, TD><<<grid, 256, 0, h->st>>>(h->d_ni, h->d_nI, h->d_ld, h->d_foff, h->d_off, src, dst,
                                                h->d_lump, last_pivot, h->d_pf, h->d_toff, h->d_tg);
  A2LS_LAUNCH();
}
template void schur_copy<double, double>(a2ls_handle*, const double*, double*, const double*);
template void schur_copy<double, float>(a2ls_handle*, const double*, float*, const double*);
template void schur_copy<float, double>(a2ls_handle*, const float*, double*, const double*);
template void schur_copy<float, float>(a2ls_handle*, const float*, float*, const double*);
template void schur_copy<dfloat, double>(a2ls_handle*, const dfloat*, double*, const double*);
template void schur_copy<dfloat, float>(a2ls_handle*, const dfloat*, float*, const double*);

// ---------------------------------------------------------------------------
// inversion of the diagonal tiles (in place): inv(L_bb) strictly lower, inv(U_bb) upper
// ---------------------------------------------------------------------------
// arithmetic of the tile inverses: FP64 for FP64 factors, double-float for FP32 and double-float ones
template <class T> struct InvAcc { using type = dfloat; };
template <> struct InvAcc<double> { using type = double; };

// one CTA of 256 threads per (subdomain, diagonal tile), in shared memory
template <class T>
__global__ void __launch_bounds__(4 * TB) k_invert_tiles(const int* ni, const int* ld, const int64_t* foff,
                                                         T* fac) {
  using R = typename InvAcc<T>::type;
  __shared__ R t[TB][TB + 1], s[TB][TB + 1];
  __shared__ R rp[TB];
  const int i = blockIdx.x, b = blockIdx.y;
  const int n = ni[i];
  const int r0 = b * TB;
  if (r0 >= n) return;
  const int tb = min(TB, n - r0);
  const int64_t L = ld[i];
  T* A = fac + foff[i] + (int64_t)r0 * L + r0;
  for (int e = threadIdx.x; e < tb * tb; e += blockDim.x) t[e / tb][e % tb] = R(A[(e / tb) * L + e % tb]);
  __syncthreads();
  if (threadIdx.x < tb) rp[threadIdx.x] = R(1.0) / t[threadIdx.x][threadIdx.x];
  __syncthreads();
  tile_inverses<R>(t, s, rp, tb);
  __syncthreads();
  for (int e = threadIdx.x; e < tb * tb; e += blockDim.x) A[(e / tb) * L + e % tb] = (T)s[e / tb][e % tb];
}

template <class T> void invert_diag_tiles(a2ls_handle* h, T* fac) {
  dim3 grid(h->N, ceil_div(h->max_n, TB));
  k_invert_tiles<T><<<grid, 4 * TB, 0, h->st>>>(h->d_ni, h->d_ld, h->d_foff, fac);
  A2LS_LAUNCH();
}

// ---------------------------------------------------------------------------
// single right-hand-side local solves of the apply
//   mode 0: z[g] = (q ? q[g] : 0) + x_l for interior rows l < n_I (restricted, Boolean D)
//   mode 1: yloc[off + l] = D_l * x_l for every row (combined later by memberships)
//   mode 2: yloc[off + l] = x_l (ASM: no weights)
// The gathered vector lives in shared memory; 512 threads = 16 warps.
// ---------------------------------------------------------------------------
template <class T> struct Vec;
template <> struct Vec<__nv_bfloat16> { using type = uint4; static constexpr int W = 8; };
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };

template <class T, class Acc>
__device__ __forceinline__ Acc dot_vec(const typename Vec<T>::type& a, const Acc* x);
template <>
__device__ __forceinline__ float dot_vec<float, float>(const float4& a, const float* x) {
  return a.x * x[0] + a.y * x[1] + a.z * x[2] + a.w * x[3];
}
template <>
__device__ __forceinline__ double dot_vec<double, double>(const double2& a, const double* x) {
  return a.x * x[0] + a.y * x[1];
}
// eight bfloat16 values: the high half of each 32-bit word is the upper element, the low half the lower
template <>
__device__ __forceinline__ float dot_vec<__nv_bfloat16, float>(const uint4& a, const float* x) {
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    s += __uint_as_float(w[k] << 16) * x[2 * k];
    s += __uint_as_float(w[k] & 0xffff0000u) * x[2 * k + 1];
  }
  return s;
}


// part[u] += sum_{c in [c0, c1)} M[r0 + r][c] x[c] for the rows r = wid + u * warps of a 64-row tile
// (c0 and c1 multiples of the vector width, c1 up to ld with zeros in x beyond n)
template <class T, class Acc, int THREADS>
__device__ __forceinline__ void panel_accumulate(const T* __restrict__ M, int64_t L, int r0, int tb, int c0,
                                                 int c1, const Acc* x, Acc (&part)[TB / (THREADS / 32)]) {
  constexpr int LS_WARPS = THREADS / 32;
  constexpr int ROWS_PER_WARP = TB / LS_WARPS;
  using V = typename Vec<T>::type;
  constexpr int VW = Vec<T>::W;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nv = (c1 - c0 + VW - 1) / VW;
  const V* rowp[ROWS_PER_WARP];
#pragma unroll
  for (int u = 0; u < ROWS_PER_WARP; ++u) {
    int r = wid + u * LS_WARPS;
    rowp[u] = reinterpret_cast<const V*>(M + (int64_t)(r0 + min(r, tb - 1)) * L + c0);
  }
  for (int v = lane; v < nv; v += 32) {
    V a[ROWS_PER_WARP];
#pragma unroll
    for (int u = 0; u < ROWS_PER_WARP; ++u) a[u] = __ldg(rowp[u] + v);
    const Acc* xv = x + c0 + v * VW;
#pragma unroll
    for (int u = 0; u < ROWS_PER_WARP; ++u) part[u] += dot_vec<T, Acc>(a[u], xv);
  }
}

// s[r] = x[r0 + r] - (warp sum of part) for the tile's rows
template <class Acc, int THREADS>
__device__ __forceinline__ void panel_finish(Acc (&part)[TB / (THREADS / 32)], int r0, int tb, const Acc* x,
                                             Acc* s) {
  constexpr int LS_WARPS = THREADS / 32;
  constexpr int ROWS_PER_WARP = TB / LS_WARPS;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < ROWS_PER_WARP; ++u) {
    Acc p = part[u];
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    int r = wid + u * LS_WARPS;
    if (lane == 0 && r < tb) s[r] = x[r0 + r] - p;
  }
}

// x[r0 + r] = sum_c Tinv[r][c] s[c], with the tile's unit-lower (lower=1) or upper (lower=0) part
template <class T, class Acc, int THREADS>
__device__ __forceinline__ void tile_apply(const T* __restrict__ M, int64_t L, int r0, int tb, int lower,
                                           const Acc* s, Acc* x) {
  constexpr int LS_WARPS = THREADS / 32;
  constexpr int ROWS_PER_WARP = TB / LS_WARPS;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < ROWS_PER_WARP; ++u) {
    const int r = wid + u * LS_WARPS;
    Acc p = 0;
    if (r < tb) {
      const T* row = M + (int64_t)(r0 + r) * L + r0;
      for (int c = lane; c < tb; c += 32) {
        Acc a = (Acc)row[c];
        if (lower) p += (c < r) ? a * s[c] : (c == r ? s[c] : (Acc)0);
        else p += (c >= r) ? a * s[c] : (Acc)0;
      }
    }
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    if (lane == 0 && r < tb) x[r0 + r] = p;
  }
}

// Persistent over a work queue: each CTA takes the next subdomain from `counter` in the order of
// `sched` (largest first), so uneven subdomains balance across the SMs.
template <class T, int THREADS>
__global__ void __launch_bounds__(THREADS) k_local_solve(
    const int* off, const int* nI, const int* ni, const int* ld, const int64_t* foff, const int* idx,
    const double* D, const T* __restrict__ fac, const double* __restrict__ t, const double* __restrict__ q,
    double* __restrict__ out, int mode, const int* sched, int* counter, int nwork, const int* toff, const int* tf,
    const int* tg) {
  using Acc = typename AccOf<T>::type;
  constexpr int RPW = TB / (THREADS / 32);
  constexpr int VW = Vec<T>::W;
  extern __shared__ unsigned char smem_raw[];
  Acc* x = reinterpret_cast<Acc*>(smem_raw);
  __shared__ Acc s[TB];
  __shared__ int item;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int w = item;
    __syncthreads();
    if (w >= nwork) break;
    const int i = sched[w];
    const int n = ni[i], o = off[i];
    const int64_t L = ld[i];
    const T* M = fac + foff[i];
    for (int l = threadIdx.x; l < L; l += THREADS) x[l] = (l < n) ? (Acc)t[idx[o + l]] : (Acc)0;
    __syncthreads();
    const int nb = (n + TB - 1) / TB;
    const int* tfi = tf + toff[i];
    const int* tgi = tg + toff[i];
    // forward: L y = t; L[r][c] = 0 left of the block's first envelope column
    for (int b = 0; b < nb; ++b) {
      const int r0 = b * TB, tb = min(TB, n - r0);
      Acc part[RPW];
#pragma unroll
      for (int u = 0; u < RPW; ++u) part[u] = 0;
      const int fs = (tfi[b] / VW) * VW;
      if (r0 > fs) panel_accumulate<T, Acc, THREADS>(M, L, r0, tb, fs, r0, x, part);
      panel_finish<Acc, THREADS>(part, r0, tb, x, s);
      __syncthreads();
      tile_apply<T, Acc, THREADS>(M, L, r0, tb, 1, s, x);
      __syncthreads();
    }
    // backward: U x = y; the 64-column tiles whose columns all start below the block are zero
    for (int b = nb - 1; b >= 0; --b) {
      const int r0 = b * TB, tb = min(TB, n - r0);
      Acc part[RPW];
#pragma unroll
      for (int u = 0; u < RPW; ++u) part[u] = 0;
      for (int cb = b + 1; cb < nb; ++cb) {
        if (tgi[cb] > r0 + tb - 1) continue;
        const int e0 = cb * TB, e1 = (cb == nb - 1) ? (int)L : e0 + TB;
        panel_accumulate<T, Acc, THREADS>(M, L, r0, tb, e0, e1, x, part);
      }
      panel_finish<Acc, THREADS>(part, r0, tb, x, s);
      __syncthreads();
      tile_apply<T, Acc, THREADS>(M, L, r0, tb, 0, s, x);
      __syncthreads();
    }
    if (mode == 0) {
      const int n_I = nI[i];
      for (int l = threadIdx.x; l < n_I; l += THREADS) {
        const int g = idx[o + l];
        out[g] = (q ? q[g] : 0.0) + (double)x[l];
      }
    } else {
      for (int l = threadIdx.x; l < n; l += THREADS) out[o + l] = (mode == 1 ? D[o + l] : 1.0) * (double)x[l];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Pipelined local solves: the same block triangular solves, organised so that a step's memory
// latency overlaps other work.  Each CTA (THREADS threads, persistent over the same work queue) keeps
// the gathered vector in shared memory; per 64-row block the panel product reads the factor rows
// with RU independent vector loads per row in flight before they are used, and the block's 64x64
// diagonal tile (the inverted triangles) is fetched into one of two shared buffers by asynchronous
// copies (cp.async) one block ahead, so the tile product reads shared memory only.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_but_last() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// diagonal tile of block b (rows r0 .. r0 + tb, columns r0 .. min(r0 + 64, L)) into dst (64 x 64, T)
template <class T, int THREADS>
__device__ __forceinline__ void prefetch_tile(const T* __restrict__ M, int64_t L, int r0, int tb, T* dst) {
  constexpr int PER16 = 16 / sizeof(T);                   // elements per 16-byte copy
  const int cols = (int)min((int64_t)TB, L - r0);         // a multiple of 4 elements (L and r0 are)
  const int chunks = (cols + PER16 - 1) / PER16;
  for (int e = threadIdx.x; e < tb * chunks; e += THREADS) {
    const int r = e / chunks, c = (e % chunks) * PER16;
    cp_async16(dst + r * TB + c, M + (int64_t)(r0 + r) * L + r0 + c);
  }
  cp_async_commit();
}

template <class T, int THREADS, int RU>
__global__ void __launch_bounds__(THREADS) k_local_solve2(
    const int* off, const int* nI, const int* ni, const int* ld, const int64_t* foff, const int* idx,
    const double* D, const T* __restrict__ fac, const double* __restrict__ t, const double* __restrict__ q,
    double* __restrict__ out, int mode, const int* sched, int* counter, int nwork, const int* toff, const int* tf,
    const int* tg, const int* __restrict__ pf, const int* __restrict__ pg) {
  using Acc = typename AccOf<T>::type;
  using V = typename Vec<T>::type;
  constexpr int VW = Vec<T>::W;
  constexpr int WARPS = THREADS / 32;
  constexpr int RPW = TB / WARPS;   // rows of a block per warp
  extern __shared__ __align__(16) unsigned char ls2_smem[];
  T* tile = reinterpret_cast<T*>(ls2_smem);                        // 2 x 64 x 64
  Acc* x = reinterpret_cast<Acc*>(ls2_smem + 2 * TB * TB * sizeof(T));
  __shared__ Acc s[TB];
  __shared__ int item;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int w = item;
    __syncthreads();
    if (w >= nwork) break;
    const int i = sched[w];
    const int n = ni[i], o = off[i];
    const int64_t L = ld[i];
    const T* M = fac + foff[i];
    const int nb = (n + TB - 1) / TB;
    const int* tfi = tf + toff[i];
    const int* tgi = tg + toff[i];
    prefetch_tile<T, THREADS>(M, L, 0, min(TB, n), tile);
    for (int l = threadIdx.x; l < L; l += THREADS) x[l] = (l < n) ? (Acc)t[idx[o + l]] : (Acc)0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int bb = 0; bb < nb; ++bb) {
        const int b = pass == 0 ? bb : nb - 1 - bb;
        const int r0 = b * TB, tb = min(TB, n - r0);
        const int step = pass * nb + bb;
        T* cur = tile + (step & 1) * TB * TB;
        // fetch the next step's diagonal tile (the backward sweep starts at the last block again)
        if (step + 1 < 2 * nb) {
          const int nbb = (bb + 1 < nb) ? bb + 1 : 0;
          const int npass = (bb + 1 < nb) ? pass : 1;
          const int b2 = npass == 0 ? nbb : nb - 1 - nbb;
          prefetch_tile<T, THREADS>(M, L, b2 * TB, min(TB, n - b2 * TB), tile + ((step + 1) & 1) * TB * TB);
        }
        Acc part[RPW];
#pragma unroll
        for (int u = 0; u < RPW; ++u) part[u] = 0;
        // panel columns: forward [first envelope column, r0); backward the 64-column tiles right of the
        // block that reach up to it (U's column envelope)
        // Only the factor entries inside the envelope are loaded: in the forward sweep row r of L starts at
        // its first envelope column pf[r]; in the backward sweep U[r][c] can be non-zero only if column c
        // starts at or above row r (pg[c] <= r), tested per vector of VW columns.  The other lanes skip
        // their loads (the entries there are exact zeros).
        auto panel = [&](int c0, int c1) {
          const int nv = (c1 - c0) / VW;
          const V* rowp[RPW];
          int lim[RPW];   // forward: first vector of the row; backward: the row index
#pragma unroll
          for (int u = 0; u < RPW; ++u) {
            const int r = r0 + min(wid + u * WARPS, tb - 1);
            rowp[u] = reinterpret_cast<const V*>(M + (int64_t)r * L + c0);
            lim[u] = pass == 0 ? (pf[o + r] - c0) / VW : r;
          }
          const V zero = {};
          auto vec_start = [&](int vv) -> int {   // backward: smallest first row of the vector's columns
            int g = 0x7fffffff;
            const int c = c0 + vv * VW;
#pragma unroll
            for (int q = 0; q < VW; ++q)
              if (c + q < n) g = min(g, __ldg(pg + o + c + q));
            return g;
          };
          int v = lane;
          for (; v + 32 * (RU - 1) < nv; v += 32 * RU) {
            V a[RU][RPW];
#pragma unroll
            for (int k = 0; k < RU; ++k) {
              const int vv = v + 32 * k;
              const int gs = pass == 0 ? 0 : vec_start(vv);
#pragma unroll
              for (int u = 0; u < RPW; ++u) {
                const bool in = pass == 0 ? vv >= lim[u] : gs <= lim[u];
                a[k][u] = in ? __ldg(rowp[u] + vv) : zero;
              }
            }
#pragma unroll
            for (int k = 0; k < RU; ++k) {
              const Acc* xv = x + c0 + (v + 32 * k) * VW;
#pragma unroll
              for (int u = 0; u < RPW; ++u) part[u] += dot_vec<T, Acc>(a[k][u], xv);
            }
          }
          for (; v < nv; v += 32) {
            const Acc* xv = x + c0 + v * VW;
            const int gs = pass == 0 ? 0 : vec_start(v);
#pragma unroll
            for (int u = 0; u < RPW; ++u) {
              const bool in = pass == 0 ? v >= lim[u] : gs <= lim[u];
              if (in) part[u] += dot_vec<T, Acc>(__ldg(rowp[u] + v), xv);
            }
          }
        };
        if (pass == 0) {
          const int fs = (tfi[b] / VW) * VW;
          if (r0 > fs) panel(fs, r0);
        } else {
          for (int cb = b + 1; cb < nb; ++cb) {
            if (tgi[cb] > r0 + tb - 1) continue;
            const int e0 = cb * TB, e1 = (cb == nb - 1) ? (int)L : e0 + TB;
            panel(e0, e1);
          }
        }
#pragma unroll
        for (int u = 0; u < RPW; ++u) {
          Acc p = part[u];
          for (int sh = 16; sh > 0; sh >>= 1) p += __shfl_xor_sync(0xffffffffu, p, sh);
          const int r = wid + u * WARPS;
          if (lane == 0 && r < tb) s[r] = x[r0 + r] - p;
        }
        // this step's tile has landed; the next step's (the most recent group) may still be in flight
        if (step + 1 < 2 * nb) cp_async_wait_but_last();
        else cp_async_wait_all();
        __syncthreads();
        // x[r0 + r] = sum_c Tinv[r][c] s[c] with the unit-lower (forward) or upper (backward) inverse
#pragma unroll
        for (int u = 0; u < RPW; ++u) {
          const int r = wid + u * WARPS;
          Acc p = 0;
          if (r < tb) {
            for (int c = lane; c < tb; c += 32) {
              const Acc a = (Acc)cur[r * TB + c];
              if (pass == 0) p += (c < r) ? a * s[c] : (c == r ? s[c] : (Acc)0);
              else p += (c >= r) ? a * s[c] : (Acc)0;
            }
          }
          for (int sh = 16; sh > 0; sh >>= 1) p += __shfl_xor_sync(0xffffffffu, p, sh);
          if (lane == 0 && r < tb) x[r0 + r] = p;
        }
        __syncthreads();
      }
    }
    if (mode == 0) {
      const int n_I = nI[i];
      for (int l = threadIdx.x; l < n_I; l += THREADS) {
        const int g = idx[o + l];
        out[g] = (q ? q[g] : 0.0) + (double)x[l];
      }
    } else {
      for (int l = threadIdx.x; l < n; l += THREADS) out[o + l] = (mode == 1 ? D[o + l] : 1.0) * (double)x[l];
    }
    __syncthreads();
  }
}

template <class T, int THREADS, int RU>
static void launch_local_solve2(a2ls_handle* h, const T* fac, const double* t, const double* q, double* z, int mode) {
  using Acc = typename AccOf<T>::type;
  const size_t smem = 2 * TB * TB * sizeof(T) + sizeof(Acc) * round_up(h->max_n, 8);
  int per_sm = 1, sms = 152, dev = 0;
  A2LS_CUDA(cudaGetDevice(&dev));
  static bool configured[64] = {};   // per (instantiation, device), as for the one-pass kernel
  if (dev >= 64 || !configured[dev]) {
    A2LS_CUDA(cudaFuncSetAttribute(k_local_solve2<T, THREADS, RU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(2 * TB * TB * sizeof(T) + sizeof(Acc) * MAXN_LOCAL)));
    if (dev < 64) configured[dev] = true;
  }
  A2LS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_local_solve2<T, THREADS, RU>, THREADS, smem));
  A2LS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = std::max(1, std::min(h->N, sms * std::max(per_sm, 1)));
  A2LS_CUDA(cudaMemsetAsync(h->d_counter, 0, sizeof(int), h->st));
  k_local_solve2<T, THREADS, RU><<<grid, THREADS, smem, h->st>>>(
      h->d_off, h->d_nI, h->d_ni, h->d_fld, h->d_ffoff, h->d_idx, h->d_D, fac, t, q, z, mode, h->d_sched,
      h->d_counter, h->N, h->d_toff, h->d_tf, h->d_tg, h->d_pf, h->d_pg);
  A2LS_LAUNCH();
}

template <class T, int THREADS>
static void launch_local_solve(a2ls_handle* h, const T* fac, const double* t, const double* q, double* z, int mode) {
  using Acc = typename AccOf<T>::type;
  const size_t smem = sizeof(Acc) * round_up(h->max_n, 8);
  int dev = 0;
  A2LS_CUDA(cudaGetDevice(&dev));
  // the attribute belongs to this kernel instantiation on this device: set once per (instantiation, device)
  static bool configured[64] = {};
  if (dev >= 64 || !configured[dev]) {
    A2LS_CUDA(cudaFuncSetAttribute(k_local_solve<T, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(Acc) * MAXN_LOCAL)));
    if (dev < 64) configured[dev] = true;
  }
  int per_sm = 1, sms = 152;
  A2LS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_local_solve<T, THREADS>, THREADS, smem));
  A2LS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = std::max(1, std::min(h->N, sms * std::max(per_sm, 1)));
  A2LS_CUDA(cudaMemsetAsync(h->d_counter, 0, sizeof(int), h->st));
  k_local_solve<T, THREADS><<<grid, THREADS, smem, h->st>>>(h->d_off, h->d_nI, h->d_ni, h->d_fld, h->d_ffoff, h->d_idx,
                                                            h->d_D, fac, t, q, z, mode, h->d_sched, h->d_counter,
                                                            h->N, h->d_toff, h->d_tf, h->d_tg);
  A2LS_LAUNCH();
}

// configurations of the local solves the autotuner chooses from: 256 / 512 / 1024 = the one-pass kernel
// with that CTA width; 1256 / 1512 / 2256 = the pipelined kernel with 256 or 512 threads and two
// (1xxx) or four (2xxx) vector loads per row in flight; 3000 / 3004 / 3008 = the streaming kernel on
// the packed factors (FP32 and BF16 factors) with 8 consumer warps and one CTA per SM / 4 consumer
// warps and two CTAs per SM / 8 consumer warps and two CTAs per SM
template <class T>
static void launch_local_solve_width(a2ls_handle* h, int width, const T* fac, const double* t, const double* q,
                                     double* z, int mode) {
  switch (width) {
    case 256: launch_local_solve<T, 256>(h, fac, t, q, z, mode); break;
    case 1024: launch_local_solve<T, 1024>(h, fac, t, q, z, mode); break;
    case 1256: launch_local_solve2<T, 256, 2>(h, fac, t, q, z, mode); break;
    case 1512: launch_local_solve2<T, 512, 2>(h, fac, t, q, z, mode); break;
    case 2256: launch_local_solve2<T, 256, 4>(h, fac, t, q, z, mode); break;
    case LS_STREAM:
    case LS_STREAM2:
    case LS_STREAM3:
      if constexpr (!std::is_same<T, double>::value) {
        launch_local_solve_stream<T>(h, width, t, q, z, mode);
        break;
      }
      [[fallthrough]];
    default: launch_local_solve<T, 512>(h, fac, t, q, z, mode); break;
  }
}

template <class T>
void local_solves(a2ls_handle* h, const T* fac, const double* t, const double* q, double* z, int mode) {
  // algorithmic bytes: the factor entries inside the envelope (L's rows, U's columns, diagonal once),
  // the gather of t and the scatter of the solution
  double bytes = 0.0;
  if (h->opt.timing)
    for (int i = 0; i < h->N; ++i)
      bytes += (h->h_env[4 * i + 2] + h->h_env[4 * i + 3] - h->h_n[i]) * sizeof(T) + 12.0 * h->h_n[i] +
               (mode == 0 ? 20.0 * h->h_nI[i] : 12.0 * h->h_n[i]);
  KTime kt(h, KT_APPLY_LOCAL, bytes);
  launch_local_solve_width<T>(h, h->ls_width > 0 ? h->ls_width : 512, fac, t, q, z, mode);
}

// Autotuner: time the three CTA widths on the handle's own factors (inputs t, outputs scratch) and
// keep the fastest; results are cached per (precision, subdomain count, largest subdomain, mode)
// in the process and, when A2LS_AUTOTUNE_CACHE names a file, in that JSON file.
template <class T>
void autotune_local_solves(a2ls_handle* h, const T* fac, const double* t, double* scratch, int mode) {
  char key[128];
  snprintf(key, sizeof(key), "local_solve3_%s_N%d_max%d_mode%d",
           sizeof(T) == 8 ? "fp64" : (sizeof(T) == 4 ? "fp32" : "bf16"), h->N, h->max_n, mode);
  int cached = autotune_lookup(key);
  if (cached > 0 && (cached != LS_STREAM || h->ss.shape[0].ready) && (cached != LS_STREAM2 || h->ss.shape[1].ready) &&
      (cached != LS_STREAM3 || h->ss.shape[2].ready)) {
    h->ls_width = cached;
    return;
  }
  std::vector<int> widths = {256, 512, 1024, 1256, 1512, 2256};
  if (!std::is_same<T, double>::value) {
    if (h->ss.shape[0].ready) widths.push_back(LS_STREAM);
    if (h->ss.shape[1].ready) widths.push_back(LS_STREAM2);
    if (h->ss.shape[2].ready) widths.push_back(LS_STREAM3);
  }
  float best_ms = 1e30f;
  int best = 512;
  cudaEvent_t e0, e1;
  A2LS_CUDA(cudaEventCreate(&e0));
  A2LS_CUDA(cudaEventCreate(&e1));
  for (int w : widths) {
    launch_local_solve_width<T>(h, w, fac, t, nullptr, scratch, mode);  // warm-up
    A2LS_CUDA(cudaEventRecord(e0, h->st));
    for (int rep = 0; rep < 3; ++rep) launch_local_solve_width<T>(h, w, fac, t, nullptr, scratch, mode);
    A2LS_CUDA(cudaEventRecord(e1, h->st));
    A2LS_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    A2LS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = w;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->ls_width = best;
  autotune_store(key, best);
}

// ---------------------------------------------------------------------------
// multi right-hand-side solves for the eigensolver: X (n_i x p, row-major, leading
// dimension ldx, subdomain i at X + i*xstride) <- inv(U) inv(L) X (either half optional)
// ---------------------------------------------------------------------------
// One CTA per (subdomain, chunk of 8 right-hand sides): blockIdx.y selects the chunk, so that the
// FP64-bound solves of the eigen iteration spread over all SMs.
template <class T>
__global__ void __launch_bounds__(256) k_block_solve(const int* ni, const int* ld, const int64_t* foff,
                                                     const T* __restrict__ fac, T* X,
                                                     const int64_t* xoff, int col0, int ldx,
                                                     const int* pvec, const int* active, int forward,
                                                     int backward, const int* sched, const int* toff,
                                                     const int* tf, const int* tg, int skip_p_le) {
  using Acc = typename AccOf<T>::type;
  __shared__ Acc sA[GK * 65], sB[GK * 9];
  const int i = sched ? sched[blockIdx.x] : blockIdx.x;  // largest subdomains first
  if (active && !active[i]) return;
  const int p = pvec[i];
  if (p <= skip_p_le) return;
  const int c0 = blockIdx.y * 8;
  if (c0 >= p) return;
  const int pc = min(8, p - c0);
  const int n = ni[i];
  const int64_t L = ld[i];
  const T* M = fac + foff[i];
  T* Xi = X + xoff[i] + col0 + c0;
  const int tid = threadIdx.x, tx = tid & 3, ty = tid >> 2;
  const int nb = (n + TB - 1) / TB;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 0 && !forward) continue;
    if (pass == 1 && !backward) continue;
    for (int bb = 0; bb < nb; ++bb) {
      const int b = pass == 0 ? bb : nb - 1 - bb;
      const int r0 = b * TB, tb = min(TB, n - r0);
      Acc acc[2] = {};
      if (pass == 0) {
        // L[r][c] = 0 left of the block's first envelope column
        const int fs = tf[toff[i] + b];
        if (r0 > fs)
          cta_gemm_n8<T, Acc>(M + (int64_t)r0 * L + fs, L, Xi + (int64_t)fs * ldx, ldx, tb, pc, r0 - fs, 0, acc, sA,
                              sB);
      } else {
        // U[r][c] = 0 above column c's first envelope row: skip the 64-column tiles that start below
        for (int cb = b + 1; cb < nb; ++cb) {
          if (tg[toff[i] + cb] > r0 + tb - 1) continue;
          const int e0 = cb * TB;
          cta_gemm_n8<T, Acc>(M + (int64_t)r0 * L + e0, L, Xi + (int64_t)e0 * ldx, ldx, tb, pc, min(TB, n - e0), 0,
                              acc, sA, sB);
        }
      }
      // S = X_b - acc, written in place
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int c = tx * 2 + v;
        if (ty < tb && c < pc) {
          T* ptr = Xi + (int64_t)(r0 + ty) * ldx + c;
          *ptr = (T)((Acc)*ptr - acc[v]);
        }
      }
      __syncthreads();
      Acc acc2[2] = {};
      cta_gemm_n8<T, Acc>(M + (int64_t)r0 * L + r0, L, Xi + (int64_t)r0 * ldx, ldx, tb, pc, tb, pass == 0 ? 1 : 2,
                          acc2, sA, sB);
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int c = tx * 2 + v;
        if (ty < tb && c < pc) Xi[(int64_t)(r0 + ty) * ldx + c] = (T)finish(acc2[v]);
      }
      __syncthreads();
    }
  }
}

template <class T>
void block_solve(a2ls_handle* h, const T* fac, T* X, const int64_t* xoff, int col0, int ldx, const int* pvec,
                 int pmax, const int* active, int forward, int backward, int skip_p_le) {
  if (pmax <= skip_p_le) return;
  dim3 grid(h->N, (std::max(pmax, 1) + 7) / 8);
  k_block_solve<T><<<grid, 256, 0, h->st>>>(h->d_ni, h->d_ld, h->d_foff, fac, X, xoff, col0, ldx, pvec, active,
                                           forward, backward, h->d_sched, h->d_toff, h->d_tf, h->d_tg, skip_p_le);
  A2LS_LAUNCH();
}

template void lu_batched<float>(a2ls_handle*, float*, int, double*, double*, int);
template void lu_batched<double>(a2ls_handle*, double*, int, double*, double*, int);
template void invert_diag_tiles<float>(a2ls_handle*, float*);
template void invert_diag_tiles<double>(a2ls_handle*, double*);
template void local_solves<float>(a2ls_handle*, const float*, const double*, const double*, double*, int);
template void local_solves<__nv_bfloat16>(a2ls_handle*, const __nv_bfloat16*, const double*, const double*, double*,
                                          int);
template void autotune_local_solves<__nv_bfloat16>(a2ls_handle*, const __nv_bfloat16*, const double*, double*, int);
template void local_solves<double>(a2ls_handle*, const double*, const double*, const double*, double*, int);
template void autotune_local_solves<float>(a2ls_handle*, const float*, const double*, double*, int);
template void autotune_local_solves<double>(a2ls_handle*, const double*, const double*, double*, int);
template void block_solve<float>(a2ls_handle*, const float*, float*, const int64_t*, int, int, const int*, int,
                                  const int*, int, int, int);
template void block_solve<double>(a2ls_handle*, const double*, double*, const int64_t*, int, int, const int*, int,
                                   const int*, int, int, int);
template void lu_batched<dfloat>(a2ls_handle*, dfloat*, int, double*, double*, int);
template void invert_diag_tiles<dfloat>(a2ls_handle*, dfloat*);
template void block_solve<dfloat>(a2ls_handle*, const dfloat*, dfloat*, const int64_t*, int, int, const int*, int,
                                   const int*, int, int, int);

}  // namespace a2ls

namespace a2ls {

// ---------------------------------------------------------------------------
// One dense matrix (the coarse operator A_00): block-inverted LU without
// pivoting, spread over many CTAs, then the explicit inverse.
// ---------------------------------------------------------------------------
// Factor the 64x64 diagonal block at (k0, k0) and invert its triangles in place, in the arithmetic
// and storage R (FP64, or double-float in the mixed form).  256 threads.
// LU: thread (ty, tx) = (tid / 64, tid % 64) owns column tx and the rows ty, ty + 4, ...; step c
// subtracts a21 (a12 / pivot)^T from the trailing block, so that the multipliers of column c are
// formed only once, after the loop (l_rc = a_rc / pivot_c).  The owner of entry (c+1, c+1) checks the
// next pivot right after its own update, so each step needs one barrier.
// Inverses: tile_inverses (two threads per column).
template <class R>
__device__ __forceinline__ R e_recip(R x) { return R(1.0) / x; }

template <class R>
__global__ void __launch_bounds__(256) k_e_diag(R* A, int n, int64_t ld, int k0, double scale, int* st) {
  __shared__ R t[TB][TB + 1], s[TB][TB + 1];
  __shared__ R rp[TB];
  const int tb = min(TB, n - k0);
  R* D = A + (int64_t)k0 * ld + k0;
  const int tid = threadIdx.x;
  for (int e = tid; e < tb * tb; e += blockDim.x) t[e / tb][e % tb] = D[(e / tb) * ld + e % tb];
  __syncthreads();
  auto pivot = [&](int c) {
    R piv = t[c][c];
    if (fabs((double)piv) <= 1e-14 * scale) {
      raise_status(st, A2LS_ERR_SINGULAR, -1, k0 + c);
      piv = R(scale);
      t[c][c] = piv;
    }
    rp[c] = e_recip(piv);
  };
  if (tid == 0) pivot(0);
  __syncthreads();
  const int tx = tid & (TB - 1), ty = tid >> 6;
  for (int c = 0; c + 1 < tb; ++c) {
    if (tx > c && tx < tb) {
      const R u = t[c][tx] * rp[c];
      for (int r = c + 1 + ((ty - c - 1) & 3); r < tb; r += 4) t[r][tx] -= t[r][c] * u;
      if (tx == c + 1 && ty == ((c + 1) & 3)) pivot(c + 1);
    }
    __syncthreads();
  }
  // multipliers of L
  for (int e = tid; e < tb * tb; e += blockDim.x) {
    const int r = e / tb, c = e % tb;
    if (r > c) t[r][c] *= rp[c];
  }
  __syncthreads();
  tile_inverses<R>(t, s, rp, tb);
  __syncthreads();
  for (int e = tid; e < tb * tb; e += blockDim.x) {
    const int r = e / tb, c = e % tb;
    D[r * ld + c] = s[r][c];
  }
}

// One step of the coarse LU outside the diagonal block, in pieces small enough to spread over the
// SMs, in the arithmetic R of the factorisation:
//   MODE 0: L21 = A21 inv(U11), a 16-row piece per CTA (rows of A21 are independent);
//   MODE 1: U12 = inv(L11) A12, a 16-column piece per CTA (columns of A12 are independent);
//   MODE 2: A22 -= L21 U12, a 16 x 64 piece per CTA.
// The operands of a piece are staged in shared memory before it is overwritten; each thread forms
// four outputs with independent accumulators.
template <int MODE, class R>
__global__ void __launch_bounds__(256) k_e_update(R* A, int n, int64_t ld, int k0, int span) {
  constexpr int PR = (MODE == 1) ? TB : 16;
  constexpr int PC = (MODE == 1) ? 16 : TB;
  __shared__ R sa[PR][TB + 1], sb[TB][PC + 1];
  const int tb = min(TB, n - k0);
  const int first = k0 + tb;
  int r0, c0;
  if (MODE == 0) { r0 = first + blockIdx.x * 16; c0 = k0; }
  else if (MODE == 1) { r0 = k0; c0 = first + blockIdx.x * 16; }
  else { r0 = first + blockIdx.y * 16; c0 = first + blockIdx.x * TB; }
  const int end = min(n, first + span);
  if (r0 >= (MODE == 1 ? n : end) || c0 >= (MODE == 0 ? n : end)) return;
  const int rows = (MODE == 1) ? tb : min(PR, end - r0);
  const int cols = (MODE == 0) ? tb : min(PC, end - c0);
  const R* Dg = A + (int64_t)k0 * ld + k0;
  const R zero(0.0), one(1.0);
  // A operand: MODE 0 the rows of A21, MODE 1 unit-lower inv(L11), MODE 2 the rows of L21
  for (int e = threadIdx.x; e < PR * TB; e += blockDim.x) {
    const int r = e / TB, q = e % TB;
    R v = zero;
    if (r < rows && q < tb) {
      if (MODE == 1) v = (q < r) ? Dg[(int64_t)r * ld + q] : (q == r ? one : zero);
      else v = A[(int64_t)(r0 + r) * ld + k0 + q];
    }
    sa[r][q] = v;
  }
  // B operand: MODE 0 upper inv(U11), MODE 1 the columns of A12, MODE 2 the columns of U12
  for (int e = threadIdx.x; e < TB * PC; e += blockDim.x) {
    const int q = e / PC, c = e % PC;
    R v = zero;
    if (q < tb && c < cols) {
      if (MODE == 0) v = (c >= q) ? Dg[(int64_t)q * ld + c] : zero;
      else v = A[(int64_t)(k0 + q) * ld + c0 + c];
    }
    sb[q][c] = v;
  }
  __syncthreads();
  static_assert(PR * PC == 4 * 256, "four outputs per thread");
  R acc[4] = {zero, zero, zero, zero};
#pragma unroll 4
  for (int q = 0; q < TB; ++q)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = threadIdx.x + 256 * j;
      mac(acc[j], sa[o / PC][q], sb[q][o % PC]);
    }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int o = threadIdx.x + 256 * j;
    const int r = o / PC, c = o % PC;
    if (r < rows && c < cols) {
      R* dst = (MODE == 1) ? A + (int64_t)(k0 + r) * ld + c0 + c : A + (int64_t)(r0 + r) * ld + c0 + c;
      if (MODE == 2) *dst = *dst - finish(acc[j]);
      else *dst = finish(acc[j]);
    }
  }
}

// X = inv(U) inv(L) I, one 8-column slab per CTA (F holds the block-inverted LU), all in the
// arithmetic and storage R of the factorisation.  Narrow slabs give n/8 CTAs: each CTA's sweep over
// the row blocks is a chain of dependent tile products, so more and shorter chains fill the SMs.
constexpr int EINV_W = 8;
template <class R>
__global__ void __launch_bounds__(256) k_e_inverse(const R* F, int n, int64_t ld, R* X, int64_t ldx, int band) {
  __shared__ R sA[GK * 65], sB[GK * 9];
  const int c0 = blockIdx.x * EINV_W;
  const int pc = min(EINV_W, n - c0);
  const int tid = threadIdx.x, tx = tid & 3, ty = tid >> 2;
  R* Xs = X + c0;
  for (int e = tid; e < n * pc; e += 256) {
    const int r = e / pc, c = e % pc;
    Xs[(int64_t)r * ldx + c] = (r == c0 + c) ? R(1.0) : R(0.0);
  }
  __syncthreads();
  const int nb = (n + TB - 1) / TB;
  const int bstart = c0 / TB;  // rows above the slab's first unit entry stay zero in the forward pass
  for (int pass = 0; pass < 2; ++pass) {
    for (int bb = 0; bb < nb; ++bb) {
      const int b = pass == 0 ? bb : nb - 1 - bb;
      if (pass == 0 && b < bstart) continue;
      const int r0 = b * TB, tb = min(TB, n - r0);
      R acc[2] = {R(0.0), R(0.0)};
      if (pass == 0) {
        const int k0 = max(bstart * TB, r0 - band);  // L(r, c) = 0 for c < r - band
        if (r0 > k0)
          cta_gemm_n8<R, R>(F + (int64_t)r0 * ld + k0, ld, Xs + (int64_t)k0 * ldx, ldx, tb, pc, r0 - k0, 0, acc, sA,
                            sB);
      } else {
        const int e0 = r0 + tb;
        const int e1 = min(n, r0 + tb + band);       // U(r, c) = 0 for c > r + band
        if (e0 < e1)
          cta_gemm_n8<R, R>(F + (int64_t)r0 * ld + e0, ld, Xs + (int64_t)e0 * ldx, ldx, tb, pc, e1 - e0, 0, acc, sA,
                            sB);
      }
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int c = tx * 2 + v;
        if (ty < tb && c < pc) {
          R* x = Xs + (int64_t)(r0 + ty) * ldx + c;
          *x = *x - finish(acc[v]);
        }
      }
      __syncthreads();
      R acc2[2] = {R(0.0), R(0.0)};
      cta_gemm_n8<R, R>(F + (int64_t)r0 * ld + r0, ld, Xs + (int64_t)r0 * ldx, ldx, tb, pc, tb, pass == 0 ? 1 : 2,
                        acc2, sA, sB);
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int c = tx * 2 + v;
        if (ty < tb && c < pc) Xs[(int64_t)(r0 + ty) * ldx + c] = finish(acc2[v]);
      }
      __syncthreads();
    }
  }
}

// in-place conversions between an FP64 array and its double-float image (same 8-byte slots)
__global__ void k_to_dfloat_inplace(int64_t count, double* p) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const dfloat v(p[e]);
    reinterpret_cast<dfloat*>(p)[e] = v;
  }
}
__global__ void k_to_double_inplace(int64_t count, double* p) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)reinterpret_cast<const dfloat*>(p)[e];
    p[e] = v;
  }
}

template <class R>
static void dense_inverse_t(a2ls_handle* h, R* E, int n, double scale, R* Einv, int band) {
  cudaStream_t st = h->st;
  const int64_t ld = n;
  // algorithmic work of a banded LU without pivoting (bandwidth band) and of the inverse formed from
  // its factors: forward substitution of the identity with L, backward substitution of the dense
  // result with U
  double lu_flops = 0.0, inv_flops = 0.0;
  for (int k = 0; k < n; ++k) {
    const double l = std::min(band, n - 1 - k);
    lu_flops += l + 2.0 * l * l;
    const double d = n - 1 - k, dw = std::min<double>(d, band);
    inv_flops += dw * (dw + 1.0) + 2.0 * std::max(0.0, d - band) * band;  // column k of inv(L)
    inv_flops += (double)n * (2.0 * l + 1.0);                              // row k of the U solve
  }
  {
    KTime kt(h, KT_COARSE_LU, lu_flops);
    for (int k0 = 0; k0 < n; k0 += TB) {
      k_e_diag<R><<<1, 256, 0, st>>>(E, n, ld, k0, scale, h->d_status);
      A2LS_LAUNCH();
      // entries farther than the bandwidth from the diagonal are zero and stay zero
      const int rest = min(n - k0 - min(TB, n - k0), band + TB);
      if (rest <= 0) break;
      const int p16 = ceil_div(rest, 16);
      k_e_update<0, R><<<p16, 256, 0, st>>>(E, n, ld, k0, rest);
      A2LS_LAUNCH();
      k_e_update<1, R><<<p16, 256, 0, st>>>(E, n, ld, k0, rest);
      A2LS_LAUNCH();
      k_e_update<2, R><<<dim3(ceil_div(rest, TB), p16), 256, 0, st>>>(E, n, ld, k0, rest);
      A2LS_LAUNCH();
    }
  }
  KTime kt2(h, KT_COARSE_INV, inv_flops);
  k_e_inverse<R><<<ceil_div(n, EINV_W), 256, 0, st>>>(E, n, ld, Einv, ld, band);
  A2LS_LAUNCH();
}

// The coarse operator E (FP64, n x n, overwritten) factored and inverted into Einv (FP64).  The
// mixed form runs the factorisation and the inverse in double-float arithmetic on double-float
// images of E and Einv held in the same buffers.
void dense_inverse(a2ls_handle* h, double* E, int n, double scale, double* Einv, int band) {
  if (band <= 0 || band >= n) band = n;
  const int64_t nn = (int64_t)n * n;
  const int grid = (int)std::min<int64_t>(152 * 8, (nn + 255) / 256 + 1);
  if (h->opt.precision != A2LS_FP64) {
    k_to_dfloat_inplace<<<grid, 256, 0, h->st>>>(nn, E);
    A2LS_LAUNCH();
    dense_inverse_t<dfloat>(h, reinterpret_cast<dfloat*>(E), n, scale, reinterpret_cast<dfloat*>(Einv), band);
    k_to_double_inplace<<<grid, 256, 0, h->st>>>(nn, Einv);
    A2LS_LAUNCH();
  } else {
    dense_inverse_t<double>(h, E, n, scale, Einv, band);
  }
}

// row r of subdomain blockIdx.x: FP32 (leading dimension ld) to bfloat16 (leading dimension ld2 >= ld,
// padding zero)
__global__ void k_to_bf16(const int* ni, const int* ld, const int64_t* foff, const int* ld2, const int64_t* foff2,
                          const float* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  const int i = blockIdx.x;
  const int n = ni[i], L = ld[i], L2 = ld2[i];
  const float* s = src + foff[i];
  __nv_bfloat16* d = dst + foff2[i];
  for (int r = blockIdx.y; r < n; r += gridDim.y)
    for (int c = threadIdx.x; c < L2; c += blockDim.x)
      d[(int64_t)r * L2 + c] = __float2bfloat16_rn(c < L ? s[(int64_t)r * L + c] : 0.f);
}

__nv_bfloat16* factors_to_bf16(a2ls_handle* h, const float* src) {
  const int N = h->N;
  h->h_fld.assign(N, 0);
  h->h_ffoff.assign(N + 1, 0);
  for (int i = 0; i < N; ++i) {
    h->h_fld[i] = (int)round_up(h->h_n[i], 8);
    h->h_ffoff[i + 1] = h->h_ffoff[i] + (int64_t)h->h_fld[i] * h->h_n[i];
  }
  h->d_fld = dalloc<int>(h, N);
  h->d_ffoff = dalloc<int64_t>(h, N + 1);
  A2LS_CUDA(cudaMemcpyAsync(h->d_fld, h->h_fld.data(), sizeof(int) * N, cudaMemcpyHostToDevice, h->st));
  A2LS_CUDA(cudaMemcpyAsync(h->d_ffoff, h->h_ffoff.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice,
                            h->st));
  __nv_bfloat16* dst = dalloc<__nv_bfloat16>(h, (size_t)h->h_ffoff[N]);
  k_to_bf16<<<dim3(N, 64), 256, 0, h->st>>>(h->d_ni, h->d_ld, h->d_foff, h->d_fld, h->d_ffoff, src, dst);
  A2LS_LAUNCH();
  return dst;
}

void local_solves_any(a2ls_handle* h, const double* t, const double* q, double* z, int mode) {
  if (h->opt.precision == A2LS_FP64) local_solves<double>(h, static_cast<const double*>(h->d_fac), t, q, z, mode);
  else if (h->opt.precision == A2LS_BF16)
    local_solves<__nv_bfloat16>(h, static_cast<const __nv_bfloat16*>(h->d_fac), t, q, z, mode);
  else local_solves<float>(h, static_cast<const float*>(h->d_fac), t, q, z, mode);
}

}  // namespace a2ls

// Setup, part 3: the local generalized eigenproblems of Eq. 3.1 and the
// coarse-space selection of Eq. 3.2, batched over all subdomains.
//
// For subdomain i: B = D_i A_ii D_i, C = A~_ii (Definition 3.1).
//  * K_i = ker(C).  C is factored without pivoting (C = L U); for the
//    diagonally dominant splittings of the target problems dim K_i <= 1 and a
//    null direction shows up as a vanishing last pivot u_nn.  With the last
//    pivot replaced by sigma (U'), k = sigma inv(U') e_n satisfies C k = u_nn e_n,
//    so |u_nn| / ||k|| bounds the smallest singular value; C counts as singular
//    when it is at most n * eps * ||C||_inf.
//  * Kernel part of Eq. 3.2: (L_i cap K_i)^{perp K_i} = span(k) unless B k = 0.
//  * Finite part: eigenpairs of B u = lambda C u restricted to u orthogonal to K_i,
//    i.e. of T = (V_R^T C V_R)^{-1} V_R^T B V_R (Pi_i = orthogonal projector onto
//    K_i^perp).  T u is computed without forming V_R: f = B u, g = inv(L) f,
//    g <- g - (g_n / h_n) h with h = inv(L) k (makes the right-hand side consistent),
//    v = inv(U') g, u' = v - (k^T v) k.
//  * The largest |lambda| are found by a block Krylov method with explicit
//    restarts: s block-Arnoldi steps (block Gram-Schmidt twice, Cholesky QR
//    twice) build V = [V_0 .. V_s]; the Rayleigh-Ritz matrix is the block
//    Hessenberg H; its eigenpairs (dense Hessenberg QR, one warp per
//    subdomain) give Ritz pairs whose residual is ||H_{s,s-1} y_last||; the
//    next cycle restarts from the real basis of the leading Ritz vectors.
//    Small subdomains (n_i - dim K_i <= capacity) are solved in the full space.
//  * Selection: |lambda| descending, kernel part first; a conjugate pair cut
//    by the count keeps both members; a pair contributes [Re u, Im u].
#include "a2ls_internal.cuh"
#include "small_eig.cuh"

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>

namespace a2ls {

namespace se {
template <> struct SeEps<dfloat> {
  static constexpr double v = 1.4210854715202004e-14;  // 2^-46
  static constexpr double big = 1e30;                  // within FP32's exponent range
};
template <> struct SeEarlyReflector<dfloat> { static constexpr bool value = false; };
}  // namespace se

template <class T> struct EAcc;
template <> struct EAcc<float> { using type = float; };
template <> struct EAcc<double> { using type = double; };
template <> struct EAcc<dfloat> { using type = dfloat; };
// smallest Gram pivot kept finite: FP32 and double-float share FP32's exponent range
template <class T> struct Tiny { static constexpr double v = 1e-300; };
template <> struct Tiny<float> { static constexpr double v = 1e-30; };
template <> struct Tiny<dfloat> { static constexpr double v = 1e-30; };

constexpr int EIG_THREADS = 256;
constexpr int EIG_MAXP = 96;   // column capacity of the Krylov basis
constexpr int VY_RC = 32;      // rows staged per chunk in k_vy (32 rows x 8 column triples: a thread each)

__device__ __forceinline__ double hash_uniform(uint64_t seed, uint64_t a, uint64_t b, uint64_t c) {
  // splitmix64 of a counter built from (seed, a, b, c); uniform in (-1, 1)
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (a * 0x100000001B3ull + b * 0xC2B2AE3D27D4EB4Full + c + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
  __syncthreads();
  return t;
}

// X[n-1] = sigma in a zero-initialised column (input of k' = sigma inv(U') e_n)
template <class T>
__global__ void k_unit_last(const int* ni, const int64_t* xoff, const double* dscale, T* X) {
  const int i = blockIdx.x;
  if (threadIdx.x == 0) X[xoff[i] + ni[i] - 1] = (T)(dscale[i] > 0 ? dscale[i] : 1.0);
}

// Decide dim ker(A~_ii) and the kernel part of Eq. 3.2; restore U when A~_ii is non-singular.
//  * Exactly singular: A~_ii is an M-matrix splitting for the target problems (non-positive
//    couplings, weak diagonal dominance by Definition 3.1); an irreducible weakly diagonally
//    dominant matrix is singular exactly when every row is tight, and then its kernel is spanned
//    by the vector of ones.  Tested on the FP64 CSR data: every row sum within 32 eps of its
//    absolute row sum.
//  * Numerically singular in the working precision: the last pivot of the unpivoted LU is at most
//    n eps_work sigma (sigma = largest |diagonal|).  The kernel direction is then the factorisation's
//    own null vector k' = sigma inv(U') e_n, for which A~_ii k' = u_nn e_n.
//  * Otherwise non-singular: the replaced last pivot is undone.
template <class T>
__global__ void __launch_bounds__(EIG_THREADS) k_kernel_test(
    const int* ni, const int* off, const int* ld, const int64_t* foff, T* fac, const double* last_pivot,
    const double* dscale, const int64_t* lrow, const int* lcol, const double* lval, const double* lump,
    const double* D, const int64_t* xoff, const T* X, double eps_work, double* kvec, int* kd, int* kpart,
    int* st) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  const int n = ni[i], o = off[i];
  double worst = 0.0, bmax = 0.0, k2 = 0.0;
  const T* kp = X + xoff[i];
  for (int l = threadIdx.x; l < n; l += EIG_THREADS) {
    double rs = 0.0, ra = 0.0, rb = 0.0;
    for (int64_t q = lrow[o + l]; q < lrow[o + l + 1]; ++q) {
      const int lk = lcol[q];
      if (lk < 0) continue;
      double a = lval[q];
      rb += fabs(a) * D[o + lk];
      if (lk == l) a -= lump[o + l];
      rs += a;
      ra += fabs(a);
    }
    worst = fmax(worst, fabs(rs) / fmax(ra, 1e-300));
    bmax = fmax(bmax, rb * D[o + l]);
    const double v = (double)kp[l];
    k2 += v * v;
  }
  worst = block_max(worst, red);
  const double bnorm = block_max(bmax, red);
  const double knorm = sqrt(block_sum(k2, red));
  const double sigma = dscale[i] > 0 ? dscale[i] : 1.0;
  const double upiv = last_pivot[i];
  const bool exact = worst <= 32.0 * 2.220446049250313e-16;
  const bool numerical = !exact && fabs(upiv) <= (double)n * eps_work * sigma;
  if (threadIdx.x == 0) kd[i] = (exact || numerical) ? 1 : 0;
  if (!exact && !numerical) {
    // undo the pivot replacement: the last column of the last diagonal tile of inv(U) scales by sigma/u_nn
    const int r0 = ((n - 1) / TB) * TB;
    T* A = fac + foff[i];
    const int64_t L = ld[i];
    for (int r = r0 + threadIdx.x; r < n; r += EIG_THREADS) {
      T* p = A + (int64_t)r * L + (n - 1);
      *p = (T)((double)*p * (sigma / upiv));
    }
    for (int l = threadIdx.x; l < n; l += EIG_THREADS) kvec[o + l] = 0.0;
    if (threadIdx.x == 0) kpart[i] = 0;
    return;
  }
  if (numerical && !(knorm > 0.0 && isfinite(knorm))) {
    if (threadIdx.x == 0) raise_status(st, A2LS_ERR_EIGEN, i, 3);
    return;
  }
  const double kv = 1.0 / sqrt((double)n);
  for (int l = threadIdx.x; l < n; l += EIG_THREADS) kvec[o + l] = exact ? kv : (double)kp[l] / knorm;
  __syncthreads();
  // kernel part test: B k != 0, i.e. k is not in L_i = ker(D A_ii D)
  double bk = 0.0, kinf = 0.0;
  for (int l = threadIdx.x; l < n; l += EIG_THREADS) {
    double r = 0.0;
    for (int64_t q = lrow[o + l]; q < lrow[o + l + 1]; ++q) {
      const int lk = lcol[q];
      if (lk >= 0) r += lval[q] * D[o + lk] * kvec[o + lk];
    }
    bk = fmax(bk, fabs(r * D[o + l]));
    kinf = fmax(kinf, fabs(kvec[o + l]));
  }
  bk = block_max(bk, red);
  kinf = block_max(kinf, red);
  if (threadIdx.x == 0) kpart[i] = (bk > (double)n * 1e-14 * bnorm * kinf) ? 1 : 0;
}

// X[:, col0] = kvec (as T) for the kernel subdomains
template <class T>
__global__ void k_load_vec(const int* ni, const int* off, const int64_t* xoff, int ldx, const double* v,
                           const int* mask, T* X) {
  const int i = blockIdx.x;
  if (mask && !mask[i]) return;
  for (int l = threadIdx.x; l < ni[i]; l += blockDim.x) X[xoff[i] + (int64_t)l * ldx] = (T)v[off[i] + l];
}

template <class T>
__global__ void k_store_h(const int* ni, const int* off, const int64_t* xoff, int ldx, const T* X,
                          const int* kd, double* h, int* st) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  if (!kd[i]) return;
  const int n = ni[i];
  double s2 = 0.0;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    const double v = (double)X[xoff[i] + (int64_t)l * ldx];
    h[off[i] + l] = v;
    s2 += v * v;
  }
  const double hn = sqrt(block_sum(s2, red));
  if (threadIdx.x == 0) {
    // the consistency shift divides by h_n; it vanishes only if the right null vector lies in range(C)
    if (!(fabs(h[off[i] + n - 1]) > 1e-12 * hn)) raise_status(st, A2LS_ERR_EIGEN, i, 1);
  }
}

// random start block, columns [col0, col0 + p_i)
template <class T>
__global__ void k_random_block(const int* ni, const int64_t* xoff, int ldx, int col0, const int* pvec,
                               const int* active, uint64_t seed, int cycle, T* X) {
  const int i = blockIdx.x;
  if (active && !active[i]) return;
  const int n = ni[i], p = pvec[i];
  for (int e = threadIdx.x; e < n * p; e += blockDim.x) {
    const int l = e / p, c = e % p;
    X[xoff[i] + (int64_t)l * ldx + col0 + c] = (T)hash_uniform(seed, (uint64_t)i, (uint64_t)l,
                                                               (uint64_t)(c + 1000 * cycle));
  }
}

// warm start: columns c < 16 are the network's proposal Y scaled to unit norm plus a 1e-3 random
// perturbation (keeps the block full rank where the proposal is not); further columns and subdomains
// solved in the full space are random
constexpr int WARM_COLS = 16;
template <class T>
__global__ void k_warm_block(const int* ni, const int* off, const int64_t* xoff, int ldx, const int* pvec,
                             const int* active, const int* full, const float* Y, uint64_t seed, T* X) {
  __shared__ double nrm[WARM_COLS];
  const int i = blockIdx.x;
  if (active && !active[i]) return;
  const int n = ni[i], p = pvec[i], o = off[i];
  const bool use = !full[i];
  if (threadIdx.x < WARM_COLS) nrm[threadIdx.x] = 0.0;
  __syncthreads();
  if (use) {
    // column norms: 16 threads per row
    const int c = threadIdx.x & (WARM_COLS - 1);
    double a = 0.0;
    for (int l = threadIdx.x / WARM_COLS; l < n; l += blockDim.x / WARM_COLS) {
      const double v = Y[(int64_t)(o + l) * WARM_COLS + c];
      a += v * v;
    }
    atomicAdd(&nrm[c], a);
  }
  __syncthreads();
  const double pert = 1e-3 / sqrt((double)n);
  for (int e = threadIdx.x; e < n * p; e += blockDim.x) {
    const int l = e / p, c = e % p;
    const double u = hash_uniform(seed, (uint64_t)i, (uint64_t)l, (uint64_t)c);
    double v = u;
    if (use && c < WARM_COLS) {
      const double s = nrm[c] > 0.0 ? 1.0 / sqrt(nrm[c]) : 0.0;
      v = Y[(int64_t)(o + l) * WARM_COLS + c] * s + pert * u;
    }
    X[xoff[i] + (int64_t)l * ldx + c] = (T)v;
  }
}

// columns of X orthogonal to k (kernel subdomains only)
template <class T>
__global__ void __launch_bounds__(EIG_THREADS) k_project_k(const int* ni, const int* off, const int64_t* xoff,
                                                            int ldx, int col0, const int* pvec,
                                                            const int* active, const int* kd,
                                                            const typename EAcc<T>::type* kvec, T* X) {
  using Acc = typename EAcc<T>::type;
  __shared__ Acc dots[EIG_MAXP];
  const int i = blockIdx.x;
  if ((active && !active[i]) || !kd[i]) return;
  const int n = ni[i], p = pvec[i], o = off[i];
  T* Xi = X + xoff[i] + col0;
  for (int c = threadIdx.x; c < p; c += EIG_THREADS) dots[c] = 0;
  __syncthreads();
  // one warp per column
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = wid; c < p; c += EIG_THREADS / 32) {
    Acc d = 0;
    for (int l = lane; l < n; l += 32) mac(d, kvec[o + l], (Acc)Xi[(int64_t)l * ldx + c]);
    d = finish(d);
    for (int w = 16; w > 0; w >>= 1) d += warp_xor(d, w);
    if (lane == 0) dots[c] = d;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * p; e += EIG_THREADS) {
    const int l = e / p, c = e % p;
    Xi[(int64_t)l * ldx + c] = (T)((Acc)Xi[(int64_t)l * ldx + c] - dots[c] * kvec[o + l]);
  }
}

// W[:, 0:p] = B V[:, c0:c0+p], B = D A_ii D via the local CSR; one warp per row
// lval and D in the working arithmetic of the eigensolve (converted once per setup)
template <class T>
__global__ void k_convert(int64_t count, const double* __restrict__ in, T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)in[e];
}

template <class TV, class T>
__global__ void k_bmul(const int* ni, const int* off, const int64_t* xoff, int ldx, int vcol0, const int* pvec,
                       const int* active, const int64_t* lrow, const int* lcol,
                       const typename EAcc<T>::type* lval, const typename EAcc<T>::type* D, const TV* V, T* W) {
  using Acc = typename EAcc<T>::type;
  const int i = blockIdx.x;
  if (active && !active[i]) return;
  const int n = ni[i], p = pvec[i], o = off[i];
  const TV* Vi = V + xoff[i] + vcol0;
  T* Wi = W + xoff[i];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // rows spread over the gridDim.y CTAs of the subdomain and their warps
  for (int l = blockIdx.y * nw + wid; l < n; l += nw * gridDim.y) {
    const Acc dl = D[o + l];
    for (int c0 = 0; c0 < p; c0 += 32) {
      const int c = c0 + lane;
      Acc acc = 0;
      if (dl != Acc(0) && c < p) {
        for (int64_t q = lrow[o + l]; q < lrow[o + l + 1]; ++q) {
          const int lk = lcol[q];
          if (lk < 0) continue;
          const Acc dk = D[o + lk];
          if (dk == Acc(0)) continue;
          mac(acc, lval[q] * dk, (Acc)Vi[(int64_t)lk * ldx + c]);
        }
      }
      if (c < p) Wi[(int64_t)l * ldx + c] = (T)(finish(acc) * dl);
    }
  }
}

// W[:, c] -= (W[n-1][c] / h[n-1]) h  (consistency of the right-hand side with range(C))
template <class T>
__global__ void k_mu_fix(const int* ni, const int* off, const int64_t* xoff, int ldx, const int* pvec,
                         const int* active, const int* kd, const double* h, T* W) {
  using Acc = typename EAcc<T>::type;
  __shared__ Acc mu[EIG_MAXP];
  const int i = blockIdx.x;
  if ((active && !active[i]) || !kd[i]) return;
  const int n = ni[i], p = pvec[i], o = off[i];
  T* Wi = W + xoff[i];
  const double hn = h[o + n - 1];
  for (int c = threadIdx.x; c < p; c += blockDim.x) mu[c] = (Acc)((double)Wi[(int64_t)(n - 1) * ldx + c] / hn);
  __syncthreads();
  for (int e = threadIdx.x; e < n * p; e += blockDim.x) {
    const int l = e / p, c = e % p;
    Wi[(int64_t)l * ldx + c] = (T)((Acc)Wi[(int64_t)l * ldx + c] - mu[c] * (Acc)h[o + l]);
  }
}

// ---------------------------------------------------------------------------
// Orthogonalisation (k_orth and its helpers): block CGS2 of W against the basis, then Cholesky QR.
// ---------------------------------------------------------------------------

constexpr int ORTH_THREADS = 512;
constexpr int ORC_MAX = 64;              // rows staged per chunk in k_orth (64, or 32 with full-space Gram)
// row stride of the staged chunks: even, so that column pairs are 16-byte aligned for vector loads;
// 98 x 8 bytes puts consecutive rows 4 banks apart
constexpr int SROW = EIG_MAXP + 2;
constexpr int GRAM_NG_MAX = 16;          // row groups (split-K) of a Gram product

// stage rows [l0, l0 + rows) of M (cols 0:w) into S (stride SROW), zero padding to a multiple of 4
template <class Acc, class TM>
__device__ __forceinline__ void stage_rows(Acc* S, const TM* M, int64_t ldx, int l0, int rows, int w) {
  const int wp = (w + 3) & ~3;
  for (int e = threadIdx.x; e < rows * wp; e += ORTH_THREADS) {
    const int r = e / wp, c = e % wp;
    S[r * SROW + c] = c < w ? (Acc)M[(int64_t)(l0 + r) * ldx + c] : (Acc)0;
  }
}

// two consecutive staged values with one vector load (p is aligned to twice the element size)
__device__ __forceinline__ void ld2(const double* p, double& a, double& b) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ld2(const dfloat* p, dfloat& a, dfloat& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = dfloat(v.x, v.y);
  b = dfloat(v.z, v.w);
}
__device__ __forceinline__ void ld2(const float* p, float& a, float& b) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  a = v.x;
  b = v.y;
}

// Gram product G (nx x ny, row-major, stride ny) = X^T Y over the n rows of X and Y (global, leading
// dimension ldx).  Each item is a 4 x 2 output block; with fewer blocks than threads the rows are
// split into ng groups (split-K) whose partial sums are added at the end.  same (X == Y, nx == ny):
// only the blocks that reach the upper triangle are formed, the lower triangle is mirrored.
// Xs, Ys: staging chunks; Ps: scratch of ORTH_THREADS x 8 values for the partial sums (may alias
// the staging chunks).  Ends with a barrier.
template <class Acc, class TX, class TY>
__device__ void gram_product(const TX* X, const TY* Y, int64_t ldx, int n, int nx, int ny, bool same, Acc* Xs,
                             Acc* Ys, double* G, Acc* Ps, int orc) {
  const int tid = threadIdx.x;
  const int nbr = (nx + 3) / 4, nbc = (ny + 1) / 2;
  // block (br, bc) covers rows 4br..4br+3 and columns 2bc..2bc+1; with X == Y only bc >= 2br
  auto row_blocks = [&](int br) { return same ? max(0, nbc - 2 * br) : nbc; };
  int nb = 0;
  for (int br = 0; br < nbr; ++br) nb += row_blocks(br);
  auto block_of = [&](int b, int& a0, int& c0) {
    int br = 0;
    while (b >= row_blocks(br)) b -= row_blocks(br++);
    a0 = 4 * br;
    c0 = 2 * (nbc - row_blocks(br) + b);
  };
  const int ng = nb >= ORTH_THREADS ? 1 : min(GRAM_NG_MAX, ORTH_THREADS / nb);
  const int items = nb * ng;
  // more blocks than threads (full-space Gram of a small subdomain): several passes over the rows
  for (int w0 = 0; w0 < items; w0 += ORTH_THREADS) {
    const int w = w0 + tid;
    const bool valid = w < items;
    int a0 = 0, c0 = 0, g = 0;
    if (valid) {
      block_of(w % nb, a0, c0);
      g = w / nb;
    }
    Acc acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0;
    for (int l0 = 0; l0 < n; l0 += orc) {
      const int rows = min(orc, n - l0);
      stage_rows(Xs, X, ldx, l0, rows, nx);
      if (!same) stage_rows(Ys, Y, ldx, l0, rows, ny);
      __syncthreads();
      const Acc* Yr = same ? Xs : Ys;
      if (valid) {
        Acc s[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) s[q] = 0;
        for (int r = g; r < rows; r += ng) {
          Acc x[4], y[2];
          ld2(Xs + r * SROW + a0, x[0], x[1]);
          ld2(Xs + r * SROW + a0 + 2, x[2], x[3]);
          ld2(Yr + r * SROW + c0, y[0], y[1]);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            mac(s[2 * u], x[u], y[0]);
            mac(s[2 * u + 1], x[u], y[1]);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] += finish(s[q]);
      }
      __syncthreads();
    }
    if (ng == 1) {
      if (valid)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int a = a0 + (q >> 1), c = c0 + (q & 1);
          if (a < nx && c < ny && (!same || c >= a)) G[a * ny + c] = (double)acc[q];
        }
    } else {  // items <= ORTH_THREADS: a single pass
      if (valid)
#pragma unroll
        for (int q = 0; q < 8; ++q) Ps[tid * 8 + q] = acc[q];
      __syncthreads();
      if (tid < nb) {
        block_of(tid, a0, c0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          Acc sum = Ps[tid * 8 + q];
          for (int gg = 1; gg < ng; ++gg) sum += Ps[(gg * nb + tid) * 8 + q];
          const int a = a0 + (q >> 1), c = c0 + (q & 1);
          if (a < nx && c < ny && (!same || c >= a)) G[a * ny + c] = (double)sum;
        }
      }
    }
    __syncthreads();
  }
  if (same) {
    for (int e = tid; e < nx * nx; e += ORTH_THREADS) {
      const int a = e / nx, c = e % nx;
      if (c < a) G[a * nx + c] = G[c * nx + a];
    }
    __syncthreads();
  }
}

// One warp: G (p x p, stride p, upper triangle read) = R^T R by Cholesky, R into G's upper triangle,
// Ri = inv(R) (stride p).  The factorisation runs on the diagonally scaled Gram matrix
// Gs = D^-1 G D^-1, D = sqrt(diag G) (1 for a column at or below abs_floor), so that the pivot tests
// see the conditioning of W's normalised columns and not the spread of their norms (the residual
// columns of nearly converged Ritz vectors are orders of magnitude shorter than the others);
// R = Rs D and inv(R) = D^-1 inv(Rs).  shift_u > 0: Gs + shift_u tr(Gs) I (shifted Cholesky QR).
// A pivot at or below rel_floor of the largest diagonal entry of Gs (or abs_floor) marks a
// rank-deficient block: rel_floor is the squared unit roundoff of the arithmetic that formed G (at
// least 1e-28), below which a pivot is rounding noise.  The pivot is floored and the rest of its row
// of Rs set to zero, so that inv(R) amplifies that noise to O(1) at most, a zero column stays zero,
// and no later pivot inherits the floored one's growth; W = W inv(R) R still holds, and the next
// Cholesky QR pass restores the orthogonality.  Returns 1 when no pivot was floored (valid on every
// lane).  dsc: p doubles of scratch.  min_ratio (optional): the smallest squared pivot over the
// largest diagonal entry of Gs, a lower bound of 1 / cond(W D^-1)^2.
__device__ int warp_cholesky_inverse(double* G, int p, double* Ri, double* dsc, double abs_floor,
                                     double rel_floor, double shift_u = 0.0, double* min_ratio = nullptr) {
  const int lane = threadIdx.x & 31;
  for (int a = lane; a < p; a += 32) {
    const double g = G[a * p + a];
    dsc[a] = g > abs_floor ? sqrt(g) : 1.0;
  }
  __syncwarp();
  for (int e = lane; e < p * p; e += 32) {
    const int a = e / p, c = e % p;
    if (c >= a) G[e] = G[e] / dsc[a] / dsc[c];
  }
  __syncwarp();
  double tr = 0.0;
  for (int a = lane; a < p; a += 32) tr += G[a * p + a];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if (shift_u > 0.0) {
    for (int a = lane; a < p; a += 32) G[a * p + a] += shift_u * tr;
    __syncwarp();
  }
  double gm = 0.0;
  for (int a = lane; a < p; a += 32) gm = fmax(gm, G[a * p + a]);
  for (int o = 16; o > 0; o >>= 1) gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
  const double floor_d = fmax(rel_floor * gm, abs_floor);
  int ok = 1;
  double dmin = INFINITY;
  for (int a = 0; a < p; ++a) {
    double part = 0.0;
    for (int q = lane; q < a; q += 32) part += G[q * p + a] * G[q * p + a];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    double d = G[a * p + a] - part;
    dmin = fmin(dmin, d);
    const bool floored = !(d > floor_d);
    if (floored) {
      ok = 0;
      d = floor_d;
    }
    const double r = sqrt(d);
    for (int c = a + 1 + lane; c < p; c += 32) {
      double v = 0.0;
      if (!floored) {
        v = G[a * p + c];
        for (int q = 0; q < a; ++q) v -= G[q * p + a] * G[q * p + c];
        v /= r;
      }
      G[a * p + c] = v;
    }
    __syncwarp();
    if (lane == 0) G[a * p + a] = r;
    __syncwarp();
  }
  for (int c = lane; c < p; c += 32) {
    for (int a = c + 1; a < p; ++a) Ri[a * p + c] = 0.0;
    Ri[c * p + c] = 1.0 / G[c * p + c];
    for (int a = c - 1; a >= 0; --a) {
      double v = 0.0;
      for (int q = a + 1; q <= c; ++q) v += G[a * p + q] * Ri[q * p + c];
      Ri[a * p + c] = -v / G[a * p + a];
    }
  }
  __syncwarp();
  // back to the unscaled factors: R = Rs D, inv(R) = D^-1 inv(Rs)
  for (int e = lane; e < p * p; e += 32) {
    const int a = e / p, c = e % p;
    if (c >= a) {
      G[e] *= dsc[c];
      Ri[e] /= dsc[a];
    }
  }
  __syncwarp();
  if (min_ratio) *min_ratio = gm > 0.0 ? dmin / gm : 0.0;
  return ok;
}

// Orthogonalisation: block CGS2 of W against V[:, 0:jb], then Cholesky QR three times (the first
// shifted).  Writes the Gram coefficients into H[0:jb, hc:hc+p] and R into H[hr:hr+p, hc:hc+p] and
// the orthonormal block into V[:, vout:vout+p].  full != 0: only H[0:jb, hc:hc+p].  illcond (if given):
// set to 1 for a subdomain whose block needed the shifted factorisation (an ill-conditioned block).
// Shared memory: G and Ri (gcap doubles each), trow, two staging chunks of orc x EIG_MAXP.
template <class T, class TW>
__global__ void __launch_bounds__(ORTH_THREADS) k_orth(const int* ni, const int64_t* xoff, int ldx,
                                                        const int* pvec, const int* active, int jb_blocks,
                                                        int bcols, T* V, TW* W, double* H, int hr, int hc,
                                                        int vout, const int* fullv, int* rank_flag, int gcap,
                                                        int orc, int* illcond, int* status) {
  using Acc = typename EAcc<T>::type;
  extern __shared__ __align__(16) double sm[];
  const int i = blockIdx.x;
  if (active && !active[i]) return;
  const int full = fullv ? fullv[i] : 0;
  if (full && jb_blocks != 1) return;
  const int n = ni[i], p = pvec[i];
  const int jb = full ? p : jb_blocks * bcols;  // basis columns to orthogonalise against
  if (p * p > gcap || jb * p > gcap) {          // the Gram matrices would not fit the launch's space
    if (threadIdx.x == 0) raise_status(status, A2LS_ERR_EIGEN, i, 3);
    return;
  }
  T* Vi = V + xoff[i];
  TW* Wi = W + xoff[i];
  double* Hi = H + (int64_t)i * EIG_MAXP * EIG_MAXP;
  double* G = sm;                               // gcap: Gram, then R in place
  double* Ri = G + gcap;                        // gcap
  double* trow = Ri + gcap;                     // EIG_MAXP: column scales of the Cholesky
  Acc* sv = reinterpret_cast<Acc*>(trow + EIG_MAXP);           // orc * SROW
  Acc* sw = sv + orc * SROW;                                   // orc * SROW
  __shared__ int rank_ok;
  const int tid = threadIdx.x;
  // the updates W -= V G and W <- W inv(R): each thread forms one row of a group of 3 columns (with
  // 64-row chunks and p = 24 that is exactly one item per thread); coefficients padded to pp columns
  const int ncg = (p + 2) / 3, pp = 3 * ncg;
  const int npass = jb > 0 ? 2 : 0;
  for (int e = tid; e < jb * p; e += ORTH_THREADS) Hi[(e / p) * EIG_MAXP + hc + e % p] = 0.0;
  for (int pass = 0; pass < npass; ++pass) {
    // G = V[:, 0:jb]^T W[:, 0:p]
    gram_product<Acc>(Vi, Wi, (int64_t)ldx, n, jb, p, false, sv, sw, G, sv, orc);
    for (int e = tid; e < jb * p; e += ORTH_THREADS) Hi[(e / p) * EIG_MAXP + hc + e % p] += G[e];
    if (full) return;  // Rayleigh quotient only
    // W -= V G; G converted once to the working arithmetic (in Ri's space, padded to pp columns)
    Acc* Ga = reinterpret_cast<Acc*>(Ri);
    for (int e = tid; e < jb * pp; e += ORTH_THREADS) {
      const int a = e / pp, c = e % pp;
      Ga[e] = c < p ? (Acc)G[a * p + c] : (Acc)0;
    }
    __syncthreads();
    for (int l0 = 0; l0 < n; l0 += orc) {
      const int rows = min(orc, n - l0);
      stage_rows(sv, Vi, ldx, l0, rows, jb);
      __syncthreads();
      for (int e = tid; e < rows * ncg; e += ORTH_THREADS) {
        const int r = e / ncg, c = 3 * (e % ncg);
        Acc s0 = 0, s1 = 0, s2 = 0;
        for (int a = 0; a < jb; ++a) {
          const Acc v = sv[r * SROW + a];
          mac(s0, v, Ga[a * pp + c]);
          mac(s1, v, Ga[a * pp + c + 1]);
          mac(s2, v, Ga[a * pp + c + 2]);
        }
        TW* w = Wi + (int64_t)(l0 + r) * ldx + c;
        w[0] = (TW)((Acc)w[0] - s0);
        if (c + 1 < p) w[1] = (TW)((Acc)w[1] - s1);
        if (c + 2 < p) w[2] = (TW)((Acc)w[2] - s2);
      }
      __syncthreads();
    }
  }
  // Cholesky QR: a plain first pass, kept when its diagonally scaled Gram matrix is well conditioned
  // (smallest squared pivot above plain_ratio of the largest diagonal entry, i.e. cond of W's
  // normalised columns below about 1e4 in double-float and FP64), followed by one more plain pass
  // (Cholesky QR2); otherwise that factor is discarded and shifted Cholesky QR3 runs (a shifted first
  // pass keeps the factorisation defined for nearly rank-deficient blocks, two plain passes restore
  // orthogonality).
  // R_total = R_last ... R_1 goes to H[hr:hr+p, hc:hc+p]
  const double plain_ratio = fmax(1e-8, 1e3 * Unit<Acc>::u);
  __shared__ int retry_shifted;
  bool shifted = false;
  int passes = 2;
  for (int pass = 0; pass < passes; ++pass) {
    gram_product<Acc>(Wi, Wi, (int64_t)ldx, n, p, p, true, sw, sw, G, sv, orc);
    if (tid < 32) {
      // shifted pass: Gs + 11 (n p + p (p + 1)) u tr(Gs) I
      const double shift_u =
          (pass == 0 && shifted) ? 11.0 * ((double)n * p + (double)p * (p + 1)) * Unit<Acc>::u : 0.0;
      double ratio = 0.0;
      const int ok = warp_cholesky_inverse(G, p, Ri, trow, Tiny<Acc>::v, fmax(1e-28, Unit<Acc>::u * Unit<Acc>::u),
                                           shift_u, &ratio);
      if (tid == 0) {
        retry_shifted = (pass == 0 && !shifted && !(ok && ratio > plain_ratio)) ? 1 : 0;
        rank_ok = ok;
        if (!ok && !retry_shifted && rank_flag) atomicAdd(rank_flag + i, 1);
        if (retry_shifted && illcond) illcond[i] = 1;
      }
    }
    __syncthreads();
    if (retry_shifted) {  // uniform across the CTA
      shifted = true;
      passes = 3;
      pass = -1;
      continue;
    }
    if (pass == 0) {
      for (int e = tid; e < p * p; e += ORTH_THREADS) {
        const int a = e / p, c = e % p;
        Hi[(hr + a) * EIG_MAXP + hc + c] = (c >= a) ? G[a * p + c] : 0.0;
      }
    } else if ((size_t)p * p * sizeof(double) <= (size_t)orc * SROW * sizeof(Acc)) {
      // H_blk <- R H_blk (R upper triangular), through a temporary in the staging space
      double* tmp = reinterpret_cast<double*>(sw);
      for (int e = tid; e < p * p; e += ORTH_THREADS) {
        const int a = e / p, c = e % p;
        double s = 0.0;
        for (int q = a; q < p; ++q) s += G[a * p + q] * Hi[(hr + q) * EIG_MAXP + hc + c];
        tmp[e] = s;
      }
      __syncthreads();
      for (int e = tid; e < p * p; e += ORTH_THREADS) Hi[(hr + e / p) * EIG_MAXP + hc + e % p] = tmp[e];
    } else {
      // a block too wide for the staging space (a full-space subdomain): in place, row by row from
      // the top (row a of the product reads rows a .. p - 1, not yet overwritten)
      for (int a = 0; a < p; ++a) {
        double s = 0.0;
        if (tid < p)
          for (int q = a; q < p; ++q) s += G[a * p + q] * Hi[(hr + q) * EIG_MAXP + hc + tid];
        __syncthreads();
        if (tid < p) Hi[(hr + a) * EIG_MAXP + hc + tid] = s;
        __syncthreads();
      }
    }
    __syncthreads();
    // W <- W inv(R); inv(R) converted once to the working arithmetic (in G's space, padded to pp columns)
    Acc* Ra = reinterpret_cast<Acc*>(G);
    for (int e = tid; e < p * pp; e += ORTH_THREADS) {
      const int a = e / pp, c = e % pp;
      Ra[e] = c < p ? (Acc)Ri[a * p + c] : (Acc)0;
    }
    __syncthreads();
    for (int l0 = 0; l0 < n; l0 += orc) {
      const int rows = min(orc, n - l0);
      stage_rows(sw, Wi, ldx, l0, rows, p);
      __syncthreads();
      for (int e = tid; e < rows * ncg; e += ORTH_THREADS) {
        const int r = e / ncg, c = 3 * (e % ncg);
        Acc s0 = 0, s1 = 0, s2 = 0;
        for (int a = 0; a <= c + 2 && a < p; ++a) {
          const Acc v = sw[r * SROW + a];
          mac(s0, v, Ra[a * pp + c]);
          mac(s1, v, Ra[a * pp + c + 1]);
          mac(s2, v, Ra[a * pp + c + 2]);
        }
        TW* w = Wi + (int64_t)(l0 + r) * ldx + c;
        w[0] = (TW)finish(s0);
        if (c + 1 < p) w[1] = (TW)finish(s1);
        if (c + 2 < p) w[2] = (TW)finish(s2);
      }
      __syncthreads();
    }
  }
  // V[:, vout:vout+p] = W
  if (vout >= 0)
    for (int e = tid; e < n * p; e += ORTH_THREADS) {
      const int l = e / p, c = e % p;
      Vi[(int64_t)l * ldx + vout + c] = (T)Wi[(int64_t)l * ldx + c];
    }
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz on H (one CTA per subdomain): Ritz values, the real basis Y of
// the leading Ritz vectors (bcols columns), residual norms and convergence.
// ---------------------------------------------------------------------------
// Threads per subdomain of the Rayleigh-Ritz kernel (measured on the 512x512 high-contrast problem:
// 32 and 256 threads were both slower than 128)
constexpr int RR_THREADS = 128;

// arithmetic of the Rayleigh-Ritz step: FP64, or double-float when the eigensolve runs in double-float
template <class T> struct RRType { using type = double; };
template <> struct RRType<dfloat> { using type = dfloat; };

struct RRParams {
  int sb_krylov;   // s*b in Krylov mode
  int b;           // block size
  int s;           // block steps
  double tol;
  int nevmax;      // slots per subdomain in the eigenvalue export
  double tau;      // > 0: keep only |lambda| > 1 / tau (Eq. 3.2), at most nev
  double thick_spread;  // > 0: a thick restart is allowed while |theta_1| <= thick_spread |theta_b|
};

template <class R>
__global__ void k_rayleigh_ritz(RRParams prm, const int* full, const int* mfull, const int* nf,
                                const int* active, const double* H, double* Y, int* ycols, int* zcols,
                                double* eigout, int* conv, double* worst, int* illcond, int* thick, int* st) {
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  if (active && !active[i]) return;
  if (threadIdx.x == 0) thick[i] = 0;
  if (nf[i] <= 0) {
    if (threadIdx.x == 0) {
      conv[i] = 1;
      worst[i] = 0.0;
      ycols[i] = 0;
      zcols[i] = 0;
    }
    return;
  }
  const int m = full[i] ? mfull[i] : prm.sb_krylov;
  const int ld = m + 1;
  // sized for the launch's largest m and block size b (two CTAs per SM fit for m = 72, b = 24)
  R* S = reinterpret_cast<R*>(sm);   // m x ld
  R* Q = S + m * ld;                 // m x ld (an odd row stride keeps the row-wise column updates
                                     // of Q off a single shared-memory bank pair)
  R* xs = Q + m * ld;                // b lanes x m
  R* ys = xs + prm.b * m;            // b lanes x m
  R* vtmp = ys + prm.b * m;          // m (Hessenberg scratch, then the moduli)
  double* mod = reinterpret_cast<double*>(vtmp);
  double* wr = reinterpret_cast<double*>(vtmp + m);  // m
  double* wi = wr + m;               // m
  int* perm = reinterpret_cast<int*>(wi + m);  // m
  const double* Hi = H + (int64_t)i * EIG_MAXP * EIG_MAXP;
  const se::Team team{(int)threadIdx.x, (int)blockDim.x};
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    S[(e / m) * ld + e % m] = (R)Hi[(e / m) * EIG_MAXP + e % m];
    Q[(e / m) * ld + e % m] = (R)((e / m == e % m) ? 1.0 : 0.0);
  }
  __syncthreads();
  // largest |H| entry and finiteness, reduced over the CTA
  __shared__ double red_norm[RR_THREADS / 32];
  __shared__ int red_fin[RR_THREADS / 32];
  double snorm = 0.0;
  int fin = 1;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const double v = Hi[(e / m) * EIG_MAXP + e % m];
    fin &= isfinite(v) ? 1 : 0;
    snorm = fmax(snorm, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) {
    snorm = fmax(snorm, __shfl_xor_sync(0xffffffffu, snorm, o));
    fin &= __shfl_xor_sync(0xffffffffu, fin, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red_norm[threadIdx.x >> 5] = snorm;
    red_fin[threadIdx.x >> 5] = fin;
  }
  __syncthreads();
  for (int w = 0; w < (int)blockDim.x / 32; ++w) {
    snorm = fmax(snorm, red_norm[w]);
    fin &= red_fin[w];
  }
  const bool finite = fin != 0;
  if (!finite) {
    if (threadIdx.x == 0) {
      raise_status(st, A2LS_ERR_EIGEN, i, 4);
      conv[i] = 1;
      ycols[i] = 0;
      zcols[i] = 0;
    }
    return;
  }
  se::hessenberg(S, ld, Q, ld, m, vtmp, team);
  __shared__ R snap[14];
  // the Ritz pairs are wanted to a relative residual of prm.tol: a subdiagonal entry below 1e-3 tol of
  // its diagonal neighbours is already far below what the residual test resolves
  const int rc = se::schur(S, ld, Q, ld, m, snorm, team, snap, 1e-3 * prm.tol);
  if (rc != 0 && threadIdx.x == 0) raise_status(st, A2LS_ERR_EIGEN, i, 2);
  __syncthreads();
  if (threadIdx.x == 0) {
    se::schur_eigenvalues(S, ld, m, wr, wi);
    se::order_by_modulus(wr, wi, m, perm, mod);
  }
  __syncthreads();
  // plan the columns: walk eigenvalues by modulus, pairs take two columns
  // lane j handles the j-th selected eigenvalue
  __shared__ int sel_pos[32], sel_col[32], sel_two[32], nsel_s, ncol_s, zc_s;
  if (threadIdx.x == 0) {
    const int bc = full[i] ? min(prm.b, m) : prm.b;
    int col = 0, nsel = 0, cnt = 0, zc = -1;
    for (int a = 0; a < m && col < bc && nsel < 32; ++a) {
      const int pidx = perm[a];
      if (wi[pidx] < 0.0) continue;  // the partner of a pair already taken
      const int two = (wi[pidx] > 0.0) ? 1 : 0;
      // threshold selection (Eq. 3.2): the wanted set ends before the first |lambda| <= 1/tau; the
      // rest of the block is still filled, it carries the restart
      if (prm.tau > 0.0 && zc < 0 && !(mod[pidx] * prm.tau > 1.0)) zc = col;
      sel_pos[nsel] = pidx;
      sel_col[nsel] = col;
      sel_two[nsel] = (two && col + 1 < bc) ? 1 : (two ? 2 : 0);  // 2: pair truncated to its real part
      col += (sel_two[nsel] == 1) ? 2 : 1;
      cnt += two ? 2 : 1;
      ++nsel;
      if (zc < 0 && cnt >= nf[i]) zc = col;
    }
    if (zc < 0) zc = col;
    nsel_s = nsel;
    ncol_s = col;
    zc_s = zc;
    // thick restart (Krylov mode): the Arnoldi relation it carries over holds to about u |theta_1|
    // (absolute); it is used while that stays far below the kept Ritz values' tolerance and no block of
    // this cycle was ill-conditioned, otherwise the next restart is explicit
    const bool spread_ok = nsel > 0 && mod[perm[0]] <= prm.thick_spread * mod[sel_pos[nsel - 1]];
    thick[i] = (!full[i] && col == bc && spread_ok && !illcond[i]) ? 1 : 0;
    illcond[i] = 0;
  }
  __syncthreads();
  const int nsel = nsel_s;
  double* Yi = Y + (int64_t)i * EIG_MAXP * EIG_MAXP;
  int conv_all = 1;
  __shared__ unsigned long long worst_bits;   // largest res / |lambda| of the wanted pairs (>= 0)
  if (threadIdx.x == 0) worst_bits = 0ull;
  // Schur vectors: one selected eigenvalue per thread (a pair's +imag member is the first of its block)
  if ((int)threadIdx.x < nsel) {
    const int j = threadIdx.x;
    const int pidx = sel_pos[j];
    se::schur_vector(S, ld, m, pidx, wr[pidx], wi[pidx] > 0 ? wi[pidx] : 0.0, xs + j * m, ys + j * m, snorm);
  }
  __syncthreads();
  // coefficients in the V basis, Q x and Q y: one (row, vector) pair per thread; each row's sum starts
  // at its own column so that the threads of a warp read different shared-memory banks
  for (int e = threadIdx.x; e < nsel * m; e += blockDim.x) {
    const int j = e / m, a = e % m;
    const R* x = xs + j * m;
    const R* y = ys + j * m;
    const R* Qa = Q + a * ld;
    R qx = 0.0, qy = 0.0;
    for (int c = 0, cc = a; c < m; ++c, cc = (cc + 1 == m) ? 0 : cc + 1) {
      mac(qx, Qa[cc], x[cc]);
      mac(qy, Qa[cc], y[cc]);
    }
    Yi[a * EIG_MAXP + sel_col[j]] = (double)finish(qx);
    if (sel_two[j] == 1) Yi[a * EIG_MAXP + sel_col[j] + 1] = (double)finish(qy);
  }
  __syncthreads();
  if ((int)threadIdx.x < nsel) {
    const int j = threadIdx.x;
    const int pidx = sel_pos[j];
    const int two = sel_two[j];
    // norms
    double nx = 0.0, ny = 0.0;
    for (int a = 0; a < m; ++a) {
      const double qx = Yi[a * EIG_MAXP + sel_col[j]];
      nx += qx * qx;
      if (two == 1) {
        const double qy = Yi[a * EIG_MAXP + sel_col[j] + 1];
        ny += qy * qy;
      }
    }
    const double nrm = sqrt(nx + (two ? ny : 0.0));
    for (int a = 0; a < m; ++a) {
      Yi[a * EIG_MAXP + sel_col[j]] /= (two == 2 ? sqrt(nx) : nrm);
      if (two == 1) Yi[a * EIG_MAXP + sel_col[j] + 1] /= nrm;
    }
    // residual ||H_{s,s-1} y_last|| (Krylov mode); zero in the full space
    double res = 0.0;
    if (!full[i]) {
      const int b = prm.b, r0 = prm.sb_krylov, c0 = prm.sb_krylov - b;
      double rr = 0.0;
      for (int a = 0; a < b; ++a) {
        double ux = 0.0, uy = 0.0;
        for (int c = 0; c < b; ++c) {
          const double hv = Hi[(r0 + a) * EIG_MAXP + c0 + c];
          ux += hv * Yi[(c0 + c) * EIG_MAXP + sel_col[j]];
          if (two == 1) uy += hv * Yi[(c0 + c) * EIG_MAXP + sel_col[j] + 1];
        }
        rr += ux * ux + uy * uy;
      }
      res = sqrt(rr);
    }
    const double lam = hypot(wr[pidx], wi[pidx]);
    const bool wanted = sel_col[j] < zc_s;
    if (wanted && !(res <= prm.tol * lam)) conv_all = 0;
    if (wanted) {
      const double ratio = res / lam;
      // non-negative doubles order like their bit patterns; a NaN or infinite ratio counts as huge
      atomicMax(&worst_bits, (unsigned long long)__double_as_longlong(ratio < 1e300 ? ratio : 1e300));
      double* eo = eigout + (int64_t)i * prm.nevmax * 2;
      // slot order follows the columns; the kernel part is stored separately by the host
      eo[2 * j] = wr[pidx];
      eo[2 * j + 1] = wi[pidx] > 0 ? wi[pidx] : 0.0;
    }
  }
  // slots past this cycle's wanted set must not keep values written by an earlier cycle
  for (int j = threadIdx.x; j < prm.nevmax; j += blockDim.x)
    if (!(j < nsel && sel_col[j] < zc_s)) {
      double* eo = eigout + (int64_t)i * prm.nevmax * 2;
      eo[2 * j] = nan("");
      eo[2 * j + 1] = nan("");
    }
  conv_all = __syncthreads_and(conv_all);
  if (threadIdx.x == 0) {
    conv[i] = conv_all;
    worst[i] = __longlong_as_double((long long)worst_bits);
    ycols[i] = ncol_s;
    zcols[i] = zc_s;
  }
}

// X[:, 0:q] = V[:, 0:m] Y[0:m, 0:q] (q = qvec[i]); rows staged through shared memory
template <class T, class TX>
__global__ void __launch_bounds__(EIG_THREADS) k_vy(const int* ni, const int64_t* xoff, int ldx, const int* mvec,
                                                     const int* qvec, const int* active, const T* V,
                                                     const double* Y, TX* X) {
  using Acc = typename EAcc<T>::type;
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  if (active && !active[i]) return;
  const int n = ni[i], m = mvec[i], q = qvec[i];
  Acc* sy = reinterpret_cast<Acc*>(sm);             // m x q (padded to 3 ncg columns with zeros)
  Acc* sv = sy + EIG_MAXP * EIG_MAXP;               // VY_RC x m
  const double* Yi = Y + (int64_t)i * EIG_MAXP * EIG_MAXP;
  const int ncg = (q + 2) / 3, qp = 3 * ncg;        // groups of 3 output columns, one per thread
  for (int e = threadIdx.x; e < m * qp; e += EIG_THREADS) {
    const int a = e / qp, c = e % qp;
    sy[a * EIG_MAXP + c] = c < q ? (Acc)Yi[a * EIG_MAXP + c] : (Acc)0;
  }
  const T* Vi = V + xoff[i];
  TX* Xi = X + xoff[i];
  for (int l0 = 0; l0 < n; l0 += VY_RC) {
    const int rows = min(VY_RC, n - l0);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * m; e += EIG_THREADS)
      sv[(e / m) * EIG_MAXP + e % m] = (Acc)Vi[(int64_t)(l0 + e / m) * ldx + e % m];
    __syncthreads();
    for (int e = threadIdx.x; e < rows * ncg; e += EIG_THREADS) {
      const int r = e / ncg, c = 3 * (e % ncg);
      Acc s0 = 0, s1 = 0, s2 = 0;
      for (int a = 0; a < m; ++a) {
        const Acc v = sv[r * EIG_MAXP + a];
        mac(s0, v, sy[a * EIG_MAXP + c]);
        mac(s1, v, sy[a * EIG_MAXP + c + 1]);
        mac(s2, v, sy[a * EIG_MAXP + c + 2]);
      }
      TX* x = Xi + (int64_t)(l0 + r) * ldx + c;
      x[0] = (TX)finish(s0);
      if (c + 1 < q) x[1] = (TX)finish(s1);
      if (c + 2 < q) x[2] = (TX)finish(s2);
    }
  }
}

// Z (FP64, n_i x zld per subdomain at zoff) = [k (if kernel part), X[:, 0:zc]]
template <class T>
__global__ void k_final_z(const int* ni, const int* off, const int64_t* xoff, int ldx, const int* zcols,
                          const int* kpart, const double* kvec, const T* X, const int64_t* zoff, int zld,
                          double* Z) {
  const int i = blockIdx.x;
  const int n = ni[i], o = off[i], kp = kpart[i], zc = zcols[i];
  double* Zi = Z + zoff[i];
  for (int e = threadIdx.x; e < n * zld; e += blockDim.x) {
    const int l = e / zld, c = e % zld;
    double v = 0.0;
    if (kp && c == 0) v = kvec[o + l];
    else if (c - kp >= 0 && c - kp < zc) v = (double)X[xoff[i] + (int64_t)l * ldx + (c - kp)];
    Zi[(int64_t)l * zld + c] = v;
  }
}

// ---------------------------------------------------------------------------
// Thick restart of the block Krylov iteration.  A cycle ends with T V_m = V_{m+b} Hb, Hb = H[0:m+b, 0:m]
// (m = s b).  With Q an orthonormal basis of the kept Ritz coefficients Y[0:m, 0:b],
//     T (V_m Q) = V_{m+b} Hb Q = (V_m Q) G + V_{m+b} E,   G = Q^T Hb[0:m] Q,   E = Hb Q - [Q; 0] G,
// and E = Q2 R2 with Q2 orthonormal and orthogonal to [Q; 0].  The restarted basis is
// V' = V_{m+b} U, U = [[Q; 0], Q2] (2b columns), and the first block column of H becomes [G; R2], so the
// block Arnoldi relation T V'_0 = V'_0 G + V'_1 R2 holds and the cycle goes on with block step 1: the
// space it builds is the block Krylov space of V_m Q that an explicit restart from V_m Q builds, with
// one application of T fewer per cycle.  No invariance of span Q is assumed (a complex pair cut at the
// block edge keeps its real part only).
// One CTA per subdomain, in the arithmetic R of the Rayleigh-Ritz step (FP64, or double-float in the
// mixed form, where it runs on the FP32 pipe instead of GB300's slow FP64 units).  Writes U ((m+b) x 2b,
// stride EIG_MAXP) into Uout and H[0:m+b, 0:m] (zero but for [G; R2] in the first block column).
constexpr int TR_THREADS = 128;  // >= m + b (at most EIG_MAXP)

__device__ __forceinline__ double tr_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ dfloat tr_sqrt(dfloat v) { return se_sqrt(v); }

template <class R>
__device__ R tr_cta_sum(R v, R* red) {
  for (int o = 16; o > 0; o >>= 1) v += warp_xor<R>(v, o);
  __syncthreads();  // red may still be read by the previous call
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  R s = R(0.0);
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// Column c of U (mb rows, stride ld) orthogonalised against columns 0..c-1 by classical Gram-Schmidt:
// at least two passes, more (up to four) while a pass removes more than half of the norm.  The
// coefficients are added to coef[0..c-1] (if given).  *n0: the norm before; *ok: false when the fourth
// pass still cancelled (numerically dependent); returns the norm after (the column is not
// normalised).  Whole CTA; mb <= blockDim.x.
template <class R>
__device__ R tr_orth_column(R* U, int ld, int mb, int c, R* coef, R* dots, R* red, double* n0, bool* ok) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  R x = tid < mb ? U[tid * ld + c] : R(0.0);
  R sq = R(0.0);
  mac(sq, x, x);
  R nrm = tr_sqrt(finish(tr_cta_sum(finish(sq), red)));
  *n0 = (double)nrm;
  *ok = true;
  if (c == 0) return nrm;
  for (int pass = 0; pass < 4; ++pass) {
    for (int k = wid; k < c; k += nw) {
      R d = R(0.0);
      for (int a = lane; a < mb; a += 32) mac(d, U[a * ld + k], U[a * ld + c]);
      d = finish(d);
      for (int o = 16; o > 0; o >>= 1) d += warp_xor<R>(d, o);
      if (lane == 0) dots[k] = d;
    }
    __syncthreads();
    if (tid < mb) {
      R v = U[tid * ld + c];
      for (int k = 0; k < c; ++k) mac(v, -dots[k], U[tid * ld + k]);
      v = finish(v);
      U[tid * ld + c] = v;
      x = v;
    }
    if (coef && tid < c) coef[tid] += dots[tid];
    sq = R(0.0);
    mac(sq, x, x);
    const R nn = tr_sqrt(finish(tr_cta_sum(finish(sq), red)));
    const bool again = pass == 0 || (double)nn < 0.5 * (double)nrm;
    nrm = nn;
    if (!again) return nrm;
  }
  *ok = false;
  return nrm;
}

template <class R>
__global__ void __launch_bounds__(TR_THREADS) k_thick_restart(const int* active, int m, int b, const double* Y,
                                                           double* H, double* Uout, int* st) {
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  if (active && !active[i]) return;
  const int tid = threadIdx.x, mb = m + b, ld = 2 * b;
  R* U = reinterpret_cast<R*>(sm);  // mb x 2b
  R* Gs = U + mb * ld;              // b x b
  R* R2 = Gs + b * b;               // b x b
  R* coef = R2 + b * b;             // 2b
  R* dots = coef + ld;              // 2b
  __shared__ R red[TR_THREADS / 32];
  const double* Yi = Y + (int64_t)i * EIG_MAXP * EIG_MAXP;
  double* Hi = H + (int64_t)i * EIG_MAXP * EIG_MAXP;
  double* Ui = Uout + (int64_t)i * EIG_MAXP * EIG_MAXP;
  for (int e = tid; e < mb * b; e += blockDim.x) {
    const int a = e / b, c = e % b;
    U[a * ld + c] = a < m ? R(Yi[a * EIG_MAXP + c]) : R(0.0);
  }
  for (int e = tid; e < 2 * b * b; e += blockDim.x) Gs[e] = R(0.0);  // Gs and R2
  __syncthreads();
  // Q: a column (numerically) dependent on the ones before it is replaced by the first unit vector
  // e_r (r < m) that is not
  int cand = 0;
  for (int c = 0; c < b; ++c) {
    double n0 = 0.0;
    bool ok = true;
    R nrm = tr_orth_column(U, ld, mb, c, (R*)nullptr, dots, red, &n0, &ok);
    while (!(ok && (double)nrm > 1e-12 * n0) && cand < m) {
      if (tid < mb) U[tid * ld + c] = R((tid == cand) ? 1.0 : 0.0);
      ++cand;
      nrm = tr_orth_column(U, ld, mb, c, (R*)nullptr, dots, red, &n0, &ok);
    }
    if (!((double)nrm > 0.0)) {
      if (tid == 0) raise_status(st, A2LS_ERR_EIGEN, i, 5);
      return;  // uniform: every thread holds the same norm
    }
    if (tid < mb) U[tid * ld + c] /= nrm;
  }
  __syncthreads();
  // Hb Q into U[:, b:2b]
  for (int e = tid; e < mb * b; e += blockDim.x) {
    const int a = e / b, c = e % b;
    const double* Ha = Hi + a * EIG_MAXP;
    R sum = R(0.0);
    for (int k = 0; k < m; ++k) mac(sum, R(Ha[k]), U[k * ld + c]);
    U[a * ld + b + c] = finish(sum);
  }
  __syncthreads();
  // G and R2 by Gram-Schmidt of Hb Q against [Q; 0] and the second block's earlier columns.  Any
  // remainder the Gram-Schmidt passes leave orthogonal is kept, however small (a nearly exact Ritz
  // vector has a tiny one: its direction is then arbitrary, and R2's diagonal entry keeps the relation
  // exact).  Only a remainder that four passes keep cancelling (rounding noise) or an exact zero is
  // dropped: R2's diagonal entry 0, the column replaced by a unit vector, the residual rows first.
  // No threshold scales with |Hb|: one huge Ritz value (a nearly singular splitting) would then
  // drop the residuals of all the others.
  int cand2 = 0;
  for (int c = 0; c < b; ++c) {
    __syncthreads();  // coef of the previous column read
    if (tid < ld) coef[tid] = R(0.0);
    __syncthreads();
    double n0 = 0.0;
    bool ok = true;
    R nrm = tr_orth_column(U, ld, mb, b + c, coef, dots, red, &n0, &ok);
    if (tid < b) Gs[tid * b + c] = coef[tid];
    if (tid < c) R2[tid * b + c] = coef[b + tid];
    if (ok && (double)nrm > 0.0) {
      if (tid == 0) R2[c * b + c] = nrm;
    } else {
      while (!(ok && (double)nrm > 1e-12 * n0) && cand2 < mb) {
        const int r = cand2 < b ? m + cand2 : cand2 - b;
        if (tid < mb) U[tid * ld + b + c] = R((tid == r) ? 1.0 : 0.0);
        ++cand2;
        nrm = tr_orth_column(U, ld, mb, b + c, (R*)nullptr, dots, red, &n0, &ok);
      }
      if (!((double)nrm > 0.0)) {
        if (tid == 0) raise_status(st, A2LS_ERR_EIGEN, i, 5);
        return;
      }
    }
    if (tid < mb) U[tid * ld + b + c] /= nrm;
  }
  __syncthreads();
  for (int e = tid; e < mb * ld; e += blockDim.x) Ui[(e / ld) * EIG_MAXP + e % ld] = (double)U[e];
  for (int e = tid; e < mb * m; e += blockDim.x) {
    const int a = e / m, c = e % m;
    double v = 0.0;
    if (c < b) v = a < b ? (double)Gs[a * b + c] : (a < 2 * b ? (double)R2[(a - b) * b + c] : 0.0);
    Hi[a * EIG_MAXP + c] = v;
  }
}

// ---------------------------------------------------------------------------
// driver
// ---------------------------------------------------------------------------
// T: the factors of A~_ii and the applications of T; TV: the Krylov basis and its orthogonalisation
template <class T, class TV>
static void eigensolve_t(a2ls_handle* h, T* fac, const double* last_pivot, const double* dscale) {
  cudaStream_t st = h->st;
  const int N = h->N;
  const double tol = h->opt.eig_tol > 0 ? h->opt.eig_tol : (h->opt.precision == A2LS_FP64 ? 1e-10 : 1e-4);
  const int nev = h->nev;

  // --- kernel detection ------------------------------------------------------
  std::vector<int64_t> hoff1(N + 1, 0);
  for (int i = 0; i < N; ++i) hoff1[i + 1] = hoff1[i] + h->h_n[i];
  int64_t* d_off1 = dalloc<int64_t>(h, N + 1);
  A2LS_CUDA(cudaMemcpyAsync(d_off1, hoff1.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
  std::vector<int> ones(N, 1);
  int* d_ones = dalloc<int>(h, N);
  A2LS_CUDA(cudaMemcpyAsync(d_ones, ones.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  T* X1 = dalloc<T>(h, hoff1[N]);
  A2LS_CUDA(cudaMemsetAsync(X1, 0, sizeof(T) * hoff1[N], st));
  double* kvec = dalloc<double>(h, h->sum_n);
  double* hvec = dalloc<double>(h, h->sum_n);
  int* d_kd = dalloc<int>(h, N);
  int* d_kpart = dalloc<int>(h, N);
  k_unit_last<T><<<N, 32, 0, st>>>(h->d_ni, d_off1, dscale, X1);
  A2LS_LAUNCH();
  block_solve<T>(h, fac, X1, d_off1, 0, 1, d_ones, 1, nullptr, 0, 1);  // k' = sigma inv(U') e_n
  const double eps_work = 2.0 * Unit<T>::u;
  k_kernel_test<T><<<N, EIG_THREADS, 0, st>>>(h->d_ni, h->d_off, h->d_ld, h->d_foff, fac, last_pivot, dscale,
                                               h->d_lrow, h->d_lcol, h->d_lval, h->d_lump, h->d_D, d_off1, X1,
                                               eps_work, kvec, d_kd, d_kpart, h->d_status);
  A2LS_LAUNCH();
  cudaEvent_t tested;  // the factors are final from here on
  A2LS_CUDA(cudaEventCreateWithFlags(&tested, cudaEventDisableTiming));
  A2LS_CUDA(cudaEventRecord(tested, st));
  struct EventGuard {
    cudaEvent_t e;
    ~EventGuard() { cudaEventDestroy(e); }
  } tested_guard{tested};
  A2LS_CUDA(cudaMemsetAsync(X1, 0, sizeof(T) * hoff1[N], st));
  k_load_vec<T><<<N, 256, 0, st>>>(h->d_ni, h->d_off, d_off1, 1, kvec, d_kd, X1);
  A2LS_LAUNCH();
  block_solve<T>(h, fac, X1, d_off1, 0, 1, d_ones, 1, d_kd, 1, 0);
  k_store_h<T><<<N, 256, 0, st>>>(h->d_ni, h->d_off, d_off1, 1, X1, d_kd, hvec, h->d_status);
  A2LS_LAUNCH();
  std::vector<int> kd(N), kpart(N);
  A2LS_CUDA(cudaMemcpyAsync(kd.data(), d_kd, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaMemcpyAsync(kpart.data(), d_kpart, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  // double-float solves on the tensor cores for the subdomains with at most 32 columns (the others,
  // small full-space subdomains, on the FP32 pipe).  Their factor digits depend only on the factors as
  // the kernel test left them: they are prepared on a second stream while the rest of the kernel
  // detection above runs, and the cycles below wait for them.
  TcSolve tcs;
  struct TcsGuard {
    a2ls_handle* h;
    TcSolve& t;
    ~TcsGuard() { tc_solve_release(h, t); }
  } tcs_guard{h, tcs};
  struct PrepStream {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    ~PrepStream() {
      if (done) cudaEventDestroy(done);
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    }
  } prep;
  if constexpr (std::is_same<T, dfloat>::value) {
    if (h->opt.tensor_cores) {
      A2LS_CUDA(cudaStreamCreateWithFlags(&prep.s, cudaStreamNonBlocking));
      A2LS_CUDA(cudaEventCreateWithFlags(&prep.done, cudaEventDisableTiming));
      A2LS_CUDA(cudaStreamWaitEvent(prep.s, tested, 0));
      {
        struct Restore {  // the handle's stream comes back on every exit path
          a2ls_handle* h;
          cudaStream_t st;
          ~Restore() { h->st = st; }
        } restore{h, st};
        h->st = prep.s;
        tc_solve_prepare(h, fac, tcs);
      }
      A2LS_CUDA(cudaEventRecord(prep.done, prep.s));
    }
  }
  sync_and_check(h, "kernel detection of the local splittings");
  dfree(h, X1);

  // --- sizes ------------------------------------------------------------------
  std::vector<int> nf(N), full(N), mfull(N), pv(N);
  int nfmax = 0;
  for (int i = 0; i < N; ++i) {
    nf[i] = std::max(0, std::min(nev - kpart[i], h->h_n[i] - kd[i]));
    nfmax = std::max(nfmax, nf[i]);
  }
  if (nfmax + 4 > 32)
    fail(A2LS_ERR_ARG, "nev = %d is too large for the local eigensolver (at most 28 eigenpairs per subdomain)", nev);
  // block size: by default nev + max(4, nev / 2), raised towards 2 nev while 3 block steps still fit
  // the Krylov capacity ((s + 1) b <= EIG_MAXP): a wider block converges in fewer cycles (96^3 case,
  // nev 12: 5-9 cycles with 18 columns, 4-7 with 24, eigen phase -6 % in double-float and -5 % in
  // FP64); or the option (at least nev + 1, at most 32)
  const int b = h->opt.eig_block_size > 0
                    ? std::min(32, std::max(nfmax + 1, (int)h->opt.eig_block_size))
                    : std::min(32, std::max(nfmax + std::max(4, (nfmax + 1) / 2), std::min(2 * nfmax, EIG_MAXP / 4)));
  int s = h->opt.eig_block_steps > 0 ? h->opt.eig_block_steps : 3;
  if ((s + 1) * b > EIG_MAXP) s = EIG_MAXP / b - 1;
  if (s < 1) fail(A2LS_ERR_ARG, "nev = %d is too large for the local eigensolver (at most %d)", nev, EIG_MAXP / 2 - 8);
  const int P = EIG_MAXP;  // column stride of V and W
  for (int i = 0; i < N; ++i) {
    const int mdim = h->h_n[i] - kd[i];
    full[i] = (mdim <= (s + 1) * b) ? 1 : 0;
    mfull[i] = full[i] ? std::min(mdim, EIG_MAXP) : 0;
    pv[i] = full[i] ? mfull[i] : b;
  }
  int pmax = 1;
  for (int i = 0; i < N; ++i) pmax = std::max(pmax, pv[i]);
  std::vector<int64_t> hvo(N + 1, 0);
  for (int i = 0; i < N; ++i) hvo[i + 1] = hvo[i] + (int64_t)h->h_n[i] * P;
  int64_t* d_vo = dalloc<int64_t>(h, N + 1);
  A2LS_CUDA(cudaMemcpyAsync(d_vo, hvo.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
  int* d_full = dalloc<int>(h, N);
  int* d_mfull = dalloc<int>(h, N);
  int* d_pv = dalloc<int>(h, N);
  int* d_nf = dalloc<int>(h, N);
  int* d_active = dalloc<int>(h, N);
  int* d_conv = dalloc<int>(h, N);
  double* d_worst = dalloc<double>(h, N);
  int* d_ycols = dalloc<int>(h, N);
  int* d_zcols = dalloc<int>(h, N);
  int* d_msb = dalloc<int>(h, N);
  int* d_rank = dalloc<int>(h, N);
  std::vector<int> msb(N), act(N);
  for (int i = 0; i < N; ++i) {
    msb[i] = full[i] ? mfull[i] : s * b;
    act[i] = nf[i] > 0 ? 1 : 0;
  }
  A2LS_CUDA(cudaMemcpyAsync(d_full, full.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(d_mfull, mfull.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(d_pv, pv.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(d_nf, nf.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(d_active, act.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(d_msb, msb.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemsetAsync(d_rank, 0, sizeof(int) * N, st));
  A2LS_CUDA(cudaMemsetAsync(d_ycols, 0, sizeof(int) * N, st));
  A2LS_CUDA(cudaMemsetAsync(d_zcols, 0, sizeof(int) * N, st));
  TV* V = dalloc<TV>(h, hvo[N]);
  T* W = dalloc<T>(h, hvo[N]);
  double* H = dalloc<double>(h, (size_t)N * P * P);
  double* Y = dalloc<double>(h, (size_t)N * P * P);
  double* Rscr = dalloc<double>(h, (size_t)N * P * P);
  const int nevmax = std::max(nev, 1) + 1;
  double* eigout = dalloc<double>(h, (size_t)N * nevmax * 2);
  A2LS_CUDA(cudaMemsetAsync(V, 0, sizeof(TV) * hvo[N], st));
  A2LS_CUDA(cudaMemsetAsync(W, 0, sizeof(T) * hvo[N], st));
  A2LS_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * N * P * P, st));
  A2LS_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * N * P * P, st));
  {
    std::vector<double> nanv((size_t)N * nevmax * 2, std::nan(""));
    A2LS_CUDA(cudaMemcpyAsync(eigout, nanv.data(), sizeof(double) * nanv.size(), cudaMemcpyHostToDevice, st));
    A2LS_CUDA(cudaStreamSynchronize(st));
  }

  using Acc = typename EAcc<TV>::type;
  // Gram space: jb x p <= EIG_MAXP x 32 in Krylov mode; EIG_MAXP^2 where a full-space subdomain is
  // orthogonalised (first block step only)
  bool any_full = false;
  for (int i = 0; i < N; ++i) any_full = any_full || (full[i] && act[i]);
  const int gcap_k = EIG_MAXP * 32, gcap_f = any_full ? EIG_MAXP * EIG_MAXP : gcap_k;
  auto orc_for = [&](int gcap) { return gcap > gcap_k ? 32 : ORC_MAX; };
  auto orth_smem_for = [&](int gcap) {
    return sizeof(double) * (2 * (size_t)gcap + EIG_MAXP) + sizeof(Acc) * 2 * (size_t)orc_for(gcap) * SROW;
  };
  const size_t orth_smem = orth_smem_for(gcap_f);
  using RT = typename RRType<T>::type;
  int m_max = s * b;
  for (int i = 0; i < N; ++i)
    if (full[i]) m_max = std::max(m_max, mfull[i]);
  const size_t rr_smem = sizeof(double) * ((size_t)m_max * (m_max + 1) + (size_t)m_max * (m_max + 1) + 2 * (size_t)b * m_max +
                                           3 * (size_t)m_max) +
                         sizeof(int) * EIG_MAXP + 64;
  const size_t vy_smem = sizeof(Acc) * (EIG_MAXP * EIG_MAXP + VY_RC * EIG_MAXP);
  A2LS_CUDA(cudaFuncSetAttribute(k_orth<TV, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)orth_smem));
  A2LS_CUDA(cudaFuncSetAttribute(k_rayleigh_ritz<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rr_smem));
  A2LS_CUDA(cudaFuncSetAttribute(k_vy<TV, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vy_smem));
  A2LS_CUDA(cudaFuncSetAttribute(k_vy<TV, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vy_smem));
  // thick restart (needs a block step after the kept block: s >= 2)
  const bool thick = h->opt.eig_thick_restart != 0 && s >= 2;
  const size_t tr_smem = sizeof(double) * ((size_t)(s + 1) * b * 2 * b + 2 * (size_t)b * b + 4 * (size_t)b);
  A2LS_CUDA(cudaFuncSetAttribute(k_thick_restart<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tr_smem));
  int* d_illcond = dalloc<int>(h, N);  // per cycle: a block step needed the shifted factorisation
  int* d_thick = dalloc<int>(h, N);    // per cycle: the next restart may be thick
  A2LS_CUDA(cudaMemsetAsync(d_illcond, 0, sizeof(int) * N, st));
  A2LS_CUDA(cudaMemsetAsync(d_thick, 0, sizeof(int) * N, st));
  int* d_mb = dalloc<int>(h, N);  // rows of U: (s + 1) b
  int* d_b2 = dalloc<int>(h, N);  // columns of U: 2 b
  {
    std::vector<int> mbv(N, (s + 1) * b), b2v(N, 2 * b);
    A2LS_CUDA(cudaMemcpyAsync(d_mb, mbv.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
    A2LS_CUDA(cudaMemcpyAsync(d_b2, b2v.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
    A2LS_CUDA(cudaStreamSynchronize(st));
  }

  // T applied to V[:, vcol : vcol + p] -> W[:, 0:p]; fwd/bwd_flops: the two triangular halves over the
  // active set, counted inside the envelope of the factors
  double fwd_flops = 0.0, bwd_flops = 0.0;
  // local CSR values, partition of unity and kernel vectors in the arithmetic of the eigensolve
  using BAcc = typename EAcc<T>::type;
  const BAcc* lvalB = nullptr;
  const BAcc* DB = nullptr;
  const BAcc* kvB = nullptr;
  if constexpr (std::is_same<BAcc, double>::value) {
    lvalB = h->d_lval;
    DB = h->d_D;
    kvB = kvec;
  } else {
    BAcc* kv = dalloc<BAcc>(h, h->sum_n);
    k_convert<BAcc><<<std::min<int64_t>(152 * 8, (h->sum_n + 255) / 256 + 1), 256, 0, st>>>(h->sum_n, kvec, kv);
    A2LS_LAUNCH();
    kvB = kv;
    int64_t lnnz = 0;
    A2LS_CUDA(cudaMemcpyAsync(&lnnz, h->d_lrow + h->sum_n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    A2LS_CUDA(cudaStreamSynchronize(st));
    BAcc* lv = dalloc<BAcc>(h, lnnz);
    BAcc* dv = dalloc<BAcc>(h, h->sum_n);
    k_convert<BAcc><<<std::min<int64_t>(152 * 8, (lnnz + 255) / 256 + 1), 256, 0, st>>>(lnnz, h->d_lval, lv);
    A2LS_LAUNCH();
    k_convert<BAcc><<<std::min<int64_t>(152 * 8, (h->sum_n + 255) / 256 + 1), 256, 0, st>>>(h->sum_n, h->d_D, dv);
    A2LS_LAUNCH();
    lvalB = lv;
    DB = dv;
  }
  if (prep.done) A2LS_CUDA(cudaStreamWaitEvent(st, prep.done, 0));  // the factor digits are ready
  auto solve_sweep = [&](const int* actv, int forward) {
    if constexpr (std::is_same<T, dfloat>::value) {
      if (tcs.ready) {
        tc_block_solve(h, tcs, W, d_vo, 0, P, d_pv, actv, forward);
        block_solve<T>(h, fac, W, d_vo, 0, P, d_pv, pmax, actv, forward, !forward, TC_SOLVE_MAX_P);
        return;
      }
    }
    block_solve<T>(h, fac, W, d_vo, 0, P, d_pv, pmax, actv, forward, !forward);
  };
  auto apply_T = [&](int vcol, const int* actv) {
    k_bmul<TV, T><<<dim3(N, 8), 256, 0, st>>>(h->d_ni, h->d_off, d_vo, P, vcol, d_pv, actv, h->d_lrow, h->d_lcol,
                                             lvalB, DB, V, W);
    A2LS_LAUNCH();
    {
      KTime kt(h, KT_EIG_SOLVE, fwd_flops);
      solve_sweep(actv, 1);
    }
    k_mu_fix<T><<<N, 256, 0, st>>>(h->d_ni, h->d_off, d_vo, P, d_pv, actv, d_kd, hvec, W);
    A2LS_LAUNCH();
    {
      KTime kt(h, KT_EIG_SOLVE, bwd_flops);
      solve_sweep(actv, 0);
    }
    k_project_k<T><<<N, EIG_THREADS, 0, st>>>(h->d_ni, h->d_off, d_vo, P, 0, d_pv, actv, d_kd, kvB, W);
    A2LS_LAUNCH();
  };
  // full = the subdomains in the launch may include full-space ones, whose block has up to EIG_MAXP
  // columns (their Gram matrices need gcap_f)
  auto orthonormalize_W_into_V0 = [&](const int* actv, bool with_full) {
    k_project_k<T><<<N, EIG_THREADS, 0, st>>>(h->d_ni, h->d_off, d_vo, P, 0, d_pv, actv, d_kd, kvB, W);
    A2LS_LAUNCH();
    // no previous basis: jb = 0; R written into H's last rows (discarded)
    const int gcap = with_full ? gcap_f : gcap_k;
    k_orth<TV, T><<<N, ORTH_THREADS, orth_smem_for(gcap), st>>>(h->d_ni, d_vo, P, d_pv, actv, 0, b, V, W, Rscr, 0,
                                                                0, 0, nullptr, d_rank, gcap, orc_for(gcap), nullptr,
                                                                h->d_status);
    A2LS_LAUNCH();
  };

  // initial block: random or the warm-start network's proposal, then orthogonal to k, orthonormal
  if (h->opt.warm_start) {
    float* Yw = dalloc<float>(h, (size_t)h->sum_n * WARM_COLS);
    gnn_infer(h, h->opt.warm_start, Yw);
    k_warm_block<T><<<N, 256, 0, st>>>(h->d_ni, h->d_off, d_vo, P, d_pv, d_active, d_full, Yw, h->opt.seed, W);
    A2LS_LAUNCH();
    dfree(h, Yw);
  } else {
    k_random_block<T><<<N, 256, 0, st>>>(h->d_ni, d_vo, P, 0, d_pv, d_active, h->opt.seed, 0, W);
    A2LS_LAUNCH();
  }
  orthonormalize_W_into_V0(d_active, any_full);
  A2LS_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * N * P * P, st));

  // --- restarted block Krylov cycles, in two interleaved groups of subdomains --------------------
  // The subdomains alternate between two groups, each with its own stream.  After a group's
  // Rayleigh-Ritz step the host reads that group's convergence flags and queues its next cycle while
  // the other group still runs: the latency-bound Rayleigh-Ritz and the tails of the block solves of
  // one group overlap the other group's work.  Each group touches only its own subdomains' slices of
  // V, W, H and Y.  With per-kernel timing on, one group on the handle's stream keeps the kernels'
  // times free of overlap.
  const int ngroups = h->opt.timing ? 1 : 2;
  // thick restarts while u |theta_1| stays below 1e-2 tol |theta_b| with a margin of 64 for the rounding
  // of the block steps
  RRParams prm{s * b, b, s, tol, nevmax, h->opt.tau, thick ? 1e-2 * tol / (64.0 * Unit<T>::u) : 0.0};
  const int max_cycles = h->opt.eig_max_cycles > 0 ? h->opt.eig_max_cycles : 60;
  const int stall_cycles = h->opt.eig_stall_cycles;
  std::vector<int> cycles(N, 0), best_cycle(N, 0), stalled(N, 0);
  std::vector<double> best(N, INFINITY), worst(N, 0.0);
  struct Group {
    std::vector<int> act, actk, thk, exl;  // exl/thk: restarted explicitly / thick
    int* d_act = nullptr;
    int* d_actk = nullptr;
    int* d_thk = nullptr;
    int* d_exl = nullptr;
    int* h_conv = nullptr;  // pinned: N convergence flags, N thick-restart flags, then the status words
    double* h_worst = nullptr;  // pinned: N worst relative residuals of the wanted Ritz pairs
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    int cycle = 0;
    bool finished = false;
  };
  Group grp[2];
  struct GroupStreams {  // the second stream and the pinned buffers, released on every exit path
    a2ls_handle* h;
    cudaStream_t orig, s1 = nullptr;
    Group* g;
    ~GroupStreams() {
      if (s1) {
        cudaStreamSynchronize(s1);
        cudaStreamDestroy(s1);
      }
      for (int q = 0; q < 2; ++q) {
        if (g[q].done) cudaEventDestroy(g[q].done);
        if (g[q].h_conv) cudaFreeHost(g[q].h_conv);
        if (g[q].h_worst) cudaFreeHost(g[q].h_worst);
      }
      h->st = orig;
    }
  } guard{h, st, nullptr, grp};
  grp[0].s = st;
  if (ngroups == 2) {
    A2LS_CUDA(cudaStreamCreateWithFlags(&guard.s1, cudaStreamNonBlocking));
    grp[1].s = guard.s1;
    cudaEvent_t ready;
    A2LS_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    A2LS_CUDA(cudaEventRecord(ready, st));
    A2LS_CUDA(cudaStreamWaitEvent(guard.s1, ready, 0));
    A2LS_CUDA(cudaEventDestroy(ready));
  }
  for (int g = 0; g < ngroups; ++g) {
    Group& G = grp[g];
    G.act.assign(N, 0);
    G.actk.assign(N, 0);
    for (int i = g; i < N; i += ngroups) G.act[i] = act[i];
    G.d_act = dalloc<int>(h, N);
    G.d_actk = dalloc<int>(h, N);
    G.thk.assign(N, 0);
    G.exl.assign(N, 0);
    G.d_thk = dalloc<int>(h, N);
    G.d_exl = dalloc<int>(h, N);
    A2LS_CUDA(cudaMallocHost(&G.h_conv, sizeof(int) * (2 * N + ST_WORDS)));
    A2LS_CUDA(cudaMallocHost(&G.h_worst, sizeof(double) * N));
    A2LS_CUDA(cudaEventCreateWithFlags(&G.done, cudaEventDisableTiming));
    A2LS_CUDA(cudaMemcpyAsync(G.d_act, G.act.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  }
  A2LS_CUDA(cudaStreamSynchronize(st));
  auto use_stream = [&](cudaStream_t s2) {
    st = s2;
    h->st = s2;
  };
  // one cycle of group g: s block steps, Rayleigh-Ritz, then the flags and status copied to the host
  // j0 = 1 after a thick restart: block 0 and block 1 of V and H's first block column are in place
  // block step j over the subdomains actv (acth on the host): T V_j, orthogonalised -> V_{j+1}, H
  auto block_step = [&](int j, const int* actv, const std::vector<int>& acth) {
      fwd_flops = bwd_flops = 0.0;
      double orth_flops = 0.0;
      for (int i = 0; i < N; ++i) {
        if (!acth[i]) continue;
        const double ni = h->h_n[i], pi = pv[i], jb = full[i] ? pi : (double)(j + 1) * b;
        fwd_flops += 2.0 * h->h_env[4 * i + 2] * pi;
        bwd_flops += 2.0 * h->h_env[4 * i + 3] * pi;
        orth_flops += 8.0 * ni * jb * pi + 9.0 * ni * pi * pi;
      }
      apply_T(j * b, actv);
      // Krylov subdomains: block CGS2 + CholQR2 -> V_{j+1}, H[:, j-th block];
      // full-space subdomains (j == 0 only): H = V0^T (T V0)
      {
        KTime kt(h, KT_EIG_ORTH, orth_flops);
        const int gcap = (j == 0) ? gcap_f : gcap_k;
        k_orth<TV, T><<<N, ORTH_THREADS, orth_smem_for(gcap), st>>>(h->d_ni, d_vo, P, d_pv, actv, j + 1, b, V, W, H,
                                                      (j + 1) * b, j * b, (j + 1) * b, d_full, d_rank, gcap,
                                                      orc_for(gcap), d_illcond, h->d_status);
        A2LS_LAUNCH();
      }
  };
  auto queue_cycle = [&](int g, int j0) {
    Group& G = grp[g];
    use_stream(G.s);
    for (int i = 0; i < N; ++i) G.actk[i] = G.act[i] && !full[i];
    A2LS_CUDA(cudaMemcpyAsync(G.d_actk, G.actk.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
    for (int j = j0; j < s; ++j) {
      if (j == 0)
        block_step(j, G.d_act, G.act);
      else
        block_step(j, G.d_actk, G.actk);
    }
    {
      // algorithmic work: a real Schur form with its orthogonal factor (25 m^3, the usual count for
      // Hessenberg reduction plus Francis iteration) and the coefficients of b Ritz vectors (2 b m^2)
      double rr_flops = 0.0;
      for (int i = 0; i < N; ++i) {
        if (!G.act[i]) continue;
        const double m = full[i] ? (double)mfull[i] : (double)s * b;
        rr_flops += 25.0 * m * m * m + 2.0 * b * m * m;
      }
      KTime kt(h, KT_EIG_RR, rr_flops);
      k_rayleigh_ritz<RT><<<N, RR_THREADS, rr_smem, st>>>(prm, d_full, d_mfull, d_nf, G.d_act, H, Y, d_ycols, d_zcols,
                                              eigout, d_conv, d_worst, d_illcond, d_thick, h->d_status);
      A2LS_LAUNCH();
    }
    A2LS_CUDA(cudaMemcpyAsync(G.h_conv, d_conv, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    A2LS_CUDA(cudaMemcpyAsync(G.h_conv + N, d_thick, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
    A2LS_CUDA(cudaMemcpyAsync(G.h_conv + 2 * N, h->d_status, sizeof(int) * ST_WORDS, cudaMemcpyDeviceToHost, st));
    A2LS_CUDA(cudaMemcpyAsync(G.h_worst, d_worst, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    A2LS_CUDA(cudaEventRecord(G.done, st));
  };
  for (int g = 0; g < ngroups; ++g) queue_cycle(g, 0);
  if (ngroups == 1) grp[1].finished = true;
  while (!grp[0].finished || !grp[1].finished) {
    for (int g = 0; g < ngroups; ++g) {
      Group& G = grp[g];
      if (G.finished) continue;
      A2LS_CUDA(cudaEventSynchronize(G.done));
      if (G.h_conv[2 * N + ST_CODE] != 0) sync_and_check(h, "local eigensolve");  // raises the recorded error
      int remaining = 0;
      for (int i = g; i < N; i += ngroups) {
        if (G.act[i]) {
          cycles[i] = G.cycle + 1;
          const double w = G.h_worst[i];
          worst[i] = w;
          if (G.h_conv[i] || full[i]) {
            G.act[i] = 0;
            continue;
          }
          // stagnation stop: a subdomain whose worst wanted residual has not halved over the last
          // eig_stall_cycles cycles keeps the Ritz vectors it has (still a valid coarse space)
          if (w < 0.5 * best[i]) {
            best[i] = w;
            best_cycle[i] = G.cycle;
          } else if (stall_cycles > 0 && G.cycle - best_cycle[i] >= stall_cycles) {
            G.act[i] = 0;
            stalled[i] = 1;
            continue;
          }
          ++remaining;
        }
      }
      // after the last cycle V and Y stay as they are: the unconverged subdomains keep their Ritz vectors
      if (remaining == 0 || G.cycle + 1 == max_cycles) {
        G.finished = true;
        continue;
      }
      ++G.cycle;
      use_stream(G.s);
      A2LS_CUDA(cudaMemcpyAsync(G.d_act, G.act.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
      // thick restart where the Rayleigh-Ritz step allowed it, explicit restart elsewhere
      int nthk = 0, nexl = 0;
      for (int i = 0; i < N; ++i) {
        G.thk[i] = G.act[i] && thick && G.h_conv[N + i];
        G.exl[i] = G.act[i] && !G.thk[i];
        nthk += G.thk[i];
        nexl += G.exl[i];
      }
      if (nthk) {
        // V[:, 0:2b] = V[:, 0:(s+1)b] U in place, H's first block column [G; R2]
        A2LS_CUDA(cudaMemcpyAsync(G.d_thk, G.thk.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
        k_thick_restart<RT><<<N, TR_THREADS, tr_smem, st>>>(G.d_thk, s * b, b, Y, H, Rscr, h->d_status);
        A2LS_LAUNCH();
        k_vy<TV, TV><<<N, EIG_THREADS, vy_smem, st>>>(h->d_ni, d_vo, P, d_mb, d_b2, G.d_thk, V, Rscr, V);
        A2LS_LAUNCH();
      }
      if (nexl) {
        // explicit restart block: W = V[:, 0:sb] Y[:, 0:b], orthonormalised into V_0; with thick
        // restarts elsewhere in the group, block step 0 of these subdomains runs here
        A2LS_CUDA(cudaMemcpyAsync(G.d_exl, G.exl.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
        k_vy<TV, T><<<N, EIG_THREADS, vy_smem, st>>>(h->d_ni, d_vo, P, d_msb, d_pv, G.d_exl, V, Y, W);
        A2LS_LAUNCH();
        orthonormalize_W_into_V0(G.d_exl, false);  // restarted subdomains are Krylov ones
        if (thick) block_step(0, G.d_exl, G.exl);
      }
      queue_cycle(g, thick ? 1 : 0);
    }
  }
  // both groups done: continue on the handle's stream after the second stream's work
  if (ngroups == 2) {
    cudaEvent_t joined;
    A2LS_CUDA(cudaEventCreateWithFlags(&joined, cudaEventDisableTiming));
    A2LS_CUDA(cudaEventRecord(joined, guard.s1));
    A2LS_CUDA(cudaStreamWaitEvent(guard.orig, joined, 0));
    A2LS_CUDA(cudaEventDestroy(joined));
  }
  use_stream(guard.orig);
  sync_and_check(h, "local eigensolve");
  for (int i = 0; i < N; ++i) act[i] = grp[i % ngroups].act[i];
  for (int g = 0; g < ngroups; ++g) {
    dfree(h, grp[g].d_act);
    dfree(h, grp[g].d_actk);
  }
  int unconverged = 0, nstalled = 0;
  for (int i = 0; i < N; ++i) {
    unconverged += act[i] || stalled[i];
    nstalled += stalled[i];
  }
  h->eig_unconverged = unconverged;
  h->eig_stalled = nstalled;
  h->h_eigres = worst;
  if (unconverged && h->opt.eig_strict)
    fail(A2LS_ERR_EIGEN,
         "local eigensolve did not reach tolerance %.1e for %d subdomains (%d stagnated, the others ran %d cycles)",
         tol, unconverged, nstalled, max_cycles);

  // --- final coarse vectors: Z = [k | V Y[:, 0:zc]] ------------------------------------------
  for (int i = 0; i < N; ++i) act[i] = nf[i] > 0 ? 1 : 0;
  A2LS_CUDA(cudaMemcpyAsync(d_active, act.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  std::vector<int> zc(N), yc(N);
  A2LS_CUDA(cudaMemcpyAsync(zc.data(), d_zcols, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  k_vy<TV, T><<<N, EIG_THREADS, vy_smem, st>>>(h->d_ni, d_vo, P, d_msb, d_zcols, d_active, V, Y, W);
  A2LS_LAUNCH();
  const int zld = nev + 2;
  std::vector<int64_t> hzo(N + 1, 0);
  std::vector<int> mcols(N);
  for (int i = 0; i < N; ++i) {
    hzo[i + 1] = hzo[i] + (int64_t)h->h_n[i] * zld;
    mcols[i] = kpart[i] + (nf[i] > 0 ? zc[i] : 0);
  }
  int64_t* d_zo = dalloc<int64_t>(h, N + 1);
  A2LS_CUDA(cudaMemcpyAsync(d_zo, hzo.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
  double* Z = dalloc<double>(h, hzo[N]);
  // subdomains without a finite part still need their kernel column
  int* d_zc_eff = dalloc<int>(h, N);
  std::vector<int> zc_eff(N);
  for (int i = 0; i < N; ++i) zc_eff[i] = nf[i] > 0 ? zc[i] : 0;
  A2LS_CUDA(cudaMemcpyAsync(d_zc_eff, zc_eff.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  k_final_z<T><<<N, 256, 0, st>>>(h->d_ni, h->d_off, d_vo, P, d_zc_eff, d_kpart, kvec, W, d_zo, zld, Z);
  A2LS_LAUNCH();

  // eigenvalue export: kernel part as (+inf, 0) first
  std::vector<double> ev((size_t)N * nevmax * 2);
  A2LS_CUDA(cudaMemcpyAsync(ev.data(), eigout, sizeof(double) * ev.size(), cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  h->h_eigvals.assign((size_t)N * nevmax * 2, std::nan(""));
  h->h_eigstats.assign(2 * N, 0);
  for (int i = 0; i < N; ++i) {
    double* dst = &h->h_eigvals[(size_t)i * nevmax * 2];
    int slot = 0;
    if (kpart[i]) {
      dst[0] = INFINITY;
      dst[1] = 0.0;
      slot = 1;
    }
    // eigout holds one slot per selected eigenvalue (pairs once, with +imag)
    for (int j = 0; j < nevmax && slot < nevmax; ++j) {
      const double re = ev[(size_t)i * nevmax * 2 + 2 * j], im = ev[(size_t)i * nevmax * 2 + 2 * j + 1];
      if (std::isnan(re)) break;
      dst[2 * slot] = re;
      dst[2 * slot + 1] = im;
      ++slot;
      if (im > 0 && slot < nevmax) {
        dst[2 * slot] = re;
        dst[2 * slot + 1] = -im;
        ++slot;
      }
    }
    h->h_eigstats[2 * i] = cycles[i];
    h->h_eigstats[2 * i + 1] = kd[i];
  }
  orthonormalize_and_set_W(h, Z, mcols.data(), zld);
  dfree(h, V);
  dfree(h, W);
  dfree(h, H);
  dfree(h, Y);
  dfree(h, Rscr);
  if constexpr (!std::is_same<BAcc, double>::value) {
    dfree(h, const_cast<BAcc*>(lvalB));
    dfree(h, const_cast<BAcc*>(DB));
    dfree(h, const_cast<BAcc*>(kvB));
  }
  // keep Z (the eigenvectors behind the coarse space) as the warm-start network's training target
  if (h->d_zev) dfree(h, h->d_zev);
  if (h->d_zoff) dfree(h, h->d_zoff);
  h->d_zev = Z;
  h->d_zoff = d_zo;
  h->zld = zld;
  h->h_zcols = mcols;
}

// The local eigenproblems run in the precision of the local factors.  In FP32 the
// factorisation of A~_ii with its last pivot replaced has condition numbers of
// 1e8-1e9 for the target problems, but the error of a solve concentrates along the
// kernel vector that the operator projects out: applications of T carry relative
// errors of 1e-6 to 4e-3, which bounds how well the FP32 coarse space matches the
// FP64 one (the flexible outer iteration absorbs the difference).
// The Krylov basis has the precision of the solves with A~_ii.  (An FP32 basis with FP64 solves
// produced non-finite Rayleigh-Ritz matrices on the high-contrast problem and is not used.)
void eigensolve(a2ls_handle* h, void* fac_tilde, const double* last_pivot, const double* diag_scale) {
  if (h->opt.eig_precision == A2LS_FP32)
    eigensolve_t<float, float>(h, static_cast<float*>(fac_tilde), last_pivot, diag_scale);
  else if (h->opt.eig_precision == A2LS_FP32X2)
    eigensolve_t<dfloat, dfloat>(h, static_cast<dfloat*>(fac_tilde), last_pivot, diag_scale);
  else
    eigensolve_t<double, double>(h, static_cast<double*>(fac_tilde), last_pivot, diag_scale);
}

}  // namespace a2ls

// The apply of the preconditioners of Section 2 (Eqs. 2.1-2.4) and the
// right-preconditioned restarted (F)GMRES of Section 4, all vectors FP64.
//
// Deflated RAS (Eq. 2.4), the default:
//   g = R_0 r            (tall-skinny W_i^T r(Omega_i), warp-shuffle reductions)
//   c = A_00^{-1} g      (dense FP64 matrix-vector product with the inverse)
//   q = R_0^H c          (prolongation)
//   t = r - A q          (CSR SpMV)
//   z = q + sum_i R_i^T D_i A_ii^{-1} R_i t   (gather, two triangular solves, weighted scatter)
#include "a2ls_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace a2ls {

// ---------------------------------------------------------------------------
// CSR SpMV: y = A x, or y = bm - A x when bm != nullptr; one warp per 32 rows,
// 4 lanes per row for short rows
// ---------------------------------------------------------------------------
__global__ void k_spmv(int n, const int* __restrict__ rowptr, const int* __restrict__ colind,
                       const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                       const double* __restrict__ bm) {
  const int sub = threadIdx.x & 3;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 2; r < n; r += (gridDim.x * blockDim.x) >> 2) {
    double s = 0.0;
    const int a = rowptr[r], b = rowptr[r + 1];
    for (int q = a + sub; q < b; q += 4) s += val[q] * __ldg(x + colind[q]);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (sub == 0) y[r] = bm ? bm[r] - s : s;
  }
}

void spmv(a2ls_handle* h, const double* x, double* y, const double* b_minus, cudaStream_t st) {
  const int threads = 256;
  const int blocks = std::min(152 * 8, ceil_div((int64_t)h->n * 4, threads));
  k_spmv<<<blocks, threads, 0, st>>>(h->n, h->rowptr, h->colind, h->val, x, y, b_minus);
  A2LS_LAUNCH();
}

// ---------------------------------------------------------------------------
// g[coff_i + a] = sum_l W_i[l][a] r[idx[off_i + l]] over rows with D != 0.
// Lanes are split into groups of G >= m_i columns; the 32/G row groups of a warp
// are combined by warp shuffles, the warps of the CTA through shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_restrict(const int* ni, const int* nI, const int* off, const int* idx,
                                                  const int* m, const int* coff, const int64_t* woff,
                                                  const double* __restrict__ W, const double* __restrict__ r,
                                                  double* g, int boolean_pou) {
  __shared__ double part[8][MAXM];
  const int i = blockIdx.x;
  const int mi = m[i];
  if (mi == 0) return;
  const int rows = boolean_pou ? nI[i] : ni[i];
  const int o = off[i];
  const double* Wi = W + woff[i];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int G = 1;
  while (G < mi && G < 32) G <<= 1;
  const int rg = 32 / G;          // row groups per warp
  const int sub = lane / G, a = lane % G;
  for (int c0 = 0; c0 < mi; c0 += 32) {
    double acc = 0.0;
    const int col = c0 + a;
    for (int l = wid * rg + sub; l < rows; l += 8 * rg) {
      const double rv = __ldg(r + idx[o + l]);
      if (col < mi) acc += Wi[(int64_t)l * mi + col] * rv;
    }
    for (int s = G; s < 32; s <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    if (sub == 0 && col < mi) part[wid][col] = acc;
    __syncthreads();
    if (threadIdx.x < 32 && c0 + threadIdx.x < mi) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += part[w][c0 + threadIdx.x];
      g[coff[i] + c0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// c = Einv g; one warp per row, 16-byte loads
__global__ void __launch_bounds__(256) k_gemv(int n0, const double* __restrict__ Einv,
                                              const double* __restrict__ g, double* __restrict__ c) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const bool even = (n0 & 1) == 0;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n0; row += warps) {
    const double* er = Einv + (int64_t)row * n0;
    double s = 0.0;
    if (even) {
      const double2* e2 = reinterpret_cast<const double2*>(er);
      const double2* g2 = reinterpret_cast<const double2*>(g);
      for (int k = lane; k < n0 / 2; k += 32) {
        const double2 a = __ldg(e2 + k), b = __ldg(g2 + k);
        s += a.x * b.x + a.y * b.y;
      }
    } else {
      for (int k = lane; k < n0; k += 32) s += __ldg(er + k) * __ldg(g + k);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) c[row] = s;
  }
}

// q[g] = sum over memberships (j, pos) of node g with D != 0 of W_j[pos - off_j, :] . c_j
__global__ void k_prolong(int n, const int* mrow, const int* mpos, const int* msub, const int* off, const int* m,
                          const int* coff, const int64_t* woff, const double* D, const double* __restrict__ W,
                          const double* __restrict__ c, double* q) {
  for (int gI = blockIdx.x * blockDim.x + threadIdx.x; gI < n; gI += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = mrow[gI]; t < mrow[gI + 1]; ++t) {
      const int p = mpos[t];
      if (D[p] == 0.0) continue;
      const int j = msub[t], mj = m[j];
      const double* w = W + woff[j] + (int64_t)(p - off[j]) * mj;
      const double* cj = c + coff[j];
      for (int a = 0; a < mj; ++a) s += w[a] * cj[a];
    }
    q[gI] = s;
  }
}

// z[g] = (q ? q[g] : 0) + sum over memberships of yloc[pos]
__global__ void k_combine(int n, const int* mrow, const int* mpos, const double* __restrict__ yloc,
                          const double* __restrict__ q, double* z) {
  for (int gI = blockIdx.x * blockDim.x + threadIdx.x; gI < n; gI += gridDim.x * blockDim.x) {
    double s = q ? q[gI] : 0.0;
    for (int t = mrow[gI]; t < mrow[gI + 1]; ++t) s += yloc[mpos[t]];
    z[gI] = s;
  }
}

static int grid1d(int64_t n, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(152 * 8, (n + threads - 1) / threads));
}

static void local_part(a2ls_handle* h, const double* t, const double* q, double* z, bool ras) {
  const bool boolean = h->opt.pou == A2LS_POU_BOOLEAN;
  const int mode = ras ? (boolean ? 0 : 1) : 2;
  double* out = (mode == 0) ? z : h->d_yloc;
  local_solves_any(h, t, q, out, mode);
  if (mode != 0) {
    k_combine<<<grid1d(h->n), 256, 0, h->st>>>(h->n, h->d_mrow, h->d_mpos, h->d_yloc, q, z);
    A2LS_LAUNCH();
  }
}

static void coarse_correction(a2ls_handle* h, const double* r, double* q) {
  cudaStream_t st = h->st;
  k_restrict<<<h->N, 256, 0, st>>>(h->d_ni, h->d_nI, h->d_off, h->d_idx, h->d_m, h->d_coff, h->d_woff, h->d_W,
                                   r, h->d_g, h->opt.pou == A2LS_POU_BOOLEAN);
  A2LS_LAUNCH();
  k_gemv<<<std::min(152 * 8, ceil_div((int64_t)h->n0 * 32, 256)), 256, 0, st>>>(h->n0, h->d_Einv, h->d_g, h->d_c);
  A2LS_LAUNCH();
  k_prolong<<<grid1d(h->n), 256, 0, st>>>(h->n, h->d_mrow, h->d_mpos, h->d_msub, h->d_off, h->d_m, h->d_coff,
                                          h->d_woff, h->d_D, h->d_W, h->d_c, q);
  A2LS_LAUNCH();
}

void apply_preconditioner(a2ls_handle* h, const double* r, double* z) {
  const int v = h->opt.variant;
  const bool ras = (v == A2LS_DEFLATED_RAS || v == A2LS_ADDITIVE_RAS || v == A2LS_ONE_LEVEL_RAS);
  const bool coarse = (v != A2LS_ONE_LEVEL_RAS && v != A2LS_ONE_LEVEL_ASM) && h->n0 > 0;
  const bool deflated = (v == A2LS_DEFLATED_RAS || v == A2LS_DEFLATED_ASM);
  if (!coarse) {
    local_part(h, r, nullptr, z, ras);
    return;
  }
  coarse_correction(h, r, h->d_q);
  if (deflated) {
    spmv(h, h->d_q, h->d_t, r, h->st);  // t = r - A q
    local_part(h, h->d_t, h->d_q, z, ras);
  } else {
    local_part(h, r, h->d_q, z, ras);
  }
}

// The apply as a CUDA graph, captured once per (r, z) pair on an internal stream and replayed on
// the handle's stream: GMRES applies the preconditioner to the same m basis vectors every cycle.
void apply_preconditioner_graph(a2ls_handle* h, const double* r, double* z) {
  if (!h->opt.graphs) {
    apply_preconditioner(h, r, z);
    return;
  }
  for (const auto& g : h->graphs)
    if (g.r == r && g.z == z) {
      A2LS_CUDA(cudaGraphLaunch(g.exec, h->st));
      h->launches += 1;
      return;
    }
  if (!h->cap_st) A2LS_CUDA(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
  cudaStream_t user = h->st;
  const int timing = h->opt.timing;
  h->opt.timing = 0;
  h->st = h->cap_st;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    try {
      apply_preconditioner(h, r, z);
    } catch (...) {
      cudaStreamEndCapture(h->cap_st, &graph);
      if (graph) cudaGraphDestroy(graph);
      h->st = user;
      h->opt.timing = timing;
      throw;
    }
    e = cudaStreamEndCapture(h->cap_st, &graph);
  }
  h->st = user;
  h->opt.timing = timing;
  A2LS_CUDA(e);
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  A2LS_CUDA(ei);
  h->graphs.push_back({r, z, exec});
  A2LS_CUDA(cudaGraphLaunch(exec, h->st));
  h->launches += 1;
}

// ---------------------------------------------------------------------------
// reductions for GMRES: multi-dot with a last-block-done final reduction
// out[k] = sum_r V[k][r] * w[r] for k < nv, out[nv] = w . w (if with_self)
// ---------------------------------------------------------------------------
constexpr int MD_MAX = 33;
constexpr int MD_BLOCKS = 304;

__global__ void __launch_bounds__(256) k_multidot(int n, const double* __restrict__ V, int64_t ldv, int nv,
                                                  const double* __restrict__ w, int with_self,
                                                  double* partial, unsigned* counter, double* out) {
  __shared__ double red[8][MD_MAX];
  __shared__ bool last;
  const int nd = nv + (with_self ? 1 : 0);
  double acc[MD_MAX];
#pragma unroll
  for (int k = 0; k < MD_MAX; ++k) acc[k] = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const double wr = w[r];
#pragma unroll
    for (int k = 0; k < MD_MAX; ++k) {
      if (k < nv) acc[k] += V[(int64_t)k * ldv + r] * wr;
      else if (k == nv && with_self) acc[k] += wr * wr;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < MD_MAX; ++k) {
    if (k < nd) {
      double v = acc[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][k] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < nd) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
    partial[(int64_t)blockIdx.x * MD_MAX + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (last) {
    __threadfence();
    if (threadIdx.x < nd) {
      double t = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) t += partial[(int64_t)b * MD_MAX + threadIdx.x];
      out[threadIdx.x] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// w -= sum_k hk V_k  (optionally accumulate hsum += h)
__global__ void k_cgs_update(int n, const double* __restrict__ V, int64_t ldv, int nv, const double* hcoef,
                             double* w, double* hsum) {
  __shared__ double hs[MD_MAX];
  if (threadIdx.x < nv) hs[threadIdx.x] = hcoef[threadIdx.x];
  __syncthreads();
  if (hsum && blockIdx.x == 0 && threadIdx.x < nv) hsum[threadIdx.x] += hs[threadIdx.x];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double s = w[r];
    for (int k = 0; k < nv; ++k) s -= hs[k] * V[(int64_t)k * ldv + r];
    w[r] = s;
  }
}

// y = x * (1 / *alpha) or y = x * alpha_host when alpha_dev == nullptr
__global__ void k_scale(int n, const double* x, double* y, const double* alpha_dev, int sqrt_of, double alpha_host) {
  double a = alpha_host;
  if (alpha_dev) a = 1.0 / (sqrt_of ? sqrt(*alpha_dev) : *alpha_dev);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) y[r] = x[r] * a;
}

// y = sum_k c_k V_k (c on device); optionally x += y
__global__ void k_lincomb(int n, const double* __restrict__ V, int64_t ldv, int nv, const double* coef, double* y,
                          double* xacc) {
  __shared__ double cs[MD_MAX];
  if (threadIdx.x < nv) cs[threadIdx.x] = coef[threadIdx.x];
  __syncthreads();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nv; ++k) s += cs[k] * V[(int64_t)k * ldv + r];
    if (xacc) xacc[r] += s;
    else y[r] = s;
  }
}

__global__ void k_axpy(int n, double a, const double* x, double* y) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) y[r] += a * x[r];
}

struct Reducer {
  double* partial = nullptr;
  unsigned* counter = nullptr;
  double* out = nullptr;
};

static Reducer& reducer(a2ls_handle* h) {
  if (!h->d_red) {
    h->d_red = dalloc<double>(h, (size_t)MD_BLOCKS * MD_MAX + 4 * MD_MAX + 16);
    A2LS_CUDA(cudaMemsetAsync(h->d_red, 0, sizeof(double) * ((size_t)MD_BLOCKS * MD_MAX + 4 * MD_MAX + 16), h->st));
  }
  static thread_local Reducer r;
  r.partial = h->d_red;
  r.out = h->d_red + (size_t)MD_BLOCKS * MD_MAX;             // 4 * MD_MAX doubles of outputs
  r.counter = reinterpret_cast<unsigned*>(r.out + 4 * MD_MAX);
  return r;
}

static void multidot(a2ls_handle* h, const double* V, int64_t ldv, int nv, const double* w, int with_self,
                     double* out) {
  Reducer& R = reducer(h);
  const int blocks = std::min(MD_BLOCKS, std::max(1, ceil_div(h->n, 256)));
  k_multidot<<<blocks, 256, 0, h->st>>>(h->n, V, ldv, nv, w, with_self, R.partial, R.counter, out);
  A2LS_LAUNCH();
}

double dot(a2ls_handle* h, const double* x, const double* y) {
  Reducer& R = reducer(h);
  multidot(h, x, 0, 1, y, 0, R.out);
  double v;
  A2LS_CUDA(cudaMemcpyAsync(&v, R.out, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  A2LS_CUDA(cudaStreamSynchronize(h->st));
  return v;
}

double nrm2(a2ls_handle* h, const double* x) {
  Reducer& R = reducer(h);
  multidot(h, x, 0, 0, x, 1, R.out);
  double v;
  A2LS_CUDA(cudaMemcpyAsync(&v, R.out, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  A2LS_CUDA(cudaStreamSynchronize(h->st));
  return std::sqrt(v);
}

// ---------------------------------------------------------------------------
// GMRES(m), right preconditioned (Section 4); flexible variant stores z_j.
// Stopping rule: the estimated residual |g_{j+1}| <= rtol ||b|| ends a cycle;
// the iterate is formed and the true residual decides; restarts otherwise.
// ---------------------------------------------------------------------------
int gmres(a2ls_handle* h, const double* b, double* x, double rtol, int* iters_out, double* relres_out) {
  cudaStream_t st = h->st;
  const int n = h->n;
  const int m = std::max(1, std::min(h->opt.restart > 0 ? h->opt.restart : 30, MD_MAX - 2));
  const bool flexible = h->opt.flexible < 0 ? (h->opt.precision != A2LS_FP64) : (h->opt.flexible != 0);
  const int max_it = h->opt.max_it > 0 ? h->opt.max_it : 1000;
  if (h->gm_restart != m || !h->d_V) {
    if (h->d_V) dfree(h, h->d_V);
    if (h->d_Z) dfree(h, h->d_Z);
    if (h->d_w) dfree(h, h->d_w);
    h->d_V = dalloc<double>(h, (size_t)(m + 1) * n);
    h->d_Z = dalloc<double>(h, (size_t)m * n);
    h->d_w = dalloc<double>(h, (size_t)2 * n);
    h->d_h = dalloc<double>(h, 4 * MD_MAX);
    h->gm_restart = m;
  }
  if (!h->h_pinned) A2LS_CUDA(cudaMallocHost(&h->h_pinned, sizeof(double) * 4 * MD_MAX));
  double* V = h->d_V;
  double* Zs = h->d_Z;
  double* w = h->d_w;
  double* tmp = h->d_w + n;
  double* dh = h->d_h;              // [0, MD_MAX): h1 (+ w.w), [MD_MAX, 2MD_MAX): h2, [2MD_MAX]: |w|^2, [3MD_MAX..): coefs
  double* hp = h->h_pinned;
  Reducer& R = reducer(h);
  const int gb = grid1d(n);
  const double bnorm = nrm2(h, b);
  if (bnorm == 0.0) {
    A2LS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return A2LS_OK;
  }
  int total = 0;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  while (true) {
    spmv(h, x, w, b, st);  // w = b - A x
    const double beta = nrm2(h, w);
    if (beta <= rtol * bnorm || total >= max_it) {
      if (iters_out) *iters_out = total;
      if (relres_out) *relres_out = beta / bnorm;
      return beta <= rtol * bnorm ? A2LS_OK : A2LS_ERR_NOT_CONVERGED;
    }
    k_scale<<<gb, 256, 0, st>>>(n, w, V, nullptr, 0, 1.0 / beta);
    A2LS_LAUNCH();
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * n;
      double* zj = flexible ? Zs + (size_t)j * n : tmp;
      apply_preconditioner_graph(h, vj, zj);
      spmv(h, zj, w, nullptr, st);  // w = A z_j
      // CGS2 against V_0..V_j
      multidot(h, V, n, j + 1, w, 1, dh);                 // h1, |w|^2
      k_cgs_update<<<gb, 256, 0, st>>>(n, V, n, j + 1, dh, w, nullptr);
      A2LS_LAUNCH();
      multidot(h, V, n, j + 1, w, 0, dh + MD_MAX);        // h2
      k_cgs_update<<<gb, 256, 0, st>>>(n, V, n, j + 1, dh + MD_MAX, w, nullptr);
      A2LS_LAUNCH();
      multidot(h, V, 0, 0, w, 1, dh + 2 * MD_MAX);        // |w|^2 after orthogonalisation
      k_scale<<<gb, 256, 0, st>>>(n, w, V + (size_t)(j + 1) * n, dh + 2 * MD_MAX, 1, 0.0);
      A2LS_LAUNCH();
      A2LS_CUDA(cudaMemcpyAsync(hp, dh, sizeof(double) * 3 * MD_MAX, cudaMemcpyDeviceToHost, st));
      A2LS_CUDA(cudaStreamSynchronize(st));
      const double wnorm0 = std::sqrt(std::max(hp[j + 1], 0.0));
      double* col = &H[0];
      for (int i2 = 0; i2 <= j; ++i2) col[i2 * m + j] = hp[i2] + hp[MD_MAX + i2];
      const double hn = std::sqrt(std::max(hp[2 * MD_MAX], 0.0));
      col[(j + 1) * m + j] = hn;
      const bool breakdown = hn <= 1e-14 * wnorm0;
      for (int i2 = 0; i2 < j; ++i2) {
        const double t = cs[i2] * H[i2 * m + j] + sn[i2] * H[(i2 + 1) * m + j];
        H[(i2 + 1) * m + j] = -sn[i2] * H[i2 * m + j] + cs[i2] * H[(i2 + 1) * m + j];
        H[i2 * m + j] = t;
      }
      const double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
      cs[j] = H[j * m + j] / den;
      sn[j] = H[(j + 1) * m + j] / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      k = j + 1;
      if (std::fabs(g[j + 1]) <= rtol * bnorm || breakdown || total >= max_it) break;
    }
    for (int i2 = k - 1; i2 >= 0; --i2) {
      double s = g[i2];
      for (int c = i2 + 1; c < k; ++c) s -= H[i2 * m + c] * y[c];
      y[i2] = s / H[i2 * m + i2];
    }
    for (int i2 = 0; i2 < k; ++i2) hp[3 * MD_MAX + i2] = y[i2];
    A2LS_CUDA(cudaMemcpyAsync(dh + 3 * MD_MAX, hp + 3 * MD_MAX, sizeof(double) * k, cudaMemcpyHostToDevice, st));
    if (flexible) {
      k_lincomb<<<gb, 256, 0, st>>>(n, Zs, n, k, dh + 3 * MD_MAX, nullptr, x);
      A2LS_LAUNCH();
    } else {
      k_lincomb<<<gb, 256, 0, st>>>(n, V, n, k, dh + 3 * MD_MAX, w, nullptr);
      A2LS_LAUNCH();
      apply_preconditioner_graph(h, w, tmp);
      k_axpy<<<gb, 256, 0, st>>>(n, 1.0, tmp, x);
      A2LS_LAUNCH();
    }
    A2LS_CUDA(cudaStreamSynchronize(st));  // the host buffer hp is reused next cycle
    (void)R;
  }
}

}  // namespace a2ls

// Learned warm start of the local eigensolves: a message-passing network over
// each subdomain's local graph proposes the starting block of the block Krylov
// iteration for the eigenproblem of Eq. 3.1.  The paper has no learned part;
// this is the project's addition, trained on the GPU by the kernels below.
//
// Network (per subdomain, local matrix A_ii, lumped sums s_i of Definition 3.1):
//   w_lk = (|a_lk| + |a_kl|) / (2 sqrt(|a_ll a_kk|)) on mutual off-diagonal entries, S = D^-1/2 W D^-1/2
//   x_l  = [1, d_l / max d, clip(log(d_l / mean d) / 10, -1, 1), [overlap row], s_l / d_l, deg_l / 4]
//   h_0  = relu(x W_in + b_in); h_t = relu(h_{t-1} W_s,t + (W h_{t-1}) W_n,t + b_t), t = 1..3
//   p_0  = h_3 W_out;  p_{k+1} = (1 - alpha) S p_k + alpha p_0, k < 32;  Y = p_32  (n_i x 16)
// Loss against a target basis Z_i (n_i x m_i) of the wanted eigenspace:
//   L_i = min_C (||Z_i - Y C||^2 + eps ||C||^2) / m_i, averaged over the subdomains with a target.
// Weights are stored in bfloat16 (biases in FP32); every product accumulates in FP32, the 16 x 16
// normal equations of the loss in FP64.  Training keeps FP32 master weights and Adam moments.
//
// Data layout: the rows of all subdomains are concatenated in the local order of the handle
// (off_i + l); activations are row-major [rows x 64] FP32, outputs [rows x 16].  The graph is the
// handle's local CSR (one entry per entry of the global row) with the column replaced by the flat
// local index of the neighbour, or -1 where the entry leaves the subdomain or is not mutual.
#include "a2ls_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>

namespace a2ls {
namespace gnn {

constexpr int F_IN = 6, FX = 8, WIDTH = 64, LAYERS = 3, OUT = 16, K_PROP = 32;
constexpr float ALPHA = 0.1f;
constexpr double LOSS_EPS = 1e-6;
constexpr int OFF_WIN = 0, OFF_BIN = F_IN * WIDTH, OFF_L1 = OFF_BIN + WIDTH;
constexpr int L_STRIDE = 2 * WIDTH * WIDTH + WIDTH;
constexpr int OFF_WOUT = OFF_L1 + LAYERS * L_STRIDE;
constexpr int NP = OFF_WOUT + WIDTH * OUT;  // 26240
constexpr int MAXZ = 32;                     // largest target width m_i
constexpr int TILE = 64;                     // rows per CTA in the dense layer kernels
constexpr int AS = 132;                      // row stride of the [h | m] tile (floats)
constexpr int BS = 68;                       // row stride of the 64-wide tiles of the backward kernel

__host__ __device__ constexpr int off_ws(int t) { return OFF_L1 + (t - 1) * L_STRIDE; }
__host__ __device__ constexpr int off_wn(int t) { return off_ws(t) + WIDTH * WIDTH; }
__host__ __device__ constexpr int off_b(int t) { return off_wn(t) + WIDTH * WIDTH; }

__device__ __forceinline__ float bf(const __nv_bfloat16* w, int p) { return __bfloat162float(w[p]); }

}  // namespace gnn
}  // namespace a2ls

using namespace a2ls;
using namespace a2ls::gnn;

// ---------------------------------------------------------------------------
// host objects
// ---------------------------------------------------------------------------
struct a2ls_gnn {
  cudaStream_t st = nullptr;
  float* theta = nullptr;        // FP32 master parameters
  float* mom1 = nullptr;         // Adam first moment
  float* mom2 = nullptr;         // Adam second moment
  float* grad = nullptr;         // accumulated gradient (sum over samples)
  __nv_bfloat16* w16 = nullptr;  // bfloat16 copy used by the forward and backward kernels
  int64_t adam_t = 0;            // Adam steps taken
  int accum = 0;                 // samples accumulated in grad
  int64_t launches = 0;
};

struct a2ls_gnn_sample {
  cudaStream_t st = nullptr;
  int N = 0, S = 0;
  int64_t E = 0;
  int ntarget = 0;
  std::vector<int> h_off;
  int* off = nullptr;       // N + 1
  int64_t* rp = nullptr;    // S + 1, entries of each row
  int* col = nullptr;       // E: flat local index of the neighbour or -1
  float* w = nullptr;       // E: symmetric edge weights
  float* s = nullptr;       // E: D^-1/2 W D^-1/2
  float* X = nullptr;       // S x 8 features (columns 6, 7 zero)
  int* zm = nullptr;        // N: target widths (0 = no target)
  int64_t* zoff = nullptr;  // N + 1: offsets of the targets
  float* Z = nullptr;       // targets, n_i x m_i row-major per subdomain
  std::vector<int> h_zm;
  std::vector<void*> allocs;
};

namespace a2ls {
namespace gnn {

static void count_launch(int64_t* counter, const char* file, int line) {
  if (counter) ++*counter;
  check_cuda(cudaGetLastError(), "kernel launch", file, line);
}
#define GNN_LAUNCH(cnt) ::a2ls::gnn::count_launch((cnt), __FILE__, __LINE__)

template <class T>
static T* galloc(std::vector<void*>& list, size_t count, cudaStream_t st) {
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, std::max<size_t>(count * sizeof(T), 16), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(A2LS_ERR_OOM, "device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
  }
  list.push_back(p);
  return static_cast<T*>(p);
}

static void gfree_all(std::vector<void*>& list, cudaStream_t st) {
  for (void* p : list) cudaFreeAsync(p, st);
  list.clear();
}

// ---------------------------------------------------------------------------
// graph and features: one CTA per subdomain
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_reduce(double v, double* red, bool is_max) {
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmax(v, u) : v + u;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red[0];
  for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = is_max ? fmax(r, red[k]) : r + red[k];
  __syncthreads();
  return r;
}

// dscr, gscr: S doubles of scratch (|a_ll| and deg_l)
__global__ void k_graph_features(const int* off, const int* nI, const int64_t* lrow, const int* lcol,
                                 const double* lval, const double* lump, int* col, float* w, float* s, float* X,
                                 double* dscr, double* gscr) {
  __shared__ double red[32];
  const int i = blockIdx.x, o = off[i], n = off[i + 1] - o, n_I = nI[i];
  double dmax = 0.0, dsum = 0.0;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    double d = 0.0;
    for (int64_t e = lrow[o + l]; e < lrow[o + l + 1]; ++e)
      if (lcol[e] == l) d = fabs(lval[e]);
    dscr[o + l] = d;
    dmax = fmax(dmax, d);
    dsum += d;
  }
  dmax = block_reduce(dmax, red, true);
  dsum = block_reduce(dsum, red, false);
  const double dmean = dsum / n;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    const double dl = dscr[o + l];
    double deg = 0.0;
    for (int64_t e = lrow[o + l]; e < lrow[o + l + 1]; ++e) {
      const int k = lcol[e];
      const double a = lval[e];
      double wv = 0.0;
      int c = -1;
      if (k >= 0 && k != l && a != 0.0 && dl > 0.0) {
        const double dk = dscr[o + k];
        double akl = 0.0;
        for (int64_t q = lrow[o + k]; q < lrow[o + k + 1]; ++q)
          if (lcol[q] == l) akl = lval[q];
        if (akl != 0.0 && dk > 0.0) {
          wv = (fabs(a) + fabs(akl)) / (2.0 * sqrt(dl * dk));
          c = o + k;
        }
      }
      col[e] = c;
      w[e] = (float)wv;
      deg += wv;
    }
    gscr[o + l] = deg;
    float* x = X + (int64_t)(o + l) * FX;
    x[0] = 1.f;
    x[1] = dmax > 0.0 ? (float)(dl / dmax) : 0.f;
    x[2] = dl > 0.0 ? (dmean > 0.0 ? (float)fmin(1.0, fmax(-1.0, log(dl / dmean) / 10.0)) : 0.f) : -1.f;
    x[3] = l >= n_I ? 1.f : 0.f;
    x[4] = dl > 0.0 ? (float)(lump[o + l] / dl) : 0.f;
    x[5] = (float)(deg / 4.0);
    x[6] = 0.f;
    x[7] = 0.f;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    const double gl = gscr[o + l];
    for (int64_t e = lrow[o + l]; e < lrow[o + l + 1]; ++e) {
      const int c = col[e];
      s[e] = c >= 0 ? (float)((double)w[e] / sqrt(gl * gscr[c])) : 0.f;
    }
  }
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
__global__ void k_layer0_fwd(int S, const float* __restrict__ X, const __nv_bfloat16* __restrict__ w16,
                             const float* __restrict__ theta, float* __restrict__ h0) {
  __shared__ float Win[F_IN * WIDTH], bin[WIDTH];
  for (int e = threadIdx.x; e < F_IN * WIDTH; e += blockDim.x) Win[e] = bf(w16, OFF_WIN + e);
  if (threadIdx.x < WIDTH) bin[threadIdx.x] = theta[OFF_BIN + threadIdx.x];
  __syncthreads();
  const int64_t total = (int64_t)S * WIDTH;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / WIDTH;
    const int j = (int)(e % WIDTH);
    float a = bin[j];
#pragma unroll
    for (int f = 0; f < F_IN; ++f) a = fmaf(X[r * FX + f], Win[f * WIDTH + j], a);
    h0[e] = fmaxf(a, 0.f);
  }
}

// h_t = relu([h_{t-1} | W h_{t-1}] [W_s; W_n] + b) for 64 rows per CTA; LAST also forms p_0 = h_3 W_out.
// TRAIN stores m_t = W h_{t-1} for the backward pass.
template <bool TRAIN, bool LAST>
__global__ void __launch_bounds__(256) k_layer_fwd(int S, const int64_t* __restrict__ rp, const int* __restrict__ col,
                                                   const float* __restrict__ w, const float* __restrict__ hin,
                                                   const __nv_bfloat16* __restrict__ w16,
                                                   const float* __restrict__ theta, int t, float* __restrict__ hout,
                                                   float* __restrict__ mout, float* __restrict__ p0) {
  extern __shared__ __align__(16) float sm[];
  float* A = sm;                     // TILE x AS: [h | m]
  float* Wt = A + TILE * AS;         // 128 x 64: [W_s; W_n]
  float* bias = Wt + 2 * WIDTH * WIDTH;
  float* Wo = bias + WIDTH;          // 64 x 16 (LAST)
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * TILE;
  const int ows = off_ws(t), own = off_wn(t);
  for (int e = tid; e < 2 * WIDTH * WIDTH; e += 256) {
    const int k = e / WIDTH, j = e % WIDTH;
    Wt[e] = bf(w16, (k < WIDTH ? ows + k * WIDTH : own + (k - WIDTH) * WIDTH) + j);
  }
  if (tid < WIDTH) bias[tid] = theta[off_b(t) + tid];
  if (LAST)
    for (int e = tid; e < WIDTH * OUT; e += 256) Wo[e] = bf(w16, OFF_WOUT + e);
  for (int e = tid; e < TILE * (WIDTH / 4); e += 256) {
    const int r = e / (WIDTH / 4), q = e % (WIDTH / 4);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r0 + r < S) v = __ldg(reinterpret_cast<const float4*>(hin + (int64_t)(r0 + r) * WIDTH) + q);
    *reinterpret_cast<float4*>(A + r * AS + q * 4) = v;
  }
  {
    // m = W h_{t-1}: 4 threads per row, 16 columns each
    const int r = tid >> 2, c0 = (tid & 3) * 16;
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.f;
    const int row = r0 + r;
    if (row < S) {
      for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
        const int k = col[e];
        if (k < 0) continue;
        const float we = w[e];
        const float4* src = reinterpret_cast<const float4*>(hin + (int64_t)k * WIDTH + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 v = __ldg(src + q);
          acc[4 * q] = fmaf(we, v.x, acc[4 * q]);
          acc[4 * q + 1] = fmaf(we, v.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(we, v.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(we, v.w, acc[4 * q + 3]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
      *reinterpret_cast<float4*>(A + r * AS + WIDTH + c0 + 4 * q) = v;
      if (TRAIN && row < S) *reinterpret_cast<float4*>(mout + (int64_t)row * WIDTH + c0 + 4 * q) = v;
    }
  }
  __syncthreads();
  const int ty = tid >> 4, tx = tid & 15;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = bias[tx * 4 + j];
#pragma unroll 4
  for (int k = 0; k < 2 * WIDTH; ++k) {
    const float4 b = *reinterpret_cast<const float4*>(Wt + k * WIDTH + tx * 4);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float a = A[(ty * 4 + i) * AS + k];
      acc[i][0] = fmaf(a, b.x, acc[i][0]);
      acc[i][1] = fmaf(a, b.y, acc[i][1]);
      acc[i][2] = fmaf(a, b.z, acc[i][2]);
      acc[i][3] = fmaf(a, b.w, acc[i][3]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = fmaxf(acc[i][j], 0.f);
    const int row = r0 + ty * 4 + i;
    if (row < S)
      *reinterpret_cast<float4*>(hout + (int64_t)row * WIDTH + tx * 4) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
  if (LAST) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<float4*>(A + (ty * 4 + i) * AS + tx * 4) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    __syncthreads();
    const int r = tid >> 2, c0 = (tid & 3) * 4;
    float o4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int k = 0; k < WIDTH; ++k) {
      const float a = A[r * AS + k];
      const float4 b = *reinterpret_cast<const float4*>(Wo + k * OUT + c0);
      o4[0] = fmaf(a, b.x, o4[0]);
      o4[1] = fmaf(a, b.y, o4[1]);
      o4[2] = fmaf(a, b.z, o4[2]);
      o4[3] = fmaf(a, b.w, o4[3]);
    }
    if (r0 + r < S)
      *reinterpret_cast<float4*>(p0 + (int64_t)(r0 + r) * OUT + c0) = make_float4(o4[0], o4[1], o4[2], o4[3]);
  }
}

// K_PROP steps of the propagation on one subdomain per CTA (16 threads per row, one per column).
// Forward (ADJ = false): p_{k+1} = (1 - alpha) S p_k + alpha p_0, p_0 = in, out = p_K.
// Adjoint (ADJ = true): the gradient with respect to p_0 of <p_K, in>; S is symmetric, so
// with g_0 = in: acc += alpha g_k, g_{k+1} = (1 - alpha) S g_k, out = g_K + acc.
// bufA, bufB, acc: scratch of the same shape as in (rows x 16).
template <bool ADJ>
__global__ void __launch_bounds__(256) k_propagate(const int* off, const int64_t* __restrict__ rp,
                                                   const int* __restrict__ col, const float* __restrict__ s,
                                                   const float* in, float* bufA, float* bufB, float* accb,
                                                   float* out) {
  const int i = blockIdx.x, o = off[i], n = off[i + 1] - o;
  const int c = threadIdx.x & 15, rr = threadIdx.x >> 4;
  const float* src = in;
  for (int k = 0; k < K_PROP; ++k) {
    float* dst = (k == K_PROP - 1) ? out : ((k & 1) ? bufB : bufA);
    for (int l = o + rr; l < o + n; l += 16) {
      float a = 0.f;
      for (int64_t e = rp[l]; e < rp[l + 1]; ++e) {
        const int q = col[e];
        if (q >= 0) a = fmaf(s[e], src[(int64_t)q * OUT + c], a);
      }
      const int64_t at = (int64_t)l * OUT + c;
      if (!ADJ) {
        dst[at] = (1.f - ALPHA) * a + ALPHA * in[at];
      } else {
        const float av = (k == 0 ? 0.f : accb[at]) + ALPHA * src[at];
        if (k == K_PROP - 1) dst[at] = (1.f - ALPHA) * a + av;
        else {
          accb[at] = av;
          dst[at] = (1.f - ALPHA) * a;
        }
      }
    }
    __syncthreads();
    src = dst;
  }
}

// ---------------------------------------------------------------------------
// loss: one CTA per subdomain
// ---------------------------------------------------------------------------
// Solves (Y^T Y + eps I) C = Y^T Z, R = Z - Y C, L_i = (||R||^2 + eps ||C||^2) / m,
// dY = -2 R C^T / m * scale (scale = 1 / number of subdomains with a target).
__global__ void __launch_bounds__(256) k_loss(const int* off, const int* zm, const int64_t* zoff,
                                              const float* __restrict__ Z, const float* __restrict__ Y, float scale,
                                              double* loss_i, float* dY) {
  __shared__ float Ys[TILE][OUT + 1];
  __shared__ float Zs[TILE][MAXZ + 1];
  __shared__ double G[OUT * OUT], B[OUT * MAXZ], red[32];
  __shared__ int okflag;
  const int i = blockIdx.x, o = off[i], n = off[i + 1] - o, m = zm[i], tid = threadIdx.x;
  if (m == 0) {
    for (int e = tid; e < n * OUT; e += blockDim.x) dY[(int64_t)o * OUT + e] = 0.f;
    if (tid == 0) loss_i[i] = 0.0;
    return;
  }
  const float* Zi = Z + zoff[i];
  const int nout = OUT * OUT + OUT * m;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int r0 = 0; r0 < n; r0 += TILE) {
    const int rows = min(TILE, n - r0);
    for (int e = tid; e < TILE * OUT; e += blockDim.x) {
      const int r = e / OUT, c = e % OUT;
      Ys[r][c] = r < rows ? Y[(int64_t)(o + r0 + r) * OUT + c] : 0.f;
    }
    for (int e = tid; e < TILE * m; e += blockDim.x) {
      const int r = e / m, c = e % m;
      Zs[r][c] = r < rows ? Zi[(int64_t)(r0 + r) * m + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int q = tid + 256 * k;
      if (q >= nout) break;
      double a = 0.0;
      if (q < OUT * OUT) {
        const int j1 = q / OUT, j2 = q % OUT;
        for (int r = 0; r < rows; ++r) a += (double)Ys[r][j1] * (double)Ys[r][j2];
      } else {
        const int j = (q - OUT * OUT) / m, c = (q - OUT * OUT) % m;
        for (int r = 0; r < rows; ++r) a += (double)Ys[r][j] * (double)Zs[r][c];
      }
      acc[k] += a;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int q = tid + 256 * k;
    if (q < OUT * OUT) G[q] = acc[k] + ((q / OUT == q % OUT) ? LOSS_EPS : 0.0);
    else if (q < nout) B[q - OUT * OUT] = acc[k];
  }
  __syncthreads();
  if (tid == 0) {
    // Cholesky G = L L^T in place (lower triangle)
    int ok = 1;
    for (int j = 0; j < OUT; ++j) {
      double d = G[j * OUT + j];
      for (int k = 0; k < j; ++k) d -= G[j * OUT + k] * G[j * OUT + k];
      if (!(d > 0.0)) { ok = 0; d = 1e-300; }
      d = sqrt(d);
      G[j * OUT + j] = d;
      for (int r = j + 1; r < OUT; ++r) {
        double v = G[r * OUT + j];
        for (int k = 0; k < j; ++k) v -= G[r * OUT + k] * G[j * OUT + k];
        G[r * OUT + j] = v / d;
      }
    }
    okflag = ok;
  }
  __syncthreads();
  if (tid < m) {
    // C[:, c] = L^-T L^-1 B[:, c], in place in B
    const int c = tid;
    for (int j = 0; j < OUT; ++j) {
      double v = B[j * m + c];
      for (int k = 0; k < j; ++k) v -= G[j * OUT + k] * B[k * m + c];
      B[j * m + c] = v / G[j * OUT + j];
    }
    for (int j = OUT - 1; j >= 0; --j) {
      double v = B[j * m + c];
      for (int k = j + 1; k < OUT; ++k) v -= G[k * OUT + j] * B[k * m + c];
      B[j * m + c] = v / G[j * OUT + j];
    }
  }
  __syncthreads();
  double rsq = 0.0;
  const float f = -2.f / (float)m * scale;
  for (int l = tid; l < n; l += blockDim.x) {
    float y[OUT];
    double dy[OUT];
#pragma unroll
    for (int j = 0; j < OUT; ++j) {
      y[j] = Y[(int64_t)(o + l) * OUT + j];
      dy[j] = 0.0;
    }
    for (int c = 0; c < m; ++c) {
      double r = Zi[(int64_t)l * m + c];
#pragma unroll
      for (int j = 0; j < OUT; ++j) r -= (double)y[j] * B[j * m + c];
      rsq += r * r;
#pragma unroll
      for (int j = 0; j < OUT; ++j) dy[j] += r * B[j * m + c];
    }
#pragma unroll
    for (int j = 0; j < OUT; ++j) dY[(int64_t)(o + l) * OUT + j] = f * (float)dy[j];
  }
  double csq = 0.0;
  for (int e = tid; e < OUT * m; e += blockDim.x) csq += B[e] * B[e];
  rsq = block_reduce(rsq, red, false);
  csq = block_reduce(csq, red, false);
  if (tid == 0) loss_i[i] = okflag ? (rsq + LOSS_EPS * csq) / m : NAN;
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
// Layer t in reverse.  dh_t = dp_0 W_out^T (FIRST, t = 3) or v_{t+1} + W u_{t+1}; dpre = dh_t * [h_t > 0];
// dW_s,t += h_{t-1}^T dpre, dW_n,t += m_t^T dpre, db_t += sum dpre, (FIRST) dW_out += h_3^T dp_0;
// v_t = dpre W_s,t^T, u_t = dpre W_n,t^T.  Persistent CTAs over 64-row tiles; each CTA writes its
// partial gradient of the parameters of the layer into part[blockIdx.x * NP + ...].
template <bool FIRST>
__global__ void __launch_bounds__(256) k_layer_bwd(int S, const int64_t* __restrict__ rp, const int* __restrict__ col,
                                                   const float* __restrict__ w, const float* __restrict__ hprev,
                                                   const float* __restrict__ mt, const float* __restrict__ ht,
                                                   const float* __restrict__ dp0, const float* __restrict__ vin,
                                                   const float* __restrict__ uin,
                                                   const __nv_bfloat16* __restrict__ w16, int t,
                                                   float* __restrict__ vout, float* __restrict__ uout,
                                                   float* __restrict__ part) {
  extern __shared__ __align__(16) float sm[];
  float* Hp = sm;                    // TILE x BS
  float* Mt = Hp + TILE * BS;        // TILE x BS
  float* D = Mt + TILE * BS;         // TILE x BS
  float* WsT = D + TILE * BS;        // 64 x 64, WsT[j][k] = W_s[k][j]
  float* WnT = WsT + WIDTH * WIDTH;
  float* Ht = WnT + WIDTH * WIDTH;   // FIRST: TILE x BS
  float* P0 = Ht + TILE * BS;        // FIRST: TILE x 16
  float* WoT = P0 + TILE * OUT;      // FIRST: 16 x 64, WoT[c][k] = W_out[k][c]
  const int tid = threadIdx.x;
  const int ows = off_ws(t), own = off_wn(t);
  for (int e = tid; e < WIDTH * WIDTH; e += 256) {
    const int j = e / WIDTH, k = e % WIDTH;
    WsT[e] = bf(w16, ows + k * WIDTH + j);
    WnT[e] = bf(w16, own + k * WIDTH + j);
  }
  if (FIRST)
    for (int e = tid; e < OUT * WIDTH; e += 256) {
      const int c = e / WIDTH, k = e % WIDTH;
      WoT[e] = bf(w16, OFF_WOUT + k * OUT + c);
    }
  const int ty = tid >> 4, tx = tid & 15;
  float gs[4][4], gn[4][4], go[4] = {0.f, 0.f, 0.f, 0.f}, gb = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) gs[i][j] = gn[i][j] = 0.f;
  const int tiles = (S + TILE - 1) / TILE;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int r0 = tile * TILE;
    __syncthreads();
    for (int e = tid; e < TILE * (WIDTH / 4); e += 256) {
      const int r = e / (WIDTH / 4), q = e % (WIDTH / 4);
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, c = a;
      if (r0 + r < S) {
        a = __ldg(reinterpret_cast<const float4*>(hprev + (int64_t)(r0 + r) * WIDTH) + q);
        b = __ldg(reinterpret_cast<const float4*>(mt + (int64_t)(r0 + r) * WIDTH) + q);
        if (FIRST) c = __ldg(reinterpret_cast<const float4*>(ht + (int64_t)(r0 + r) * WIDTH) + q);
      }
      *reinterpret_cast<float4*>(Hp + r * BS + q * 4) = a;
      *reinterpret_cast<float4*>(Mt + r * BS + q * 4) = b;
      if (FIRST) *reinterpret_cast<float4*>(Ht + r * BS + q * 4) = c;
    }
    if (FIRST)
      for (int e = tid; e < TILE * OUT; e += 256) {
        const int r = e / OUT;
        P0[e] = (r0 + r < S) ? dp0[(int64_t)r0 * OUT + e] : 0.f;
      }
    __syncthreads();
    {
      // dpre for row r, columns k0 .. k0 + 15
      const int r = tid >> 2, k0 = (tid & 3) * 16, row = r0 + r;
      float dh[16];
      if (FIRST) {
#pragma unroll
        for (int k = 0; k < 16; ++k) dh[k] = 0.f;
#pragma unroll
        for (int c = 0; c < OUT; ++c) {
          const float p = P0[r * OUT + c];
#pragma unroll
          for (int k = 0; k < 16; ++k) dh[k] = fmaf(p, WoT[c * WIDTH + k0 + k], dh[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) dh[k] = 0.f;
        if (row < S) {
          const float4* vr = reinterpret_cast<const float4*>(vin + (int64_t)row * WIDTH + k0);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 v = __ldg(vr + q);
            dh[4 * q] = v.x;
            dh[4 * q + 1] = v.y;
            dh[4 * q + 2] = v.z;
            dh[4 * q + 3] = v.w;
          }
          for (int64_t e = rp[row]; e < rp[row + 1]; ++e) {
            const int nb = col[e];
            if (nb < 0) continue;
            const float we = w[e];
            const float4* ur = reinterpret_cast<const float4*>(uin + (int64_t)nb * WIDTH + k0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 u = __ldg(ur + q);
              dh[4 * q] = fmaf(we, u.x, dh[4 * q]);
              dh[4 * q + 1] = fmaf(we, u.y, dh[4 * q + 1]);
              dh[4 * q + 2] = fmaf(we, u.z, dh[4 * q + 2]);
              dh[4 * q + 3] = fmaf(we, u.w, dh[4 * q + 3]);
            }
          }
        }
      }
      float hv[16];
      if (FIRST) {
#pragma unroll
        for (int k = 0; k < 16; ++k) hv[k] = Ht[r * BS + k0 + k];
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (row < S) v = __ldg(reinterpret_cast<const float4*>(ht + (int64_t)row * WIDTH + k0) + q);
          hv[4 * q] = v.x;
          hv[4 * q + 1] = v.y;
          hv[4 * q + 2] = v.z;
          hv[4 * q + 3] = v.w;
        }
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) D[r * BS + k0 + k] = (row < S && hv[k] > 0.f) ? dh[k] : 0.f;
    }
    __syncthreads();
    // v = D W_s^T, u = D W_n^T
    float av[4][4], au[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) av[i][j] = au[i][j] = 0.f;
#pragma unroll 4
    for (int j = 0; j < WIDTH; ++j) {
      const float4 bs = *reinterpret_cast<const float4*>(WsT + j * WIDTH + tx * 4);
      const float4 bn = *reinterpret_cast<const float4*>(WnT + j * WIDTH + tx * 4);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float d = D[(ty * 4 + i) * BS + j];
        av[i][0] = fmaf(d, bs.x, av[i][0]);
        av[i][1] = fmaf(d, bs.y, av[i][1]);
        av[i][2] = fmaf(d, bs.z, av[i][2]);
        av[i][3] = fmaf(d, bs.w, av[i][3]);
        au[i][0] = fmaf(d, bn.x, au[i][0]);
        au[i][1] = fmaf(d, bn.y, au[i][1]);
        au[i][2] = fmaf(d, bn.z, au[i][2]);
        au[i][3] = fmaf(d, bn.w, au[i][3]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = r0 + ty * 4 + i;
      if (row < S) {
        *reinterpret_cast<float4*>(vout + (int64_t)row * WIDTH + tx * 4) =
            make_float4(av[i][0], av[i][1], av[i][2], av[i][3]);
        *reinterpret_cast<float4*>(uout + (int64_t)row * WIDTH + tx * 4) =
            make_float4(au[i][0], au[i][1], au[i][2], au[i][3]);
      }
    }
    // weight gradients: rows k = ty*4 + i of W, columns j = tx*4 + jj
#pragma unroll 4
    for (int r = 0; r < TILE; ++r) {
      const float4 hp = *reinterpret_cast<const float4*>(Hp + r * BS + ty * 4);
      const float4 mm = *reinterpret_cast<const float4*>(Mt + r * BS + ty * 4);
      const float4 d = *reinterpret_cast<const float4*>(D + r * BS + tx * 4);
      const float ha[4] = {hp.x, hp.y, hp.z, hp.w}, ma[4] = {mm.x, mm.y, mm.z, mm.w};
      const float da[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          gs[i][j] = fmaf(ha[i], da[j], gs[i][j]);
          gn[i][j] = fmaf(ma[i], da[j], gn[i][j]);
        }
    }
    if (tid < WIDTH)
      for (int r = 0; r < TILE; ++r) gb += D[r * BS + tid];
    if (FIRST) {
      const int k = tid >> 2, c0 = (tid & 3) * 4;
      for (int r = 0; r < TILE; ++r) {
        const float hk = Ht[r * BS + k];
#pragma unroll
        for (int c = 0; c < 4; ++c) go[c] = fmaf(hk, P0[r * OUT + c0 + c], go[c]);
      }
    }
  }
  float* pp = part + (int64_t)blockIdx.x * NP;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      pp[ows + (ty * 4 + i) * WIDTH + tx * 4 + j] = gs[i][j];
      pp[own + (ty * 4 + i) * WIDTH + tx * 4 + j] = gn[i][j];
    }
  if (tid < WIDTH) pp[off_b(t) + tid] = gb;
  if (FIRST) {
    const int k = tid >> 2, c0 = (tid & 3) * 4;
#pragma unroll
    for (int c = 0; c < 4; ++c) pp[OFF_WOUT + k * OUT + c0 + c] = go[c];
  }
}

// Input layer in reverse: dh_0 = v_1 + W u_1, dpre = dh_0 * [h_0 > 0], dW_in += x^T dpre, db_in += sum dpre.
__global__ void __launch_bounds__(256) k_layer0_bwd(int S, const int64_t* __restrict__ rp, const int* __restrict__ col,
                                                    const float* __restrict__ w, const float* __restrict__ X,
                                                    const float* __restrict__ h0, const float* __restrict__ v1,
                                                    const float* __restrict__ u1, float* __restrict__ part) {
  __shared__ float red[4][F_IN + 1][WIDTH];
  const int j = threadIdx.x & (WIDTH - 1), g = threadIdx.x >> 6;
  float gw[F_IN + 1];
#pragma unroll
  for (int f = 0; f <= F_IN; ++f) gw[f] = 0.f;
  for (int r = blockIdx.x * 4 + g; r < S; r += gridDim.x * 4) {
    float dh = v1[(int64_t)r * WIDTH + j];
    for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
      const int nb = col[e];
      if (nb >= 0) dh = fmaf(w[e], u1[(int64_t)nb * WIDTH + j], dh);
    }
    const float d = h0[(int64_t)r * WIDTH + j] > 0.f ? dh : 0.f;
#pragma unroll
    for (int f = 0; f < F_IN; ++f) gw[f] = fmaf(X[(int64_t)r * FX + f], d, gw[f]);
    gw[F_IN] += d;
  }
#pragma unroll
  for (int f = 0; f <= F_IN; ++f) red[g][f][j] = gw[f];
  __syncthreads();
  float* pp = part + (int64_t)blockIdx.x * NP;
  for (int e = threadIdx.x; e < (F_IN + 1) * WIDTH; e += blockDim.x) {
    const int f = e / WIDTH, jj = e % WIDTH;
    const float v = red[0][f][jj] + red[1][f][jj] + red[2][f][jj] + red[3][f][jj];
    if (f < F_IN) pp[OFF_WIN + f * WIDTH + jj] = v;
    else pp[OFF_BIN + jj] = v;
  }
}

// grad[p] += sum over the CTAs of part[c][p], in CTA order
__global__ void k_reduce_parts(int nparts, const float* __restrict__ part, float* grad) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += gridDim.x * blockDim.x) {
    float a = 0.f;
    for (int c = 0; c < nparts; ++c) a += part[(int64_t)c * NP + p];
    grad[p] += a;
  }
}

// Adam (Kingma and Ba, 2015, Algorithm 1) on the mean of the accumulated gradients; refreshes the
// bfloat16 copy and clears the accumulator.
__global__ void k_adam(float* theta, float* m1, float* m2, float* grad, __nv_bfloat16* w16, float inv_count,
                       float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += gridDim.x * blockDim.x) {
    const float g = grad[p] * inv_count;
    const float a = b1 * m1[p] + (1.f - b1) * g;
    const float b = b2 * m2[p] + (1.f - b2) * g * g;
    m1[p] = a;
    m2[p] = b;
    const float th = theta[p] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    theta[p] = th;
    w16[p] = __float2bfloat16_rn(th);
    grad[p] = 0.f;
  }
}

__global__ void k_refresh_w16(const float* theta, __nv_bfloat16* w16) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += gridDim.x * blockDim.x)
    w16[p] = __float2bfloat16_rn(theta[p]);
}

__global__ void k_target_from_handle(const int* off, const int64_t* hzoff, int zld, const double* Zh,
                                     const int* zm, const int64_t* zoff, float* Z) {
  const int i = blockIdx.x, n = off[i + 1] - off[i], m = zm[i];
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
    const int l = e / m, c = e % m;
    Z[zoff[i] + e] = (float)Zh[hzoff[i] + (int64_t)l * zld + c];
  }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
constexpr size_t FWD_SMEM = sizeof(float) * (TILE * AS + 2 * WIDTH * WIDTH + WIDTH + WIDTH * OUT);
constexpr size_t BWD_SMEM = sizeof(float) * (3 * TILE * BS + 2 * WIDTH * WIDTH);
constexpr size_t BWD1_SMEM = BWD_SMEM + sizeof(float) * (TILE * BS + TILE * OUT + OUT * WIDTH);

static void set_smem_limits() {
  static bool done = false;  // attribute set once per process (same value every time)
  if (done) return;
  A2LS_CUDA(cudaFuncSetAttribute(k_layer_fwd<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FWD_SMEM));
  A2LS_CUDA(cudaFuncSetAttribute(k_layer_fwd<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FWD_SMEM));
  A2LS_CUDA(cudaFuncSetAttribute(k_layer_fwd<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FWD_SMEM));
  A2LS_CUDA(cudaFuncSetAttribute(k_layer_fwd<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FWD_SMEM));
  A2LS_CUDA(cudaFuncSetAttribute(k_layer_bwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BWD1_SMEM));
  A2LS_CUDA(cudaFuncSetAttribute(k_layer_bwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BWD_SMEM));
  done = true;
}

// graph arrays describing rows [0, S) in the flat local order
struct Graph {
  int N, S;
  const int* off;
  const int64_t* rp;
  const int* col;
  const float* w;
  const float* s;
  const float* X;
};

// activations of one forward pass; h[0..3] and m[1..3] are kept only when training
struct Acts {
  float* h[4] = {nullptr, nullptr, nullptr, nullptr};
  float* m[4] = {nullptr, nullptr, nullptr, nullptr};
  float* p0 = nullptr;
  float* Y = nullptr;
  float* pa = nullptr;
  float* pb = nullptr;
};

static void build_graph(cudaStream_t st, int64_t* cnt, int N, const int* off, const int* nI, const int64_t* lrow,
                        const int* lcol, const double* lval, const double* lump, int S, int* col, float* w,
                        float* s, float* X, std::vector<void*>& tmp) {
  double* dscr = galloc<double>(tmp, S, st);
  double* gscr = galloc<double>(tmp, S, st);
  k_graph_features<<<N, 256, 0, st>>>(off, nI, lrow, lcol, lval, lump, col, w, s, X, dscr, gscr);
  GNN_LAUNCH(cnt);
}

static void forward(cudaStream_t st, int64_t* cnt, const Graph& g, const __nv_bfloat16* w16, const float* theta,
                    bool train, Acts& a) {
  set_smem_limits();
  const int S = g.S;
  const int tiles = (S + TILE - 1) / TILE;
  const int g0 = std::min(152 * 8, std::max(1, ceil_div((int64_t)S * WIDTH, 256)));
  k_layer0_fwd<<<g0, 256, 0, st>>>(S, g.X, w16, theta, a.h[0]);
  GNN_LAUNCH(cnt);
  for (int t = 1; t <= LAYERS; ++t) {
    // inference ping-pongs between h[0] and h[1]
    const float* hin = train ? a.h[t - 1] : a.h[(t - 1) & 1];
    float* hout = train ? a.h[t] : a.h[t & 1];
    float* mout = train ? a.m[t] : nullptr;
    if (t < LAYERS) {
      if (train)
        k_layer_fwd<true, false><<<tiles, 256, FWD_SMEM, st>>>(S, g.rp, g.col, g.w, hin, w16, theta, t, hout, mout, nullptr);
      else
        k_layer_fwd<false, false><<<tiles, 256, FWD_SMEM, st>>>(S, g.rp, g.col, g.w, hin, w16, theta, t, hout, mout, nullptr);
    } else {
      if (train)
        k_layer_fwd<true, true><<<tiles, 256, FWD_SMEM, st>>>(S, g.rp, g.col, g.w, hin, w16, theta, t, hout, mout, a.p0);
      else
        k_layer_fwd<false, true><<<tiles, 256, FWD_SMEM, st>>>(S, g.rp, g.col, g.w, hin, w16, theta, t, hout, mout, a.p0);
    }
    GNN_LAUNCH(cnt);
  }
  k_propagate<false><<<g.N, 256, 0, st>>>(g.off, g.rp, g.col, g.s, a.p0, a.pa, a.pb, nullptr, a.Y);
  GNN_LAUNCH(cnt);
}

static void alloc_acts(std::vector<void*>& tmp, cudaStream_t st, int S, bool train, Acts& a) {
  const size_t hs = (size_t)S * WIDTH, ps = (size_t)S * OUT;
  const int nh = train ? 4 : 2;
  for (int k = 0; k < nh; ++k) a.h[k] = galloc<float>(tmp, hs, st);
  if (train)
    for (int k = 1; k <= LAYERS; ++k) a.m[k] = galloc<float>(tmp, hs, st);
  a.p0 = galloc<float>(tmp, ps, st);
  a.Y = galloc<float>(tmp, ps, st);
  a.pa = galloc<float>(tmp, ps, st);
  a.pb = galloc<float>(tmp, ps, st);
}

static Graph sample_graph(const a2ls_gnn_sample* s) { return Graph{s->N, s->S, s->off, s->rp, s->col, s->w, s->s, s->X}; }

}  // namespace gnn

// Inference for the warm start of the eigensolver: Y (sum n_i x 16, FP32, caller-allocated through the
// handle) for the handle's subdomains.
void gnn_infer(a2ls_handle* h, const a2ls_gnn* model, float* Y) {
  using namespace gnn;
  cudaStream_t st = h->st;
  std::vector<void*> tmp;
  try {
    const int S = h->sum_n;
    int64_t ecount = 0;
    A2LS_CUDA(cudaMemcpyAsync(&ecount, h->d_lrow + S, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    A2LS_CUDA(cudaStreamSynchronize(st));
    int* col = galloc<int>(tmp, ecount, st);
    float* w = galloc<float>(tmp, ecount, st);
    float* sv = galloc<float>(tmp, ecount, st);
    float* X = galloc<float>(tmp, (size_t)S * FX, st);
    build_graph(st, &h->launches, h->N, h->d_off, h->d_nI, h->d_lrow, h->d_lcol, h->d_lval, h->d_lump, S, col, w,
                sv, X, tmp);
    Graph g{h->N, S, h->d_off, h->d_lrow, col, w, sv, X};
    Acts a;
    alloc_acts(tmp, st, S, false, a);
    forward(st, &h->launches, g, model->w16, model->theta, false, a);
    A2LS_CUDA(cudaMemcpyAsync(Y, a.Y, sizeof(float) * S * OUT, cudaMemcpyDeviceToDevice, st));
    gfree_all(tmp, st);
  } catch (...) {
    gfree_all(tmp, st);
    throw;
  }
}

void record_error(const char* msg);

}  // namespace a2ls

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {

template <class F>
int gnn_guarded(F&& f) {
  try {
    return f();
  } catch (const a2ls::Error& e) {
    a2ls::record_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    a2ls::record_error(e.what());
    return A2LS_ERR_CUDA;
  } catch (...) {
    a2ls::record_error("unknown error");
    return A2LS_ERR_CUDA;
  }
}

int gnn_fail(int code, const char* msg) {
  a2ls::record_error(msg);
  return code;
}

void destroy_model(a2ls_gnn* g) {
  if (!g) return;
  cudaStream_t st = g->st;
  for (void* p : {(void*)g->theta, (void*)g->mom1, (void*)g->mom2, (void*)g->grad, (void*)g->w16})
    if (p) cudaFreeAsync(p, st);
  cudaStreamSynchronize(st);
  delete g;
}

void destroy_sample(a2ls_gnn_sample* s) {
  if (!s) return;
  a2ls::gnn::gfree_all(s->allocs, s->st);
  cudaStreamSynchronize(s->st);
  delete s;
}

// He-normal initial weights (std sqrt(2 / fan_in)), zero biases, from a 64-bit Mersenne twister and
// the Box-Muller transform
std::vector<float> initial_params(uint64_t seed) {
  using namespace a2ls::gnn;
  std::mt19937_64 rng(seed);
  auto unif = [&]() { return ((rng() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
  auto normal = [&]() { return std::sqrt(-2.0 * std::log(unif())) * std::cos(6.283185307179586 * unif()); };
  std::vector<float> p(NP, 0.f);
  auto fill = [&](int off, int rows, int cols) {
    const double sd = std::sqrt(2.0 / rows);
    for (int e = 0; e < rows * cols; ++e) p[off + e] = (float)(sd * normal());
  };
  fill(OFF_WIN, F_IN, WIDTH);
  for (int t = 1; t <= LAYERS; ++t) {
    fill(off_ws(t), WIDTH, WIDTH);
    fill(off_wn(t), WIDTH, WIDTH);
  }
  fill(OFF_WOUT, WIDTH, OUT);
  return p;
}

void upload_params(a2ls_gnn* g, const float* host) {
  using namespace a2ls;
  using namespace a2ls::gnn;
  A2LS_CUDA(cudaMemcpyAsync(g->theta, host, sizeof(float) * NP, cudaMemcpyHostToDevice, g->st));
  A2LS_CUDA(cudaMemsetAsync(g->mom1, 0, sizeof(float) * NP, g->st));
  A2LS_CUDA(cudaMemsetAsync(g->mom2, 0, sizeof(float) * NP, g->st));
  A2LS_CUDA(cudaMemsetAsync(g->grad, 0, sizeof(float) * NP, g->st));
  k_refresh_w16<<<ceil_div(NP, 256), 256, 0, g->st>>>(g->theta, g->w16);
  GNN_LAUNCH(&g->launches);
  A2LS_CUDA(cudaStreamSynchronize(g->st));
  g->adam_t = 0;
  g->accum = 0;
}

}  // namespace

extern "C" {

int64_t a2ls_gnn_num_params(void) { return a2ls::gnn::NP; }

int a2ls_gnn_create(uint64_t seed, void* stream, a2ls_gnn** out) {
  using namespace a2ls::gnn;
  if (!out) return gnn_fail(A2LS_ERR_ARG, "null argument");
  *out = nullptr;
  a2ls_gnn* g = new a2ls_gnn();
  g->st = static_cast<cudaStream_t>(stream);
  int rc = gnn_guarded([&]() -> int {
    std::vector<void*> list;
    g->theta = galloc<float>(list, NP, g->st);
    g->mom1 = galloc<float>(list, NP, g->st);
    g->mom2 = galloc<float>(list, NP, g->st);
    g->grad = galloc<float>(list, NP, g->st);
    g->w16 = galloc<__nv_bfloat16>(list, NP, g->st);
    const std::vector<float> p = initial_params(seed);
    upload_params(g, p.data());
    return A2LS_OK;
  });
  if (rc != A2LS_OK) {
    destroy_model(g);
    return rc;
  }
  *out = g;
  return A2LS_OK;
}

int a2ls_gnn_destroy(a2ls_gnn* g) {
  destroy_model(g);
  return A2LS_OK;
}

int a2ls_gnn_get_params(a2ls_gnn* g, float* host, int64_t count) {
  using namespace a2ls;
  if (!g || !host) return gnn_fail(A2LS_ERR_ARG, "null argument");
  if (count != gnn::NP) return gnn_fail(A2LS_ERR_ARG, "count must equal a2ls_gnn_num_params()");
  return gnn_guarded([&]() -> int {
    A2LS_CUDA(cudaMemcpyAsync(host, g->theta, sizeof(float) * gnn::NP, cudaMemcpyDeviceToHost, g->st));
    A2LS_CUDA(cudaStreamSynchronize(g->st));
    return A2LS_OK;
  });
}

int a2ls_gnn_set_params(a2ls_gnn* g, const float* host, int64_t count) {
  using namespace a2ls;
  if (!g || !host) return gnn_fail(A2LS_ERR_ARG, "null argument");
  if (count != gnn::NP) return gnn_fail(A2LS_ERR_ARG, "count must equal a2ls_gnn_num_params()");
  return gnn_guarded([&]() -> int {
    upload_params(g, host);
    return A2LS_OK;
  });
}

int a2ls_gnn_get_grads(a2ls_gnn* g, float* host, int64_t count) {
  using namespace a2ls;
  if (!g || !host) return gnn_fail(A2LS_ERR_ARG, "null argument");
  if (count != gnn::NP) return gnn_fail(A2LS_ERR_ARG, "count must equal a2ls_gnn_num_params()");
  return gnn_guarded([&]() -> int {
    A2LS_CUDA(cudaMemcpyAsync(host, g->grad, sizeof(float) * gnn::NP, cudaMemcpyDeviceToHost, g->st));
    A2LS_CUDA(cudaStreamSynchronize(g->st));
    const float inv = g->accum > 0 ? 1.f / (float)g->accum : 0.f;
    for (int p = 0; p < gnn::NP; ++p) host[p] *= inv;
    return A2LS_OK;
  });
}

int a2ls_gnn_sample_create(a2ls_handle* h, a2ls_gnn_sample** out) {
  using namespace a2ls;
  using namespace a2ls::gnn;
  if (!h || !out) return gnn_fail(A2LS_ERR_ARG, "null argument");
  *out = nullptr;
  if (!h->d_lrow || !h->d_lump) return gnn_fail(A2LS_ERR_STATE, "the handle has no local matrices");
  a2ls_gnn_sample* s = new a2ls_gnn_sample();
  s->st = h->st;
  int rc = gnn_guarded([&]() -> int {
    cudaStream_t st = s->st;
    s->N = h->N;
    s->S = h->sum_n;
    s->h_off = h->h_off;
    A2LS_CUDA(cudaMemcpyAsync(&s->E, h->d_lrow + s->S, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    A2LS_CUDA(cudaStreamSynchronize(st));
    s->off = galloc<int>(s->allocs, s->N + 1, st);
    s->rp = galloc<int64_t>(s->allocs, s->S + 1, st);
    s->col = galloc<int>(s->allocs, s->E, st);
    s->w = galloc<float>(s->allocs, s->E, st);
    s->s = galloc<float>(s->allocs, s->E, st);
    s->X = galloc<float>(s->allocs, (size_t)s->S * FX, st);
    A2LS_CUDA(cudaMemcpyAsync(s->off, h->d_off, sizeof(int) * (s->N + 1), cudaMemcpyDeviceToDevice, st));
    A2LS_CUDA(cudaMemcpyAsync(s->rp, h->d_lrow, sizeof(int64_t) * (s->S + 1), cudaMemcpyDeviceToDevice, st));
    std::vector<void*> tmp;
    build_graph(st, &h->launches, s->N, h->d_off, h->d_nI, h->d_lrow, h->d_lcol, h->d_lval, h->d_lump, s->S, s->col,
                s->w, s->s, s->X, tmp);
    gfree_all(tmp, st);
    // target: the eigenvectors the handle's setup selected (if it ran the eigensolver)
    s->h_zm.assign(s->N, 0);
    s->zm = galloc<int>(s->allocs, s->N, st);
    s->zoff = galloc<int64_t>(s->allocs, s->N + 1, st);
    std::vector<int64_t> zo(s->N + 1, 0);
    if (h->d_zev) {
      for (int i = 0; i < s->N; ++i) s->h_zm[i] = std::min(h->h_zcols[i], MAXZ);
    }
    for (int i = 0; i < s->N; ++i) zo[i + 1] = zo[i] + (int64_t)(s->h_off[i + 1] - s->h_off[i]) * s->h_zm[i];
    s->Z = galloc<float>(s->allocs, zo[s->N], st);
    A2LS_CUDA(cudaMemcpyAsync(s->zm, s->h_zm.data(), sizeof(int) * s->N, cudaMemcpyHostToDevice, st));
    A2LS_CUDA(cudaMemcpyAsync(s->zoff, zo.data(), sizeof(int64_t) * (s->N + 1), cudaMemcpyHostToDevice, st));
    s->ntarget = 0;
    for (int i = 0; i < s->N; ++i) s->ntarget += s->h_zm[i] > 0;
    if (h->d_zev && s->ntarget) {
      k_target_from_handle<<<s->N, 256, 0, st>>>(s->off, h->d_zoff, h->zld, h->d_zev, s->zm, s->zoff, s->Z);
      GNN_LAUNCH(&h->launches);
    }
    A2LS_CUDA(cudaStreamSynchronize(st));
    return A2LS_OK;
  });
  if (rc != A2LS_OK) {
    destroy_sample(s);
    return rc;
  }
  *out = s;
  return A2LS_OK;
}

int a2ls_gnn_sample_set_target(a2ls_gnn_sample* s, const int32_t* m, const double* Z) {
  using namespace a2ls;
  using namespace a2ls::gnn;
  if (!s || !m || !Z) return gnn_fail(A2LS_ERR_ARG, "null argument");
  for (int i = 0; i < s->N; ++i)
    if (m[i] < 0 || m[i] > MAXZ) return gnn_fail(A2LS_ERR_ARG, "target widths must lie in [0, 32]");
  return gnn_guarded([&]() -> int {
    cudaStream_t st = s->st;
    std::vector<int64_t> zo(s->N + 1, 0);
    for (int i = 0; i < s->N; ++i) zo[i + 1] = zo[i] + (int64_t)(s->h_off[i + 1] - s->h_off[i]) * m[i];
    std::vector<float> zf(zo[s->N]);
    for (int64_t e = 0; e < zo[s->N]; ++e) zf[e] = (float)Z[e];
    auto it = std::find(s->allocs.begin(), s->allocs.end(), (void*)s->Z);
    if (it != s->allocs.end()) {
      s->allocs.erase(it);
      cudaFreeAsync(s->Z, st);
    }
    s->Z = galloc<float>(s->allocs, zo[s->N], st);
    s->h_zm.assign(m, m + s->N);
    A2LS_CUDA(cudaMemcpyAsync(s->Z, zf.data(), sizeof(float) * zf.size(), cudaMemcpyHostToDevice, st));
    A2LS_CUDA(cudaMemcpyAsync(s->zm, m, sizeof(int) * s->N, cudaMemcpyHostToDevice, st));
    A2LS_CUDA(cudaMemcpyAsync(s->zoff, zo.data(), sizeof(int64_t) * (s->N + 1), cudaMemcpyHostToDevice, st));
    A2LS_CUDA(cudaStreamSynchronize(st));  // the host staging vectors go out of scope
    s->ntarget = 0;
    for (int i = 0; i < s->N; ++i) s->ntarget += m[i] > 0;
    return A2LS_OK;
  });
}

int a2ls_gnn_sample_destroy(a2ls_gnn_sample* s) {
  destroy_sample(s);
  return A2LS_OK;
}

int a2ls_gnn_sample_query(a2ls_gnn_sample* s, int32_t what, void* out, int64_t capacity, int64_t* needed) {
  using namespace a2ls;
  using namespace a2ls::gnn;
  if (!s) return gnn_fail(A2LS_ERR_ARG, "null argument");
  return gnn_guarded([&]() -> int {
    const void* src = nullptr;
    int64_t bytes = 0;
    switch (what) {
      case A2LS_GQ_FEATURES: src = s->X; bytes = (int64_t)s->S * FX * sizeof(float); break;
      case A2LS_GQ_ROWPTR: src = s->rp; bytes = (int64_t)(s->S + 1) * sizeof(int64_t); break;
      case A2LS_GQ_COLS: src = s->col; bytes = s->E * (int64_t)sizeof(int); break;
      case A2LS_GQ_WEIGHTS: src = s->w; bytes = s->E * (int64_t)sizeof(float); break;
      case A2LS_GQ_SWEIGHTS: src = s->s; bytes = s->E * (int64_t)sizeof(float); break;
      case A2LS_GQ_TARGET_COLS: src = s->zm; bytes = (int64_t)s->N * sizeof(int); break;
      default: fail(A2LS_ERR_ARG, "unknown sample item %d", what);
    }
    if (needed) *needed = bytes;
    if (!out) return A2LS_OK;
    if (capacity < bytes) fail(A2LS_ERR_ARG, "capacity %lld is below the %lld bytes needed", (long long)capacity, (long long)bytes);
    A2LS_CUDA(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, s->st));
    A2LS_CUDA(cudaStreamSynchronize(s->st));
    return A2LS_OK;
  });
}

int a2ls_gnn_forward(a2ls_gnn* g, a2ls_gnn_sample* s, float* Y) {
  using namespace a2ls;
  using namespace a2ls::gnn;
  if (!g || !s || !Y) return gnn_fail(A2LS_ERR_ARG, "null argument");
  return gnn_guarded([&]() -> int {
    cudaStream_t st = s->st;
    std::vector<void*> tmp;
    try {
      Acts a;
      alloc_acts(tmp, st, s->S, false, a);
      forward(st, &g->launches, sample_graph(s), g->w16, g->theta, false, a);
      A2LS_CUDA(cudaMemcpyAsync(Y, a.Y, sizeof(float) * s->S * OUT, cudaMemcpyDeviceToHost, st));
      A2LS_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      gfree_all(tmp, st);
      throw;
    }
    gfree_all(tmp, st);
    return A2LS_OK;
  });
}

int a2ls_gnn_loss_grad(a2ls_gnn* g, a2ls_gnn_sample* s, double* loss) {
  using namespace a2ls;
  using namespace a2ls::gnn;
  if (!g || !s) return gnn_fail(A2LS_ERR_ARG, "null argument");
  if (s->ntarget == 0) return gnn_fail(A2LS_ERR_STATE, "the sample has no target eigenvectors");
  return gnn_guarded([&]() -> int {
    cudaStream_t st = s->st;
    std::vector<void*> tmp;
    try {
      const int S = s->S, N = s->N;
      const Graph gr = sample_graph(s);
      Acts a;
      alloc_acts(tmp, st, S, true, a);
      forward(st, &g->launches, gr, g->w16, g->theta, true, a);
      double* d_loss = galloc<double>(tmp, N, st);
      float* dY = galloc<float>(tmp, (size_t)S * OUT, st);
      k_loss<<<N, 256, 0, st>>>(s->off, s->zm, s->zoff, s->Z, a.Y, 1.f / (float)s->ntarget, d_loss, dY);
      GNN_LAUNCH(&g->launches);
      // dp_0 into a.p0 (p_0 itself is no longer needed), scratch a.pa / a.pb / a.Y
      k_propagate<true><<<N, 256, 0, st>>>(s->off, s->rp, s->col, s->s, dY, a.pa, a.pb, a.Y, a.p0);
      GNN_LAUNCH(&g->launches);
      const int tiles = (S + TILE - 1) / TILE;
      const int G = std::max(1, std::min(tiles, 2 * 152));
      float* part = galloc<float>(tmp, (size_t)G * NP, st);
      const size_t hs = (size_t)S * WIDTH;
      float* vb[2] = {galloc<float>(tmp, hs, st), galloc<float>(tmp, hs, st)};
      float* ub[2] = {galloc<float>(tmp, hs, st), galloc<float>(tmp, hs, st)};
      set_smem_limits();
      k_layer_bwd<true><<<G, 256, BWD1_SMEM, st>>>(S, s->rp, s->col, s->w, a.h[2], a.m[3], a.h[3], a.p0, nullptr,
                                                   nullptr, g->w16, 3, vb[0], ub[0], part);
      GNN_LAUNCH(&g->launches);
      k_layer_bwd<false><<<G, 256, BWD_SMEM, st>>>(S, s->rp, s->col, s->w, a.h[1], a.m[2], a.h[2], nullptr, vb[0],
                                                   ub[0], g->w16, 2, vb[1], ub[1], part);
      GNN_LAUNCH(&g->launches);
      k_layer_bwd<false><<<G, 256, BWD_SMEM, st>>>(S, s->rp, s->col, s->w, a.h[0], a.m[1], a.h[1], nullptr, vb[1],
                                                   ub[1], g->w16, 1, vb[0], ub[0], part);
      GNN_LAUNCH(&g->launches);
      k_layer0_bwd<<<G, 256, 0, st>>>(S, s->rp, s->col, s->w, s->X, a.h[0], vb[0], ub[0], part);
      GNN_LAUNCH(&g->launches);
      k_reduce_parts<<<ceil_div(NP, 256), 256, 0, st>>>(G, part, g->grad);
      GNN_LAUNCH(&g->launches);
      std::vector<double> li(N);
      A2LS_CUDA(cudaMemcpyAsync(li.data(), d_loss, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
      A2LS_CUDA(cudaStreamSynchronize(st));
      double L = 0.0;
      for (int i = 0; i < N; ++i)
        if (s->h_zm[i] > 0) L += li[i];
      if (loss) *loss = L / s->ntarget;
      g->accum += 1;
    } catch (...) {
      gfree_all(tmp, st);
      throw;
    }
    gfree_all(tmp, st);
    return A2LS_OK;
  });
}

int a2ls_gnn_adam_step(a2ls_gnn* g, double lr) {
  using namespace a2ls;
  using namespace a2ls::gnn;
  if (!g) return gnn_fail(A2LS_ERR_ARG, "null argument");
  if (!(lr > 0.0)) return gnn_fail(A2LS_ERR_ARG, "the learning rate must be positive");
  if (g->accum == 0) return gnn_fail(A2LS_ERR_STATE, "no gradient accumulated since the last step");
  return gnn_guarded([&]() -> int {
    g->adam_t += 1;
    const double c1 = 1.0 - std::pow(0.9, (double)g->adam_t), c2 = 1.0 - std::pow(0.999, (double)g->adam_t);
    k_adam<<<ceil_div(NP, 256), 256, 0, g->st>>>(g->theta, g->mom1, g->mom2, g->grad, g->w16, 1.f / (float)g->accum,
                                                 (float)lr, (float)c1, (float)c2);
    GNN_LAUNCH(&g->launches);
    A2LS_CUDA(cudaStreamSynchronize(g->st));
    g->accum = 0;
    return A2LS_OK;
  });
}

int64_t a2ls_gnn_launches(const a2ls_gnn* g) { return g ? g->launches : 0; }

}  // extern "C"

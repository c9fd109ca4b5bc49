// Setup, part 4: the coarse space and the coarse operator (Section 3.2, Eq. 2.2).
//
//   R_0^H = [R_1^T W_1 ... R_N^T W_N] with W_i an orthonormal basis of range(D_i Z_i)
//   A_00  = R_0 A R_0^H, assembled block by block over pairs of subdomains whose
//           coarse columns couple through A, then inverted (exact LU, Section 4).
#include "a2ls_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace a2ls {

__device__ __forceinline__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

// Orthonormal basis of range(D_i Z_i): classical Gram-Schmidt applied twice per
// column; a column whose remaining norm is at most 1e-12 of the largest column norm
// of D_i Z_i is dropped.  Output columns are written in place (first mkeep columns).
__global__ void k_orth_w(const int* ni, const int* off, const double* D, double* Z, const int64_t* zoff,
                         int zld, const int* mcols, int* mkeep) {
  __shared__ double red[32];
  __shared__ double dots[MAXM + 2];
  const int i = blockIdx.x;
  const int n = ni[i], o = off[i], mc = mcols[i];
  double* Zi = Z + zoff[i];
  // D scaling and the largest column norm
  double cmax = 0.0;
  for (int c = 0; c < mc; ++c) {
    double s = 0.0;
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      const double v = D[o + l] * Zi[(int64_t)l * zld + c];
      Zi[(int64_t)l * zld + c] = v;
      s += v * v;
    }
    cmax = fmax(cmax, sqrt(cta_sum(s, red)));
  }
  int kept = 0;
  for (int c = 0; c < mc; ++c) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = 0; q < kept; ++q) {
        double s = 0.0;
        for (int l = threadIdx.x; l < n; l += blockDim.x) s += Zi[(int64_t)l * zld + q] * Zi[(int64_t)l * zld + c];
        s = cta_sum(s, red);
        if (threadIdx.x == 0) dots[q] = s;
      }
      __syncthreads();
      for (int l = threadIdx.x; l < n; l += blockDim.x) {
        double v = Zi[(int64_t)l * zld + c];
        for (int q = 0; q < kept; ++q) v -= dots[q] * Zi[(int64_t)l * zld + q];
        Zi[(int64_t)l * zld + c] = v;
      }
      __syncthreads();
    }
    double s = 0.0;
    for (int l = threadIdx.x; l < n; l += blockDim.x) s += Zi[(int64_t)l * zld + c] * Zi[(int64_t)l * zld + c];
    const double nrm = sqrt(cta_sum(s, red));
    if (nrm > 1e-12 * cmax && nrm > 0.0) {
      for (int l = threadIdx.x; l < n; l += blockDim.x)
        Zi[(int64_t)l * zld + kept] = Zi[(int64_t)l * zld + c] / nrm;
      ++kept;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) mkeep[i] = kept;
}

__global__ void k_compact_w(const int* ni, const double* Z, const int64_t* zoff, int zld, const int* m,
                            const int64_t* woff, double* W) {
  const int i = blockIdx.x;
  const int n = ni[i], mi = m[i];
  for (int e = threadIdx.x; e < n * mi; e += blockDim.x)
    W[woff[i] + e] = Z[zoff[i] + (int64_t)(e / mi) * zld + e % mi];
}

void upload_coarse_layout(a2ls_handle* h, const std::vector<int>& m) {
  const int N = h->N;
  h->h_m = m;
  h->h_coff.assign(N + 1, 0);
  h->h_woff.assign(N + 1, 0);
  for (int i = 0; i < N; ++i) {
    if (m[i] < 0 || m[i] > MAXM) fail(A2LS_ERR_ARG, "subdomain %d: %d coarse columns (at most %d)", i, m[i], MAXM);
    h->h_coff[i + 1] = h->h_coff[i] + m[i];
    h->h_woff[i + 1] = h->h_woff[i] + (int64_t)h->h_n[i] * m[i];
  }
  h->n0 = h->h_coff[N];
  if (!h->d_m) h->d_m = dalloc<int>(h, N);
  if (!h->d_coff) h->d_coff = dalloc<int>(h, N + 1);
  if (!h->d_woff) h->d_woff = dalloc<int64_t>(h, N + 1);
  A2LS_CUDA(cudaMemcpyAsync(h->d_m, m.data(), sizeof(int) * N, cudaMemcpyHostToDevice, h->st));
  A2LS_CUDA(cudaMemcpyAsync(h->d_coff, h->h_coff.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, h->st));
  A2LS_CUDA(cudaMemcpyAsync(h->d_woff, h->h_woff.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, h->st));
  if (h->d_W) dfree(h, h->d_W);
  h->d_W = dalloc<double>(h, std::max<int64_t>(h->h_woff[N], 1));
}

void orthonormalize_and_set_W(a2ls_handle* h, double* Z, const int* mcols, int zld) {
  const int N = h->N;
  cudaStream_t st = h->st;
  std::vector<int64_t> hzo(N + 1, 0);
  for (int i = 0; i < N; ++i) hzo[i + 1] = hzo[i] + (int64_t)h->h_n[i] * zld;
  int64_t* d_zo = dalloc<int64_t>(h, N + 1);
  int* d_mc = dalloc<int>(h, N);
  int* d_keep = dalloc<int>(h, N);
  A2LS_CUDA(cudaMemcpyAsync(d_zo, hzo.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(d_mc, mcols, sizeof(int) * N, cudaMemcpyHostToDevice, st));
  k_orth_w<<<N, 256, 0, st>>>(h->d_ni, h->d_off, h->d_D, Z, d_zo, zld, d_mc, d_keep);
  A2LS_LAUNCH();
  std::vector<int> keep(N);
  A2LS_CUDA(cudaMemcpyAsync(keep.data(), d_keep, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  upload_coarse_layout(h, keep);
  k_compact_w<<<N, 256, 0, st>>>(h->d_ni, Z, d_zo, zld, h->d_m, h->d_woff, h->d_W);
  A2LS_LAUNCH();
  dfree(h, d_zo);
  dfree(h, d_mc);
  dfree(h, d_keep);
  build_coarse_operator(h);
}

// pairs (i, j) whose coarse blocks couple: some row of supp(W_i) has a neighbour in supp(W_j)
__global__ void k_pair_bitmap(int N, const int* ni, const int* off, const int* idx, const double* D,
                              const int* rowptr, const int* colind, const int* mrow, const int* mpos,
                              const int* msub, const int* m, unsigned* bits) {
  const int i = blockIdx.x;
  if (m[i] == 0) return;
  const int words = (N + 31) / 32;
  const int o = off[i];
  for (int l = threadIdx.x; l < ni[i]; l += blockDim.x) {
    if (D[o + l] == 0.0) continue;
    const int g = idx[o + l];
    for (int q = rowptr[g]; q < rowptr[g + 1]; ++q) {
      const int k = colind[q];
      for (int t = mrow[k]; t < mrow[k + 1]; ++t) {
        const int j = msub[t];
        if (m[j] == 0 || D[mpos[t]] == 0.0) continue;
        atomicOr(bits + (size_t)i * words + (j >> 5), 1u << (j & 31));
      }
    }
  }
}

constexpr int EB_ROWS = 64;  // rows of Omega_i per batch in k_e_blocks

// E(i, j) = sum over rows l of supp(W_i), entries A(g(l), k), memberships (j, l') of k:
//           W_i[l, :]^T A(g, k) W_j[l', :]
// formed as W_i^T Y with Y = A(Omega_i, Omega_j) W_j, a batch of EB_ROWS rows of Omega_i at a time:
// one warp per row builds Y's row (lane c owns columns c and c + 32, every lane walks the row's
// couplings), then the CTA adds W_i(batch)^T Y to its m_i x m_j outputs.
__global__ void __launch_bounds__(256) k_e_blocks(const int2* pairs, const int* ni, const int* off,
                                                  const int* idx, const double* D, const int* rowptr,
                                                  const int* colind, const double* val, const int* mrow,
                                                  const int* mpos, const int* msub, const int* m,
                                                  const int* coff, const int64_t* woff, const double* W,
                                                  double* E, int n0) {
  __shared__ double Ys[EB_ROWS][MAXM + 1];
  const int i = pairs[blockIdx.x].x, j = pairs[blockIdx.x].y;
  const int mi = m[i], mj = m[j], oi = off[i], oj = off[j];
  const double* Wi = W + woff[i];
  const double* Wj = W + woff[j];
  constexpr int PER = (MAXM * MAXM + 255) / 256;
  double acc[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) acc[u] = 0.0;
  const int nout = mi * mj;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n = ni[i];
  for (int l0 = 0; l0 < n; l0 += EB_ROWS) {
    const int rows = min(EB_ROWS, n - l0);
    for (int r = wid; r < rows; r += 8) {
      const int l = l0 + r;
      double y0 = 0.0, y1 = 0.0;
      if (D[oi + l] != 0.0) {
        const int g = idx[oi + l];
        for (int q = rowptr[g]; q < rowptr[g + 1]; ++q) {
          const int k = colind[q];
          const double a = val[q];
          for (int t = mrow[k]; t < mrow[k + 1]; ++t) {
            if (msub[t] != j || D[mpos[t]] == 0.0) continue;
            const double* wr = Wj + (int64_t)(mpos[t] - oj) * mj;
            if (lane < mj) y0 += a * wr[lane];
            if (lane + 32 < mj) y1 += a * wr[lane + 32];
          }
        }
      }
      if (lane < mj) Ys[r][lane] = y0;
      if (lane + 32 < mj) Ys[r][lane + 32] = y1;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * 256;
      if (e < nout) {
        const int a = e / mj, c = e % mj;
        double sum = 0.0;
        for (int r = 0; r < rows; ++r) sum += Wi[(int64_t)(l0 + r) * mi + a] * Ys[r][c];
        acc[u] += sum;
      }
    }
    __syncthreads();
  }
  const int ci = coff[i], cj = coff[j];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int e = threadIdx.x + u * 256;
    if (e < nout) E[(int64_t)(ci + e / mj) * n0 + cj + e % mj] = acc[u];
  }
}

__global__ void k_diag_absmax(const double* E, int n, double* out) {
  double v = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    v = fmax(v, fabs(E[(int64_t)r * n + r]));
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(v));
}

// Order the coarse blocks (subdomains) so that A_00 has a small bandwidth: the
// natural order or reverse Cuthill-McKee on the subdomain coupling graph,
// whichever gives the narrower band.  The LU without pivoting keeps its fill
// inside the band, and the inverse is formed from the banded factors.
static int band_of(const std::vector<int2>& pairs, const std::vector<int>& coff, const std::vector<int>& m) {
  int w = 0;
  for (const int2& p : pairs) {
    if (m[p.x] == 0 || m[p.y] == 0) continue;
    w = std::max(w, coff[p.x] + m[p.x] - 1 - coff[p.y]);
    w = std::max(w, coff[p.y] + m[p.y] - 1 - coff[p.x]);
  }
  return w;
}

static std::vector<int> offsets_for(const std::vector<int>& order, const std::vector<int>& m) {
  std::vector<int> coff(m.size() + 1, 0);
  int acc = 0;
  for (int i : order) {
    coff[i] = acc;
    acc += m[i];
  }
  coff[m.size()] = acc;
  return coff;
}

void choose_coarse_order(a2ls_handle* h, const std::vector<int2>& pairs) {
  const int N = h->N;
  std::vector<std::vector<int>> adj(N);
  for (const int2& p : pairs)
    if (p.x != p.y) adj[p.x].push_back(p.y);
  std::vector<int> natural(N);
  for (int i = 0; i < N; ++i) natural[i] = i;
  // reverse Cuthill-McKee from a minimum-degree node of every component
  std::vector<int> order, seen(N, 0);
  for (int start = 0; (int)order.size() < N;) {
    int best = -1;
    for (int i = 0; i < N; ++i)
      if (!seen[i] && (best < 0 || adj[i].size() < adj[best].size())) best = i;
    start = best;
    std::vector<int> queue{start};
    seen[start] = 1;
    for (size_t q = 0; q < queue.size(); ++q) {
      std::vector<int> nb;
      for (int j : adj[queue[q]])
        if (!seen[j]) {
          seen[j] = 1;
          nb.push_back(j);
        }
      std::sort(nb.begin(), nb.end(), [&](int a, int b) { return adj[a].size() < adj[b].size() || (adj[a].size() == adj[b].size() && a < b); });
      queue.insert(queue.end(), nb.begin(), nb.end());
    }
    order.insert(order.end(), queue.begin(), queue.end());
  }
  std::reverse(order.begin(), order.end());
  std::vector<int> c_nat = offsets_for(natural, h->h_m), c_rcm = offsets_for(order, h->h_m);
  const int w_nat = band_of(pairs, c_nat, h->h_m), w_rcm = band_of(pairs, c_rcm, h->h_m);
  h->h_coff = (w_rcm < w_nat) ? c_rcm : c_nat;
  h->coarse_band = std::min(w_nat, w_rcm);
  A2LS_CUDA(cudaMemcpyAsync(h->d_coff, h->h_coff.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, h->st));
}

void build_coarse_operator(a2ls_handle* h) {
  const int N = h->N, n0 = h->n0;
  cudaStream_t st = h->st;
  if (h->d_Einv) {
    dfree(h, h->d_Einv);
    h->d_Einv = nullptr;
  }
  if (n0 == 0) return;
  const int words = (N + 31) / 32;
  unsigned* bits = dalloc<unsigned>(h, (size_t)N * words);
  A2LS_CUDA(cudaMemsetAsync(bits, 0, sizeof(unsigned) * N * words, st));
  k_pair_bitmap<<<N, 256, 0, st>>>(N, h->d_ni, h->d_off, h->d_idx, h->d_D, h->rowptr, h->colind, h->d_mrow,
                                    h->d_mpos, h->d_msub, h->d_m, bits);
  A2LS_LAUNCH();
  std::vector<unsigned> hb((size_t)N * words);
  A2LS_CUDA(cudaMemcpyAsync(hb.data(), bits, sizeof(unsigned) * hb.size(), cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  std::vector<int2> pairs;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      if (hb[(size_t)i * words + (j >> 5)] & (1u << (j & 31))) pairs.push_back(make_int2(i, j));
  dfree(h, bits);
  choose_coarse_order(h, pairs);
  double* E = dalloc<double>(h, (size_t)n0 * n0);
  A2LS_CUDA(cudaMemsetAsync(E, 0, sizeof(double) * n0 * n0, st));
  if (!pairs.empty()) {
    int2* d_pairs = dalloc<int2>(h, pairs.size());
    A2LS_CUDA(cudaMemcpyAsync(d_pairs, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice, st));
    k_e_blocks<<<(int)pairs.size(), 256, 0, st>>>(d_pairs, h->d_ni, h->d_off, h->d_idx, h->d_D, h->rowptr,
                                                   h->colind, h->val, h->d_mrow, h->d_mpos, h->d_msub, h->d_m,
                                                   h->d_coff, h->d_woff, h->d_W, E, n0);
    A2LS_LAUNCH();
    A2LS_CUDA(cudaStreamSynchronize(st));
    dfree(h, d_pairs);
  }
  double* dmax = dalloc<double>(h, 1);
  A2LS_CUDA(cudaMemsetAsync(dmax, 0, sizeof(double), st));
  k_diag_absmax<<<ceil_div(n0, 256), 256, 0, st>>>(E, n0, dmax);
  A2LS_LAUNCH();
  double scale = 0.0;
  A2LS_CUDA(cudaMemcpyAsync(&scale, dmax, sizeof(double), cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  dfree(h, dmax);
  if (!(scale > 0.0)) fail(A2LS_ERR_SINGULAR, "coarse operator has a zero diagonal");
  h->d_Einv = dalloc<double>(h, (size_t)n0 * n0);
  dense_inverse(h, E, n0, scale, h->d_Einv, h->coarse_band);
  sync_and_check(h, "coarse operator");
  dfree(h, E);
  // apply workspace sized by n0
  if (h->d_g) dfree(h, h->d_g);
  if (h->d_c) dfree(h, h->d_c);
  h->d_g = dalloc<double>(h, n0);
  h->d_c = dalloc<double>(h, n0);
}

}  // namespace a2ls

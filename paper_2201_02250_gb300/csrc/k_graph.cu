// Setup, part 1: input validation, algebraic overlap, subdomain index lists,
// memberships, partition of unity and extraction of the local matrices.
//
//   Section 2: Omega_Gamma_i = nodes at distance one from Omega_Ii in G(A);
//              delta layers repeat the step; Omega_i = [Omega_Ii, Omega_Gamma_i].
//   Definition 3.1: s_i(j) = sum_k |A(j,k)| over k outside Omega_i for j in
//              Omega_Gamma_i, and A~_ii = A_ii - diag(0, s_i).
#include "a2ls_internal.cuh"

#include <algorithm>
#include <cstring>

namespace a2ls {

// ---------------------------------------------------------------------------
// generic exclusive scan over int64 (3-phase, recursive on the block sums)
// ---------------------------------------------------------------------------
constexpr int SCAN_BLOCK = 1024;

__global__ void k_scan_block(const int64_t* in, int64_t* out, int64_t* block_sums, int n) {
  __shared__ int64_t s[SCAN_BLOCK];
  int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int64_t v = (i < n) ? in[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
    int64_t t = (threadIdx.x >= off) ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;  // exclusive
  if (threadIdx.x == SCAN_BLOCK - 1) block_sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_add(int64_t* out, const int64_t* block_offsets, int n) {
  int i = blockIdx.x * SCAN_BLOCK + threadIdx.x;
  if (i < n) out[i] += block_offsets[blockIdx.x];
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int n, cudaStream_t st, a2ls_handle* h) {
  if (n <= 0) return;
  int nb = ceil_div(n, SCAN_BLOCK);
  int64_t* sums = dalloc<int64_t>(h, nb);
  int64_t* offs = dalloc<int64_t>(h, nb);
  k_scan_block<<<nb, SCAN_BLOCK, 0, st>>>(in, out, sums, n);
  A2LS_LAUNCH();
  if (nb > 1) {
    exclusive_scan_i64(sums, offs, nb, st, h);
    k_scan_add<<<nb, SCAN_BLOCK, 0, st>>>(out, offs, n);
    A2LS_LAUNCH();
  }
  dfree(h, sums);
  dfree(h, offs);
}

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
__global__ void k_validate_csr(int n, int nnz, const int* rowptr, const int* colind, int* st) {
  int r0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (r0 == 0 && (rowptr[0] != 0 || rowptr[n] != nnz)) raise_status(st, A2LS_ERR_ARG, -1, 1);
  for (int r = r0; r < n; r += gridDim.x * blockDim.x) {
    int a = rowptr[r], b = rowptr[r + 1];
    if (a < 0 || a > b || b > nnz) {
      raise_status(st, A2LS_ERR_ARG, r, 2);
      continue;
    }
    for (int p = a; p < b; ++p) {
      int c = colind[p];
      if (c < 0 || c >= n) raise_status(st, A2LS_ERR_ARG, r, 3);
    }
  }
}

__global__ void k_part_range(int n, const int* part, int* minmax) {
  int lo = INT32_MAX, hi = INT32_MIN;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    lo = min(lo, part[j]);
    hi = max(hi, part[j]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(minmax, lo);
    atomicMax(minmax + 1, hi);
  }
}

// ---------------------------------------------------------------------------
// transposed pattern (for the graph of A + A^T)
// ---------------------------------------------------------------------------
__global__ void k_col_counts(int nnz, const int* colind, int64_t* counts) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long*>(counts + colind[p]), 1ull);
}

__global__ void k_fill_transpose(int n, const int* rowptr, const int* colind, const int64_t* trow,
                                 int* cursor, int* tcol) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      int c = colind[p];
      int at = atomicAdd(cursor + c, 1);
      tcol[trow[c] + at] = r;
    }
}

// ---------------------------------------------------------------------------
// overlap growth on per-subdomain bitmaps
// ---------------------------------------------------------------------------
__global__ void k_bitmap_interior(int n, int W, const int* part, unsigned* interior) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    atomicOr(interior + (size_t)part[j] * W + (j >> 5), 1u << (j & 31));
}

// next |= adj(frontier) \ member, over the graph of A + A^T
__global__ void k_bitmap_expand(int N, int W, const unsigned* frontier, const unsigned* member,
                                unsigned* next, const int* rowptr, const int* colind,
                                const int64_t* trow, const int* tcol) {
  size_t total = (size_t)N * W;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
       q += (size_t)gridDim.x * blockDim.x) {
    unsigned bits = frontier[q];
    if (!bits) continue;
    size_t base = q - q % W;  // start of this subdomain's bitmap
    int w = (int)(q % W);
    while (bits) {
      int b = __ffs(bits) - 1;
      bits &= bits - 1;
      int j = w * 32 + b;
      for (int p = rowptr[j]; p < rowptr[j + 1]; ++p) {
        int k = colind[p];
        unsigned bit = 1u << (k & 31);
        if (!(member[base + (k >> 5)] & bit)) atomicOr(next + base + (k >> 5), bit);
      }
      for (int64_t p = trow[j]; p < trow[j + 1]; ++p) {
        int k = tcol[p];
        unsigned bit = 1u << (k & 31);
        if (!(member[base + (k >> 5)] & bit)) atomicOr(next + base + (k >> 5), bit);
      }
    }
  }
}

__global__ void k_bitmap_merge(size_t total, unsigned* frontier, unsigned* member, unsigned* next) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total;
       q += (size_t)gridDim.x * blockDim.x) {
    unsigned nx = next[q] & ~member[q];
    frontier[q] = nx;
    member[q] |= nx;
    next[q] = 0;
  }
}

// per subdomain: |Omega_Ii| and |Omega_Gamma_i|
__global__ void k_bitmap_count(int W, const unsigned* interior, const unsigned* member, int* cI,
                               int* cG) {
  int i = blockIdx.x;
  const unsigned* ib = interior + (size_t)i * W;
  const unsigned* mb = member + (size_t)i * W;
  int a = 0, g = 0;
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    a += __popc(ib[w]);
    g += __popc(mb[w] & ~ib[w]);
  }
  __shared__ int sa[32], sg[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    g += __shfl_xor_sync(0xffffffffu, g, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    sg[threadIdx.x >> 5] = g;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int ta = 0, tg = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      ta += sa[k];
      tg += sg[k];
    }
    cI[i] = ta;
    cG[i] = tg;
  }
}

// Emit the ordered index list of every subdomain: interior ascending, then the overlap layer by
// layer (the nodes the first growth step adds, ascending, then those of the second step, ...).
// Listing the layer next to the interior first keeps the overlap nodes without interior couplings
// out of the interior columns' envelope of the local factors.  One CTA per subdomain, one word per
// thread per chunk, block-wide exclusive scans.
__global__ void k_bitmap_emit(int N, int W, const unsigned* interior, const unsigned* layers, int delta,
                              const int* off, int* idx, int* ipos, int* gstart) {
  const int i = blockIdx.x;
  __shared__ int warp_c[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int o_i = off[i];
  for (int g = 0; g <= delta; ++g) {
    if (threadIdx.x == 0) gstart[(size_t)i * (delta + 2) + g] = base;
    const unsigned* gb = (g == 0) ? interior + (size_t)i * W : layers + ((size_t)(g - 1) * N + i) * W;
    for (int w0 = 0; w0 < W; w0 += blockDim.x) {
      const int w = w0 + threadIdx.x;
      unsigned bits = (w < W) ? gb[w] : 0u;
      const int c = __popc(bits);
      int x = c;  // inclusive warp scan
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) warp_c[wid] = x;
      __syncthreads();
      int p = base;
      for (int k = 0; k < wid; ++k) p += warp_c[k];
      p += x - c;
      while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        const int j = w * 32 + b;
        idx[o_i + p] = j;
        if (g == 0) ipos[j] = p;
        ++p;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 0;
        for (int k = 0; k < nw; ++k) t += warp_c[k];
        base += t;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) gstart[(size_t)i * (delta + 2) + delta + 1] = base;
}

// ---------------------------------------------------------------------------
// memberships: node -> flat local positions, sorted by subdomain
// ---------------------------------------------------------------------------
__global__ void k_psub(int N, const int* off, int* psub) {
  int i = blockIdx.x;
  for (int p = off[i] + threadIdx.x; p < off[i + 1]; p += blockDim.x) psub[p] = i;
}

__global__ void k_member_count(int total, const int* idx, int64_t* mcount) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long*>(mcount + idx[p]), 1ull);
}

__global__ void k_member_fill(int total, const int* idx, const int64_t* mrow64, int* cursor,
                              int* mpos) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
    int j = idx[p];
    int at = atomicAdd(cursor + j, 1);
    mpos[mrow64[j] + at] = p;
  }
}

// sort each node's list by position (= by subdomain, since offsets grow with i),
// set msub, the 32-bit row pointer and the partition-of-unity weights
__global__ void k_member_finish(int n, const int64_t* mrow64, int* mrow, int* mpos, int* msub,
                                const int* psub) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int a = (int)mrow64[j], b = (int)mrow64[j + 1];
    for (int x = a + 1; x < b; ++x) {  // insertion sort: lists are short
      int v = mpos[x], y = x - 1;
      while (y >= a && mpos[y] > v) {
        mpos[y + 1] = mpos[y];
        --y;
      }
      mpos[y + 1] = v;
    }
    for (int x = a; x < b; ++x) msub[x] = psub[mpos[x]];
    mrow[j] = a;
    if (j == n - 1) mrow[n] = b;
  }
}

__global__ void k_pou(int total, int pou, const int* psub, const int* off, const int* nI,
                      const int* idx, const int* mrow, double* D) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
    int i = psub[p];
    int l = p - off[i];
    if (pou == A2LS_POU_BOOLEAN) {
      D[p] = (l < nI[i]) ? 1.0 : 0.0;
    } else {
      int j = idx[p];
      D[p] = 1.0 / (double)(mrow[j + 1] - mrow[j]);
    }
  }
}

__global__ void k_row_lengths(int total, const int* idx, const int* rowptr, int64_t* len) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x)
    len[p] = rowptr[idx[p] + 1] - rowptr[idx[p]];
}

static int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

void build_subdomains(a2ls_handle* h) {
  cudaStream_t st = h->st;
  const int n = h->n;
  // CSR structure
  k_validate_csr<<<grid_for(n, 256), 256, 0, st>>>(n, h->nnz, h->rowptr, h->colind, h->d_status);
  A2LS_LAUNCH();
  sync_and_check(h, "CSR validation");

  // partition range and part sizes
  int* mm = dalloc<int>(h, 2);
  int init[2] = {INT32_MAX, INT32_MIN};
  A2LS_CUDA(cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, st));
  k_part_range<<<grid_for(n, 256), 256, 0, st>>>(n, h->part, mm);
  A2LS_LAUNCH();
  int hm[2];
  A2LS_CUDA(cudaMemcpyAsync(hm, mm, sizeof(hm), cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  dfree(h, mm);
  if (hm[0] < 0) fail(A2LS_ERR_ARG, "partition has a negative entry (%d)", hm[0]);
  const int N = hm[1] + 1;
  if (N > n) fail(A2LS_ERR_ARG, "partition has %d parts for %d nodes", N, n);
  h->N = N;

  // transposed pattern
  int64_t* tcnt = dalloc<int64_t>(h, n + 1);
  int64_t* trow = dalloc<int64_t>(h, n + 1);
  A2LS_CUDA(cudaMemsetAsync(tcnt, 0, sizeof(int64_t) * (n + 1), st));
  k_col_counts<<<grid_for(h->nnz, 256), 256, 0, st>>>(h->nnz, h->colind, tcnt);
  A2LS_LAUNCH();
  exclusive_scan_i64(tcnt, trow, n + 1, st, h);
  int* tcol = dalloc<int>(h, h->nnz);
  int* cursor = dalloc<int>(h, n);
  A2LS_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * n, st));
  k_fill_transpose<<<grid_for(n, 256), 256, 0, st>>>(n, h->rowptr, h->colind, trow, cursor, tcol);
  A2LS_LAUNCH();

  // bitmaps
  const int W = ceil_div(n, 32);
  const size_t bw = (size_t)N * W;
  unsigned* interior = dalloc<unsigned>(h, bw);
  unsigned* member = dalloc<unsigned>(h, bw);
  unsigned* frontier = dalloc<unsigned>(h, bw);
  unsigned* next = dalloc<unsigned>(h, bw);
  A2LS_CUDA(cudaMemsetAsync(interior, 0, bw * 4, st));
  A2LS_CUDA(cudaMemsetAsync(next, 0, bw * 4, st));
  k_bitmap_interior<<<grid_for(n, 256), 256, 0, st>>>(n, W, h->part, interior);
  A2LS_LAUNCH();
  A2LS_CUDA(cudaMemcpyAsync(member, interior, bw * 4, cudaMemcpyDeviceToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(frontier, interior, bw * 4, cudaMemcpyDeviceToDevice, st));
  // the nodes each step adds (the overlap layers), kept to order Omega_Gamma by layer
  unsigned* layers = dalloc<unsigned>(h, bw * std::max(h->delta, 1));
  for (int layer = 0; layer < h->delta; ++layer) {
    k_bitmap_expand<<<grid_for((int64_t)bw, 256), 256, 0, st>>>(N, W, frontier, member, next,
                                                                 h->rowptr, h->colind, trow, tcol);
    A2LS_LAUNCH();
    k_bitmap_merge<<<grid_for((int64_t)bw, 256), 256, 0, st>>>(bw, frontier, member, next);
    A2LS_LAUNCH();
    A2LS_CUDA(cudaMemcpyAsync(layers + (size_t)layer * bw, frontier, bw * 4, cudaMemcpyDeviceToDevice, st));
  }
  int* cI = dalloc<int>(h, N);
  int* cG = dalloc<int>(h, N);
  k_bitmap_count<<<N, 256, 0, st>>>(W, interior, member, cI, cG);
  A2LS_LAUNCH();
  std::vector<int> hI(N), hG(N);
  A2LS_CUDA(cudaMemcpyAsync(hI.data(), cI, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaMemcpyAsync(hG.data(), cG, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  h->h_off.assign(N + 1, 0);
  h->h_nI = hI;
  h->h_n.resize(N);
  h->h_ld.resize(N);
  h->h_foff.assign(N + 1, 0);
  int64_t tot = 0;
  h->max_n = 0;
  for (int i = 0; i < N; ++i) {
    if (hI[i] == 0) fail(A2LS_ERR_ARG, "part %d of the partition is empty", i);
    h->h_n[i] = hI[i] + hG[i];
    if (h->h_n[i] > MAXN_LOCAL)
      fail(A2LS_ERR_ARG, "subdomain %d has %d rows; at most %d are supported", i, h->h_n[i], MAXN_LOCAL);
    h->h_ld[i] = (int)round_up(h->h_n[i], 4);
    h->h_off[i + 1] = h->h_off[i] + h->h_n[i];
    h->h_foff[i + 1] = h->h_foff[i] + (int64_t)h->h_ld[i] * h->h_n[i];
    h->max_n = std::max(h->max_n, h->h_n[i]);
    tot += h->h_n[i];
  }
  if (tot > INT32_MAX / 2) fail(A2LS_ERR_ARG, "sum of subdomain sizes too large");
  h->sum_n = (int)tot;
  h->d_off = dalloc<int>(h, N + 1);
  h->d_nI = dalloc<int>(h, N);
  h->d_ni = dalloc<int>(h, N);
  h->d_ld = dalloc<int>(h, N);
  h->d_foff = dalloc<int64_t>(h, N + 1);
  A2LS_CUDA(cudaMemcpyAsync(h->d_off, h->h_off.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(h->d_nI, h->h_nI.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(h->d_ni, h->h_n.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(h->d_ld, h->h_ld.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(h->d_foff, h->h_foff.data(), sizeof(int64_t) * (N + 1),
                            cudaMemcpyHostToDevice, st));
  h->d_idx = dalloc<int>(h, h->sum_n);
  h->d_ipos = dalloc<int>(h, n);
  {
    // work order of the batched kernels: largest subdomains first (longest-processing-time rule)
    std::vector<int> order(N);
    for (int i = 0; i < N; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h->h_n[a] > h->h_n[b]; });
    h->d_sched = dalloc<int>(h, N);
    h->d_counter = dalloc<int>(h, 4);
    A2LS_CUDA(cudaMemcpyAsync(h->d_sched, order.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
    A2LS_CUDA(cudaStreamSynchronize(st));
  }
  h->d_gstart = dalloc<int>(h, (size_t)N * (h->delta + 2));
  k_bitmap_emit<<<N, 256, 0, st>>>(N, W, interior, layers, h->delta, h->d_off, h->d_idx, h->d_ipos, h->d_gstart);
  A2LS_LAUNCH();
  dfree(h, layers);
  dfree(h, interior);
  dfree(h, member);
  dfree(h, frontier);
  dfree(h, next);
  dfree(h, cI);
  dfree(h, cG);
  dfree(h, tcnt);
  dfree(h, trow);
  dfree(h, tcol);
  dfree(h, cursor);

  // memberships and partition of unity
  const int S = h->sum_n;
  int* psub = dalloc<int>(h, S);
  k_psub<<<N, 256, 0, st>>>(N, h->d_off, psub);
  A2LS_LAUNCH();
  int64_t* mcnt = dalloc<int64_t>(h, n + 1);
  int64_t* mrow64 = dalloc<int64_t>(h, n + 1);
  A2LS_CUDA(cudaMemsetAsync(mcnt, 0, sizeof(int64_t) * (n + 1), st));
  k_member_count<<<grid_for(S, 256), 256, 0, st>>>(S, h->d_idx, mcnt);
  A2LS_LAUNCH();
  exclusive_scan_i64(mcnt, mrow64, n + 1, st, h);
  int* mcur = dalloc<int>(h, n);
  A2LS_CUDA(cudaMemsetAsync(mcur, 0, sizeof(int) * n, st));
  h->d_mrow = dalloc<int>(h, n + 1);
  h->d_mpos = dalloc<int>(h, S);
  h->d_msub = dalloc<int>(h, S);
  k_member_fill<<<grid_for(S, 256), 256, 0, st>>>(S, h->d_idx, mrow64, mcur, h->d_mpos);
  A2LS_LAUNCH();
  k_member_finish<<<grid_for(n, 256), 256, 0, st>>>(n, mrow64, h->d_mrow, h->d_mpos, h->d_msub, psub);
  A2LS_LAUNCH();
  h->d_D = dalloc<double>(h, S);
  k_pou<<<grid_for(S, 256), 256, 0, st>>>(S, h->opt.pou, psub, h->d_off, h->d_nI, h->d_idx,
                                          h->d_mrow, h->d_D);
  A2LS_LAUNCH();
  // local CSR row pointers
  int64_t* len = dalloc<int64_t>(h, S + 1);
  A2LS_CUDA(cudaMemsetAsync(len, 0, sizeof(int64_t) * (S + 1), st));
  k_row_lengths<<<grid_for(S, 256), 256, 0, st>>>(S, h->d_idx, h->rowptr, len);
  A2LS_LAUNCH();
  h->d_lrow = dalloc<int64_t>(h, S + 1);
  exclusive_scan_i64(len, h->d_lrow, S + 1, st, h);
  int64_t lnnz = 0;
  A2LS_CUDA(cudaMemcpyAsync(&lnnz, h->d_lrow + S, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  h->d_lcol = dalloc<int>(h, lnnz);
  h->d_lval = dalloc<double>(h, lnnz);
  dfree(h, psub);
  dfree(h, mcnt);
  dfree(h, mrow64);
  dfree(h, mcur);
  dfree(h, len);
  sync_and_check(h, "overlap construction");
}

// ---------------------------------------------------------------------------
// extraction of A_ii, A~_ii (dense, precision T), s_i and the local CSR
// One warp per local row.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // v >= 0: the IEEE bit pattern of non-negative doubles orders like int64
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <class T, class TT>
__global__ void k_extract(int S, int N, const int* off, const int* nI, const int* ni, const int* ld,
                          const int64_t* foff, const int* idx, const int* ipos, const int* gstart, int delta,
                          const int* part,
                          const int* rowptr, const int* colind, const double* val, const int64_t* lrow,
                          int* lcol, double* lval, double* lump, T* dA, TT* dAt, double* dscale) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < S; p += warps) {
    // subdomain of position p (binary search over the offsets)
    int lo = 0, hi = N;  // off[lo] <= p < off[hi]
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (off[mid] <= p) lo = mid; else hi = mid;
    }
    const int i = lo, o = off[i], l = p - o, n_I = nI[i];
    const int j = idx[p];
    const int64_t base = foff[i] + (int64_t)l * ld[i];
    const int r0 = rowptr[j], r1 = rowptr[j + 1];
    const int64_t lb = lrow[p];
    double s = 0.0, ajj = 0.0;
    for (int q = r0 + lane; q < r1; q += 32) {
      const int k = colind[q];
      const double a = val[q];
      int lk = -1;
      if (part[k] == i) {
        lk = ipos[k];
      } else {
        // the overlap list is ascending within each layer: search the layers in turn
        const int* gs = gstart + (size_t)i * (delta + 2);
        for (int g = 1; g <= delta && lk < 0; ++g) {
          int a0 = o + gs[g], b0 = o + gs[g + 1];
          const int e0 = b0;
          while (a0 < b0) {
            int mid = (a0 + b0) >> 1;
            int v = idx[mid];
            if (v < k) a0 = mid + 1; else b0 = mid;
          }
          if (a0 < e0 && idx[a0] == k) lk = a0 - o;
        }
      }
      lcol[lb + (q - r0)] = lk;
      lval[lb + (q - r0)] = a;
      if (lk >= 0) {
        dA[base + lk] = (T)a;
        if (dAt) dAt[base + lk] = (TT)a;
        if (k == j) ajj = a;
      } else if (l >= n_I) {
        s += fabs(a);
      }
    }
    for (int w = 16; w > 0; w >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, w);
      ajj += __shfl_xor_sync(0xffffffffu, ajj, w);
    }
    if (lane == 0) {
      lump[p] = (l >= n_I) ? s : 0.0;
      if (dAt && l >= n_I) dAt[base + l] = (TT)(ajj - s);
      atomic_max_pos(dscale + i, fabs(ajj));
    }
  }
}

template <class TA, class TT>
static void launch_extract(a2ls_handle* h, void* dense_A, void* dense_At, double* dense_scale, int blocks) {
  k_extract<TA, TT><<<blocks, 256, 0, h->st>>>(
      h->sum_n, h->N, h->d_off, h->d_nI, h->d_ni, h->d_ld, h->d_foff, h->d_idx, h->d_ipos, h->d_gstart, h->delta,
      h->part, h->rowptr,
      h->colind, h->val, h->d_lrow, h->d_lcol, h->d_lval, h->d_lump, static_cast<TA*>(dense_A),
      static_cast<TT*>(dense_At), dense_scale);
  A2LS_LAUNCH();
}

// ---------------------------------------------------------------------------
// envelope of the local matrices (A_ii and A~_ii share their pattern): for row l the first column
// f_l with a nonzero, for column c the first row g_c with a nonzero.  Gaussian elimination without
// pivoting keeps L inside the row envelope (L[l][c] = 0 for c < f_l) and U inside the column
// envelope (U[r][c] = 0 for r < g_c), so tiles outside them stay exactly zero and are skipped.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int subdomain_of(int p, int N, const int* off) {
  int lo = 0, hi = N;  // off[lo] <= p < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

// g_c starts at c (the diagonal)
__global__ void k_profile_init(int S, int N, const int* off, int* pg) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < S; p += gridDim.x * blockDim.x)
    pg[p] = p - off[subdomain_of(p, N, off)];
}

__global__ void k_profile_rows(int S, int N, const int* off, const int64_t* lrow, const int* lcol, int* pf, int* pg) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < S; p += gridDim.x * blockDim.x) {
    const int o = off[subdomain_of(p, N, off)], l = p - o;
    int f = l;
    for (int64_t q = lrow[p]; q < lrow[p + 1]; ++q) {
      const int k = lcol[q];
      if (k < 0) continue;
      f = min(f, k);
      atomicMin(pg + o + k, l);
    }
    pf[p] = f;
  }
}

// minima of f over the 64-row tiles and of g over the 64-column tiles of each subdomain
__global__ void k_profile_tiles(const int* off, const int* ni, const int* toff, const int* pf, const int* pg,
                                int* tf, int* tg) {
  const int i = blockIdx.x, o = off[i], n = ni[i], nt = toff[i + 1] - toff[i];
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    int a = n, b = n;
    for (int l = t * TB; l < min(n, (t + 1) * TB); ++l) {
      a = min(a, pf[o + l]);
      b = min(b, pg[o + l]);
    }
    tf[toff[i] + t] = a;
    tg[toff[i] + t] = b;
  }
}

// Algorithmic work of the envelope-aware kernels per subdomain: out[4i] = LU flops over all pivots,
// out[4i+1] = LU flops over the overlap pivots (k >= n_I), out[4i+2] = entries of L's row envelope
// (sum_r r - f_r + 1), out[4i+3] = entries of U's column envelope (sum_c c - g_c + 1).  Pivot k updates
// (#rows r > k with f_r <= k) x (#columns c > k with g_c <= k) entries, two flops each.
__global__ void k_envelope_counts(const int* off, const int* ni, const int* nI, const int* pf, const int* pg,
                                  double* out) {
  extern __shared__ int cnt[];  // 2n: histograms of f and g
  __shared__ double red[2][32];
  const int i = blockIdx.x, o = off[i], n = ni[i], n_I = nI[i];
  for (int e = threadIdx.x; e < 2 * n; e += blockDim.x) cnt[e] = 0;
  __syncthreads();
  double sf = 0.0, sg = 0.0;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    atomicAdd(&cnt[pf[o + l]], 1);
    atomicAdd(&cnt[n + pg[o + l]], 1);
    sf += (double)(l - pf[o + l] + 1);
    sg += (double)(l - pg[o + l] + 1);
  }
  for (int q = 16; q > 0; q >>= 1) {
    sf += __shfl_xor_sync(0xffffffffu, sf, q);
    sg += __shfl_xor_sync(0xffffffffu, sg, q);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sf;
    red[1][threadIdx.x >> 5] = sg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tf = 0.0, tg = 0.0, full = 0.0, gam = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tf += red[0][w];
      tg += red[1][w];
    }
    long long cf = 0, cg = 0;
    for (int k = 0; k < n; ++k) {
      cf += cnt[k];
      cg += cnt[n + k];
      const double t = 2.0 * (double)(cf - k - 1) * (double)(cg - k - 1);
      full += t;
      if (k >= n_I) gam += t;
    }
    out[4 * i] = full;
    out[4 * i + 1] = gam;
    out[4 * i + 2] = tf;
    out[4 * i + 3] = tg;
  }
}

void compute_profiles(a2ls_handle* h) {
  cudaStream_t st = h->st;
  const int S = h->sum_n, N = h->N;
  h->d_pf = dalloc<int>(h, S);
  h->d_pg = dalloc<int>(h, S);
  k_profile_init<<<grid_for(S, 256), 256, 0, st>>>(S, N, h->d_off, h->d_pg);
  A2LS_LAUNCH();
  k_profile_rows<<<grid_for(S, 256), 256, 0, st>>>(S, N, h->d_off, h->d_lrow, h->d_lcol, h->d_pf, h->d_pg);
  A2LS_LAUNCH();
  h->h_toff.assign(N + 1, 0);
  for (int i = 0; i < N; ++i) h->h_toff[i + 1] = h->h_toff[i] + (h->h_n[i] + TB - 1) / TB;
  h->d_toff = dalloc<int>(h, N + 1);
  A2LS_CUDA(cudaMemcpyAsync(h->d_toff, h->h_toff.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st));
  h->d_tf = dalloc<int>(h, h->h_toff[N]);
  h->d_tg = dalloc<int>(h, h->h_toff[N]);
  k_profile_tiles<<<N, 64, 0, st>>>(h->d_off, h->d_ni, h->d_toff, h->d_pf, h->d_pg, h->d_tf, h->d_tg);
  A2LS_LAUNCH();
  double* d_env = dalloc<double>(h, 4 * (size_t)N);
  const size_t smem = sizeof(int) * 2 * (size_t)h->max_n;
  A2LS_CUDA(cudaFuncSetAttribute(k_envelope_counts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_envelope_counts<<<N, 256, smem, st>>>(h->d_off, h->d_ni, h->d_nI, h->d_pf, h->d_pg, d_env);
  A2LS_LAUNCH();
  h->h_env.assign(4 * (size_t)N, 0.0);
  A2LS_CUDA(cudaMemcpyAsync(h->h_env.data(), d_env, sizeof(double) * 4 * N, cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  dfree(h, d_env);
}

void extract_local(a2ls_handle* h, void* dense_A, void* dense_At, double* dense_scale) {
  cudaStream_t st = h->st;
  h->d_lump = dalloc<double>(h, h->sum_n);
  A2LS_CUDA(cudaMemsetAsync(dense_scale, 0, sizeof(double) * h->N, st));
  const size_t ea = (h->opt.precision == A2LS_FP64) ? 8 : 4;
  const size_t et = (h->opt.eig_precision == A2LS_FP32) ? 4 : 8;
  A2LS_CUDA(cudaMemsetAsync(dense_A, 0, h->fac_elems * ea, st));
  if (dense_At) A2LS_CUDA(cudaMemsetAsync(dense_At, 0, h->fac_elems * et, st));
  const int blocks = std::min(152 * 16, ceil_div((int64_t)h->sum_n * 32, 256));
  const int ep = h->opt.eig_precision;
  if (ea == 8) {
    if (ep == A2LS_FP32) launch_extract<double, float>(h, dense_A, dense_At, dense_scale, blocks);
    else if (ep == A2LS_FP32X2) launch_extract<double, dfloat>(h, dense_A, dense_At, dense_scale, blocks);
    else launch_extract<double, double>(h, dense_A, dense_At, dense_scale, blocks);
  } else {
    if (ep == A2LS_FP32) launch_extract<float, float>(h, dense_A, dense_At, dense_scale, blocks);
    else if (ep == A2LS_FP32X2) launch_extract<float, dfloat>(h, dense_A, dense_At, dense_scale, blocks);
    else launch_extract<float, double>(h, dense_A, dense_At, dense_scale, blocks);
  }
  compute_profiles(h);
}

}  // namespace a2ls

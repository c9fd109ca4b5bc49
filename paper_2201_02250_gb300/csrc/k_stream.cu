// Streaming local solves of the apply: z_i = inv(U_i) inv(L_i) R_i r for every subdomain (the local
// solves of the deflated RAS apply, Eq. 2.4), organised so that the factor bytes flow from HBM at the
// copy engine's rate while the dependent triangular-solve chain runs on the SMs.
//
// Apply format.  After the factorisation the block-inverted LU factors of each subdomain are packed
// once into one contiguous stream in the order the solves consume them:
//   forward, block b = 0 .. nb-1:   LP  panel L[r0 .. r0 + 64)[c_b .. r0), column-major (64 rows a
//                                       column), c_b the first envelope column of the block's rows
//                                   LD  row rr of inv(L_bb): columns r0 .. r0 + rr   (strictly lower)
//   backward, block b = nb-1 .. 0:  UD  row rr of inv(U_bb): columns r0 + rr .. r0 + 64
//                                   UP  panel U[g_b .. r0)[r0 .. r0 + 64), in row blocks stored
//                                       column-major, g_b the first envelope row of the block's columns
// The panels are dense over the block (the entries outside a row's or column's own envelope are exact
// zeros: 19 % more bytes than the envelope on the 96^3 convection-diffusion subdomains) because a dense
// panel is a plain product in shared memory: a thread takes a few rows and a subset of the columns, with
// no per-row reductions.  U's panel runs along the block's columns, the envelope that U keeps, so the
// backward sweep is right-looking: once x_b is known, every earlier row r receives
// -U[r][r0 .. r0 + 64) x_b.  The diagonal triangles are stored by rows, each row on 16-byte
// boundaries (its column range rounded outwards; the entries added are zeros).
// Chunks hold at most 32 KB: 128 (FP32) or 256 (BF16) columns of an L panel, 28 groups of 16 bytes of
// rows of a U panel (a column stride of 64 bytes modulo 128 keeps the reads conflict-free), or one
// diagonal triangle (its row offsets are prefix sums of the rounded row lengths).
//
// Kernel.  One or two CTAs per SM, persistent over a work queue of the subdomains (largest first).
// One producer warp streams the chunks through a ring of shared-memory stages with bulk asynchronous
// copies (cp.async.bulk, completion counted in bytes on an mbarrier per stage); each stage also
// receives the chunk's header, so that the consumers read no global memory but the right-hand side
// and their outputs.  The consumer warps run the solves from shared memory: the panel products, the
// 64 x 64 triangle products of the diagonal blocks and the right-looking updates, with the gathered
// right-hand side and the solution held in shared memory.  The producer runs ahead across block and
// subdomain boundaries, so the loads never wait for the solve chain.
// Every wait is bounded; a wait that gives up records A2LS_ERR_TIMEOUT and the CTA leaves after its
// copies in flight have landed.
#include "a2ls_internal.cuh"
#include "tc_sm100.cuh"

#include <algorithm>
#include <queue>

namespace a2ls {
namespace lss {

constexpr int STAGE_DATA = 32768;                // factor bytes per stage
constexpr int STAGE_META = 16;                   // the chunk's header
constexpr int STAGE_BYTES = STAGE_META + STAGE_DATA;
constexpr int MAX_STAGES = 8;
constexpr long WAIT_LIMIT = 1L << 26;            // polls of an mbarrier before giving up
enum { LP = 0, LD = 1, UD = 2, UP = 3 };

// The diagonal triangles of a block (tb rows) are stored by rows rounded to W elements: row rr of
// inv(L_bb) holds columns r0 .. r0 + up(rr), row rr of inv(U_bb) columns r0 + lo(rr) .. r0 + up(tb).
// Their offsets are prefix sums with closed forms: sum_{j < m} lo(j) and sum_{j < m} up(j).
template <int W> __host__ __device__ __forceinline__ int tri_sumlo(int m) {
  const int q = m / W, r = m % W;
  return W * (W * q * (q - 1) / 2 + r * q);
}
template <int W> __host__ __device__ __forceinline__ int tri_sumup(int m) {
  return tri_sumlo<W>(m) + W * (m - (m + W - 1) / W);
}
template <int W> __host__ __device__ __forceinline__ int tri_lo(int v) { return v / W * W; }
template <int W> __host__ __device__ __forceinline__ int tri_up(int v) { return (v + W - 1) / W * W; }
// elements of a block's triangles and the offset of row rr in them
template <int W> __host__ __device__ __forceinline__ int ld_elems(int tb) { return tri_sumup<W>(tb); }
template <int W> __host__ __device__ __forceinline__ int ld_off(int rr) { return tri_sumup<W>(rr); }
template <int W> __host__ __device__ __forceinline__ int ud_elems(int tb) { return tb * tri_up<W>(tb) - tri_sumlo<W>(tb); }
template <int W> __host__ __device__ __forceinline__ int ud_off(int rr, int tb) {
  return rr * tri_up<W>(tb) - tri_sumlo<W>(rr);
}

template <class T> struct V16;                   // elements per 16 bytes
template <> struct V16<float> { static constexpr int W = 4; };
template <> struct V16<__nv_bfloat16> { static constexpr int W = 8; };

// the W values of the 16 bytes at d (shared memory)
__device__ __forceinline__ void unpack16(const float* d, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(d);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void unpack16(const __nv_bfloat16* d, float (&v)[8]) {
  const uint4 a = *reinterpret_cast<const uint4*>(d);
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = __uint_as_float(w[k] << 16);
    v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned), completion
// counted on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}
// named barrier 1 over the NT consumer threads; returns the OR of v over them (uniform)
template <int NT>
__device__ __forceinline__ int consumer_sync_or(int v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(v), "n"(NT)
      : "memory");
  return r;
}

// meta: per chunk a header int4 {first column (LP) or row (UP) of the panel, kind | block << 2,
// elements, element offset of its data in the subdomain's stream}.
// xcap: floats of each shared vector (the largest subdomain rounded up to 64 rows).
// CW consumer warps and one producer warp; CTAS_PER_SM CTAs share an SM, each on its own subdomains, so
// that one CTA's dependent chain of diagonal steps overlaps the others' panel streaming.  Work queue:
// the producer claims the next subdomain (in the order sched, largest first; *counter zero at launch)
// when it reaches that subdomain's first chunk, and every stage carries the subdomain it belongs to; a
// stage marked -1 ends the work.
template <class T, int CW, int CTAS_PER_SM>
__global__ void __launch_bounds__(32 * CW + 32, CTAS_PER_SM) k_local_solve_stream(
    int nstages, int xcap, int nwork, const int* __restrict__ sched, int* __restrict__ counter,
    const int* __restrict__ choff, const int4* __restrict__ meta, const int64_t* __restrict__ soff,
    const T* __restrict__ stream, const int* __restrict__ off,
    const int* __restrict__ nI, const int* __restrict__ ni, const int* __restrict__ idx, const double* __restrict__ D,
    const double* __restrict__ t, const double* __restrict__ q, double* __restrict__ out, int mode, int* st) {
  constexpr int W = V16<T>::W;
  constexpr int CONSUMER_WARPS = CW, CONSUMERS = 32 * CW;
  // diagonal blocks: LPR lanes a row (one 16-byte vector each), RPI rows a warp step, RPW rows a warp,
  // IT steps
  constexpr int LPR = 64 / W, RPI = 32 / LPR, RPW = 64 / CW, IT = RPW / RPI;
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char* stages = sm;                                                  // nstages x STAGE_BYTES
  float* rhs = reinterpret_cast<float*>(sm + (size_t)nstages * STAGE_BYTES);  // xcap: R_i r, then the solution
  float* x = rhs + xcap;                                                       // xcap: y, then the backward work
  float* part = x + xcap;                                                      // CW x 64: each warp's panel sums
  float* s64 = part + CW * 64;                                                 // 64: the block's s = rhs - L y
  __shared__ __align__(8) uint64_t full[MAX_STAGES], empty[MAX_STAGES];
  __shared__ int stage_sub[MAX_STAGES];
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < nstages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], CONSUMER_WARPS);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == CONSUMER_WARPS) {
    // ---- producer warp: claims subdomains one after another; their chunk headers are read 32 at a time
    // (one per lane); lane 0 issues the copies of every chunk, in order
    int k = 0;
    bool ok = true;
    for (;;) {
      int i = -1;
      if (lane == 0) {
        const int w = atomicAdd(counter, 1);
        i = w < nwork ? sched[w] : -1;
      }
      i = __shfl_sync(0xffffffffu, i, 0);
      if (i < 0) {
        // the end of the work: a stage without copies, marked -1
        if (lane == 0) {
          const int s = k % nstages;
          if (tc::mbar_wait_bounded(&empty[s], ((k / nstages) & 1) ^ 1, WAIT_LIMIT) && !abort_flag) {
            stage_sub[s] = -1;
            mbar_arrive_expect_tx(&full[s], 0);
            ++k;
          } else {
            ok = false;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        break;
      }
      const T* base = stream + soff[i];
      const int c1 = choff[i + 1];
      for (int cb = choff[i]; cb < c1 && ok; cb += 32) {
        const int cnt = min(32, c1 - cb);
        int4 hd = make_int4(0, 0, 0, 0);
        if (lane < cnt) hd = meta[cb + lane];
        for (int u = 0; u < cnt; ++u, ++k) {
          const int elems = __shfl_sync(0xffffffffu, hd.z, u);
          const int doff = __shfl_sync(0xffffffffu, hd.w, u);
          const int s = k % nstages;
          int good = 1;
          if (lane == 0) {
            good = tc::mbar_wait_bounded(&empty[s], ((k / nstages) & 1) ^ 1, WAIT_LIMIT) && !abort_flag;
            if (good) {
              const uint32_t mbytes = STAGE_META, dbytes = (uint32_t)elems * (uint32_t)sizeof(T);
              unsigned char* dst = stages + (size_t)s * STAGE_BYTES;
              stage_sub[s] = i;  // published to the consumers by the arrival below
              mbar_arrive_expect_tx(&full[s], mbytes + dbytes);
              bulk_g2s(dst, meta + cb + u, mbytes, &full[s]);
              if (dbytes) bulk_g2s(dst + STAGE_META, base + doff, dbytes, &full[s]);
            }
          }
          if (!__shfl_sync(0xffffffffu, good, 0)) {
            ok = false;
            break;
          }
        }
      }
      if (!ok) break;
    }
    if (lane == 0) {
      if (!ok) {
        abort_flag = 1;
        raise_status(st, A2LS_ERR_TIMEOUT, blockIdx.x, 10);
      }
      // the copies of the last chunk of every stage have landed before the CTA may leave
      for (int j = max(0, k - nstages); j < k; ++j)
        tc::mbar_wait_bounded(&full[j % nstages], (j / nstages) & 1, WAIT_LIMIT);
    }
    __syncwarp();
    return;
  }

  // ---- consumers
  int k = 0, aborted = 0;
  for (;;) {
    // the first stage of the next subdomain (or the end mark); the barrier also keeps the previous
    // subdomain's output ahead of the gather below
    bool have0 = !aborted && tc::mbar_wait_bounded(&full[k % nstages], (k / nstages) & 1, WAIT_LIMIT);
    if (!have0) aborted = 1;
    const int i = have0 ? stage_sub[k % nstages] : -1;
    if (consumer_sync_or<CONSUMERS>(aborted)) {
      aborted = 1;
      break;
    }
    if (i < 0) break;  // the same stage for every warp: uniform
    const int n = ni[i], o = off[i];
    for (int l = tid; l < xcap; l += CONSUMERS) {
      rhs[l] = l < n ? (float)t[idx[o + l]] : 0.f;
      x[l] = 0.f;
    }
    for (int e = tid; e < CW * 64; e += CONSUMERS) part[e] = 0.f;
    if (consumer_sync_or<CONSUMERS>(aborted)) {
      aborted = 1;
      break;
    }
    const int c1 = choff[i + 1];
    for (int c = choff[i]; c < c1; ++c, ++k) {
      const int s = k % nstages;
      const unsigned char* sp = stages + (size_t)s * STAGE_BYTES;
      // (the first chunk's stage was waited for above)
      const bool have = !aborted && (c == choff[i] || tc::mbar_wait_bounded(&full[s], (k / nstages) & 1, WAIT_LIMIT));
      int4 hd;
      if (have) {
        hd = *reinterpret_cast<const int4*>(sp);
      } else {
        aborted = 1;
        hd = __ldg(&meta[c]);  // the kind keeps the barriers of this warp in step
      }
      const int kind = hd.y & 3, b = hd.y >> 2, r0 = b * 64, tb = min(64, n - r0);
      const bool diag = kind == LD || kind == UD;
      // a diagonal block needs every panel contribution before it
      if (diag && consumer_sync_or<CONSUMERS>(aborted)) {
        aborted = 1;
        break;
      }
      if (kind == LD) {
        // s = (R_i r)_b - L_b y from the warps' panel sums, which are then cleared for the next block
        if (tid < 64) {
          float sum = 0.f;
#pragma unroll
          for (int w = 0; w < CW; ++w) {
            sum += part[w * 64 + tid];
            part[w * 64 + tid] = 0.f;
          }
          s64[tid] = rhs[r0 + tid] - sum;
        }
        if (consumer_sync_or<CONSUMERS>(aborted)) {
          aborted = 1;
          break;
        }
      }
      if (have) {
        const T* data = reinterpret_cast<const T*>(sp + STAGE_META);
        if (kind == LP) {
          // part[warp][r] += sum over the chunk's columns c of L[r0 + r][c] y[c]: the chunk is column-major
          // (64 rows a column); a thread takes W rows (row group g) and the columns sub, sub + NSUB, ...
          constexpr int G = 64 / W, NSUB = CONSUMERS / G;
          const int g = tid % G, sub = tid / G;
          const int c0 = hd.x, ncols = hd.z / 64;
          const float* yc = x + c0;
          float acc[W];
#pragma unroll
          for (int v = 0; v < W; ++v) acc[v] = 0.f;
#pragma unroll 4
          for (int c = sub; c < ncols; c += NSUB) {
            float e[W];
            unpack16(data + c * 64 + g * W, e);
            const float yv = yc[c];
#pragma unroll
            for (int v = 0; v < W; ++v) acc[v] += e[v] * yv;
          }
          // the warp's 32 / G column subsets summed; lanes below G hold the sums of their W rows
#pragma unroll
          for (int o = G; o < 32; o <<= 1)
#pragma unroll
            for (int v = 0; v < W; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
          if (lane < G)
#pragma unroll
            for (int v = 0; v < W; ++v) part[warp * 64 + g * W + v] += acc[v];
        } else if (kind == LD) {
          // y[r0 + rr] = s[rr] + sum_{c < rr} inv(L_bb)[rr][c] s[c]: LPR lanes a row, one 16-byte vector
          // each; a warp's rows RPI at a time, their reductions interleaved at the end
          const int q = lane % LPR, sl = lane / LPR;
          float sv[W], e[W], acc[IT];
#pragma unroll
          for (int v = 0; v < W; ++v) sv[v] = s64[q * W + v];
#pragma unroll
          for (int it = 0; it < IT; ++it) {
            const int rr = warp * RPW + it * RPI + sl;
            float a = 0.f;
            if (rr < tb) {
              if (q * W < tri_up<W>(rr)) {
                unpack16(data + ld_off<W>(rr) + q * W, e);
#pragma unroll
                for (int v = 0; v < W; ++v)
                  if (q * W + v < rr) a += e[v] * sv[v];
              }
            }
            acc[it] = a;
          }
#pragma unroll
          for (int o = 1; o < LPR; o <<= 1)
#pragma unroll
            for (int it = 0; it < IT; ++it) acc[it] += __shfl_xor_sync(0xffffffffu, acc[it], o);
#pragma unroll
          for (int it = 0; it < IT; ++it) {
            const int rr = warp * RPW + it * RPI + sl;
            if (rr < tb && q == 0) x[r0 + rr] = s64[rr] + acc[it];
          }
        } else if (kind == UD) {
          // solution rows: rhs[r0 + rr] = sum_{c >= rr} inv(U_bb)[rr][c] y[r0 + c], mapped as above
          const int q = lane % LPR, sl = lane / LPR;
          float yv[W], e[W], acc[IT];
#pragma unroll
          for (int v = 0; v < W; ++v) yv[v] = x[r0 + q * W + v];
#pragma unroll
          for (int it = 0; it < IT; ++it) {
            const int rr = warp * RPW + it * RPI + sl;
            float a = 0.f;
            if (rr < tb) {
              const int first = tri_lo<W>(rr);  // the row's first stored column
              if (q * W >= first && q * W < tri_up<W>(tb)) {
                unpack16(data + ud_off<W>(rr, tb) + (q * W - first), e);
#pragma unroll
                for (int v = 0; v < W; ++v)
                  if (q * W + v >= rr && q * W + v < tb) a += e[v] * yv[v];
              }
            }
            acc[it] = a;
          }
#pragma unroll
          for (int o = 1; o < LPR; o <<= 1)
#pragma unroll
            for (int it = 0; it < IT; ++it) acc[it] += __shfl_xor_sync(0xffffffffu, acc[it], o);
#pragma unroll
          for (int it = 0; it < IT; ++it) {
            const int rr = warp * RPW + it * RPI + sl;
            if (rr < tb && q == 0) rhs[r0 + rr] = acc[it];
          }
        } else {
          // right-looking update of the rows above the block: y[r] -= sum_{cc < 64} U[r][r0 + cc] x[r0 + cc]
          // for the chunk's rows r = ra .. ra + R.  The chunk is column-major, R rows a column (R x the
          // element size = 64 bytes modulo 128, so that the two columns a quarter-warp reads fall on
          // different banks); a warp takes 4 groups of W rows and its lanes 8 column subsets
          const int ra = hd.x, R = hd.z / 64, ng = R / W;
          const int sub = lane >> 2;
          for (int gb = warp * 4; gb < ng; gb += 4 * CW) {
            const int gq = gb + (lane & 3);
            float acc[W];
#pragma unroll
            for (int v = 0; v < W; ++v) acc[v] = 0.f;
            if (gq < ng) {
#pragma unroll 4
              for (int cc = sub; cc < 64; cc += 8) {
                float e[W];
                unpack16(data + cc * R + gq * W, e);
                const float xv = rhs[r0 + cc];
#pragma unroll
                for (int v = 0; v < W; ++v) acc[v] += e[v] * xv;
              }
            }
#pragma unroll
            for (int o = 4; o < 32; o <<= 1)
#pragma unroll
              for (int v = 0; v < W; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
            if (gq < ng && lane < 4)
#pragma unroll
              for (int v = 0; v < W; ++v) x[ra + gq * W + v] -= acc[v];
          }
        }
      }
      __syncwarp();
      if (have && lane == 0) mbar_arrive(&empty[s]);
      if (diag && consumer_sync_or<CONSUMERS>(aborted)) {
        aborted = 1;
        break;
      }
    }
    if (aborted) break;
    // rhs holds the local solution
    if (mode == 0) {
      const int n_I = nI[i];
      for (int l = tid; l < n_I; l += CONSUMERS) {
        const int gidx = idx[o + l];
        out[gidx] = (q ? q[gidx] : 0.0) + (double)rhs[l];
      }
    } else {
      for (int l = tid; l < n; l += CONSUMERS) out[o + l] = (mode == 1 ? D[o + l] : 1.0) * (double)rhs[l];
    }
  }
  if (aborted) {
    abort_flag = 1;
    if (tid == 0) raise_status(st, A2LS_ERR_TIMEOUT, blockIdx.x, 11);
  }
}

// Pack one chunk per CTA (256 threads) from the dense block-inverted factors F (row-major, leading
// dimension ld) into the stream.  The panels are transposes of F's layout: they pass through a shared
// tile (row stride padded by one element) so that both the reads of F and the writes of the stream
// are coalesced.  Entries outside a segment's own part (the other triangle of a diagonal tile, rows or
// columns past the block, the rounding of a triangle's rows) are written as zeros.
template <class T>
__global__ void __launch_bounds__(256) k_pack_stream(int nchunks, int N, const int* __restrict__ choff,
                                                     const int4* __restrict__ meta, const int64_t* __restrict__ soff,
                                                     const int* __restrict__ ni, const int* __restrict__ ld,
                                                     const int64_t* __restrict__ foff, const T* __restrict__ fac,
                                                     T* __restrict__ stream) {
  __shared__ T tile[64 * 65];
  const int tid = threadIdx.x;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    int lo = 0, hi = N;  // choff[lo] <= c < choff[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (choff[mid] <= c) lo = mid; else hi = mid;
    }
    const int i = lo, n = ni[i];
    const int64_t L = ld[i];
    const T* F = fac + foff[i];
    const int4 hd = meta[c];
    T* dst = stream + soff[i] + hd.w;
    const int kind = hd.y & 3, r0 = (hd.y >> 2) * 64, tb = min(64, n - r0);
    if (kind == LP) {
      // column-major: (c0 + cl, rr) at cl * 64 + rr = L[r0 + rr][c0 + cl], in groups of 64 columns
      const int c0 = hd.x, ncols = hd.z / 64;
      for (int g = 0; g < ncols; g += 64) {
        const int gc = min(64, ncols - g);
        __syncthreads();
        for (int e = tid; e < 64 * 64; e += 256) {
          const int rr = e >> 6, cl = e & 63;
          if (cl < gc) tile[rr * 65 + cl] = rr < tb ? F[(int64_t)(r0 + rr) * L + c0 + g + cl] : T(0.f);
        }
        __syncthreads();
        for (int e = tid; e < gc * 64; e += 256) {
          const int cl = e >> 6, rr = e & 63;
          dst[(int64_t)(g + cl) * 64 + rr] = tile[rr * 65 + cl];
        }
      }
    } else if (kind == UP) {
      // column-major: (ra + rl, cc) at cc * R + rl = U[ra + rl][r0 + cc], in groups of 64 rows
      const int ra = hd.x, R = hd.z / 64;
      for (int g = 0; g < R; g += 64) {
        const int gr = min(64, R - g);
        __syncthreads();
        for (int e = tid; e < 64 * 64; e += 256) {
          const int rl = e >> 6, cc = e & 63;
          if (rl < gr) tile[rl * 65 + cc] = cc < tb ? F[(int64_t)(ra + g + rl) * L + r0 + cc] : T(0.f);
        }
        __syncthreads();
        for (int e = tid; e < 64 * gr; e += 256) {
          const int cc = e / gr, rl = e % gr;
          dst[(int64_t)cc * R + g + rl] = tile[rl * 65 + cc];
        }
      }
    } else {
      constexpr int W = V16<T>::W;
      const int warp = tid >> 5, lane = tid & 31;
      for (int rr = warp; rr < tb; rr += 8) {
        const int c0 = kind == LD ? 0 : tri_lo<W>(rr), c1 = kind == LD ? tri_up<W>(rr) : tri_up<W>(tb);
        T* row = dst + (kind == LD ? ld_off<W>(rr) : ud_off<W>(rr, tb)) - c0;
        for (int cc = c0 + lane; cc < c1; cc += 32) {
          T v = T(0.f);
          if (kind == LD) {
            if (cc < rr) v = F[(int64_t)(r0 + rr) * L + r0 + cc];               // inv(L_bb), strictly lower
          } else {
            if (cc >= rr && cc < tb) v = F[(int64_t)(r0 + rr) * L + r0 + cc];   // inv(U_bb), upper
          }
          row[cc] = v;
        }
      }
    }
  }
}

}  // namespace lss

// ---------------------------------------------------------------------------
// Host side: the plan of the stream (segments, chunks, offsets), the packing, the schedule.
// ---------------------------------------------------------------------------
template <class T>
void stream_prepare(a2ls_handle* h, const T* fac) {
  using namespace lss;
  constexpr int W = V16<T>::W;
  cudaStream_t st = h->st;
  const int N = h->N;
  std::vector<int> pf(h->sum_n), pg(h->sum_n);
  A2LS_CUDA(cudaMemcpyAsync(pf.data(), h->d_pf, sizeof(int) * h->sum_n, cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaMemcpyAsync(pg.data(), h->d_pg, sizeof(int) * h->sum_n, cudaMemcpyDeviceToHost, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
  auto lo = [](int v) { return v / W * W; };
  // panel chunks: L by 64-row columns (32 KB), U by 64-column row blocks of 28 groups of W rows (the
  // column stride, 448 bytes, is 64 modulo 128)
  const int lp_cols = STAGE_DATA / (64 * (int)sizeof(T));
  const int up_rows = 28 * W;
  std::vector<int4> meta;  // one header per chunk
  std::vector<int> choff(N + 1, 0);
  std::vector<int64_t> soff(N + 1, 0);
  std::vector<double> cost(N, 0.0);
  meta.reserve((size_t)h->sum_n / 8 + (size_t)N * 64);
  for (int i = 0; i < N; ++i) {
    const int n = h->h_n[i], o = h->h_off[i], nb = (n + TB - 1) / TB;
    int off = 0;
    choff[i] = (int)meta.size();
    // header {first column or row (panels), kind | block << 2, elements, data offset}
    auto chunk = [&](int kind, int b, int first, int elems) {
      meta.push_back(make_int4(first, kind | (b << 2), elems, off));
      off += elems;
    };
    for (int b = 0; b < nb; ++b) {
      const int r0 = b * TB, tb = std::min(TB, n - r0);
      // L panel of the block: columns from the first envelope column of its rows up to r0, all 64 rows
      int cmin = r0;
      for (int r = r0; r < r0 + tb; ++r) cmin = std::min(cmin, lo(pf[o + r]));
      for (int c = cmin; c < r0; c += lp_cols) chunk(LP, b, c, 64 * std::min(lp_cols, r0 - c));
      chunk(LD, b, 0, ld_elems<W>(tb));
    }
    for (int b = nb - 1; b >= 0; --b) {
      const int r0 = b * TB, tb = std::min(TB, n - r0);
      chunk(UD, b, 0, ud_elems<W>(tb));
      // U panel of the block: rows from the first envelope row of its columns up to r0, all 64 columns
      int rmin = r0;
      for (int c = r0; c < r0 + tb; ++c) rmin = std::min(rmin, lo(pg[o + c]));
      for (int r = rmin; r < r0; r += up_rows) chunk(UP, b, r, 64 * std::min(up_rows, r0 - r));
    }
    soff[i + 1] = soff[i] + off;
    // work-queue order: copy time of the bytes plus the dependent chain of 2 nb diagonal steps (about
    // 2 us each, the time the copy engine moves 64 KB for one SM)
    cost[i] = (double)off * sizeof(T) + 2.0 * nb * 65536.0;
  }
  choff[N] = (int)meta.size();
  // device copies of the plan
  StreamSolve& S = h->ss;
  S.elem_bytes = (int)sizeof(T);
  S.nchunks = (int)meta.size();
  S.stream_elems = soff[N];
  S.d_stream = dalloc<T>(h, (size_t)soff[N] + W);
  S.d_meta = dalloc<int4>(h, meta.size());
  S.d_choff = dalloc<int>(h, N + 1);
  S.d_soff = dalloc<int64_t>(h, N + 1);
  A2LS_CUDA(cudaMemcpyAsync(S.d_meta, meta.data(), sizeof(int4) * meta.size(), cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(S.d_choff, choff.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaMemcpyAsync(S.d_soff, soff.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
  int dev = 0, sms = 152, optin = 0, per_sm = 0;
  A2LS_CUDA(cudaGetDevice(&dev));
  A2LS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  A2LS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  A2LS_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  const int blocks = std::max(1, std::min(sms * 16, S.nchunks));
  k_pack_stream<T><<<blocks, 256, 0, st>>>(S.nchunks, N, S.d_choff, S.d_meta, S.d_soff, h->d_ni,
                                                h->d_fld, h->d_ffoff, fac, static_cast<T*>(S.d_stream));
  A2LS_LAUNCH();
  S.xcap = (int)round_up(h->max_n, TB);
  // the two vectors, the warps' panel sums (8 warps at most) and the block's s
  const size_t fixed = sizeof(float) * (2 * (size_t)S.xcap + 8 * 64 + 64);
  // the kernel shapes: 8 consumer warps, one CTA per SM; 4 consumer warps, two CTAs per SM; 8 consumer
  // warps, two CTAs per SM
  for (int v = 0; v < 3; ++v) {
    StreamSolve::Shape& sh = S.shape[v];
    const int ctas = v == 0 ? 1 : 2;
    // shared memory per CTA: the SM's share less the 1 KB the hardware reserves per CTA and the static part
    const size_t budget = std::min<size_t>((size_t)optin, (size_t)per_sm / ctas - 1024) - 512;
    sh.nstages = (int)std::min<size_t>(MAX_STAGES, budget > fixed ? (budget - fixed) / STAGE_BYTES : 0);
    sh.smem = (size_t)sh.nstages * STAGE_BYTES + fixed;
    if (sh.nstages < 2) continue;
    int occ = 0;
    if (v == 0) {
      A2LS_CUDA(cudaFuncSetAttribute(k_local_solve_stream<T, 8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sh.smem));
      A2LS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_local_solve_stream<T, 8, 1>, 288, sh.smem));
    } else if (v == 1) {
      A2LS_CUDA(cudaFuncSetAttribute(k_local_solve_stream<T, 4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sh.smem));
      A2LS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_local_solve_stream<T, 4, 2>, 160, sh.smem));
    } else {
      A2LS_CUDA(cudaFuncSetAttribute(k_local_solve_stream<T, 8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sh.smem));
      A2LS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_local_solve_stream<T, 8, 2>, 288, sh.smem));
    }
    if (occ < ctas) continue;
    sh.ncta = std::max(1, std::min(N, sms * ctas));
    sh.ready = true;
  }
  S.ready = S.shape[0].ready || S.shape[1].ready || S.shape[2].ready;
  // the work order of the queue: the subdomains by decreasing cost
  std::vector<int> order(N);
  for (int i = 0; i < N; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  S.d_order = dalloc<int>(h, N);
  A2LS_CUDA(cudaMemcpyAsync(S.d_order, order.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  A2LS_CUDA(cudaStreamSynchronize(st));
}

// config: LS_STREAM (8 consumer warps, one CTA per SM), LS_STREAM2 (4 consumer warps, two CTAs per SM) or
// LS_STREAM3 (8 consumer warps, two CTAs per SM)
template <class T>
void launch_local_solve_stream(a2ls_handle* h, int config, const double* t, const double* q, double* z, int mode) {
  using namespace lss;
  const StreamSolve& S = h->ss;
  const int v = config == LS_STREAM2 ? 1 : (config == LS_STREAM3 ? 2 : 0);
  const StreamSolve::Shape& sh = S.shape[v];
  if (!sh.ready || S.elem_bytes != (int)sizeof(T)) fail(A2LS_ERR_ARG, "streaming local solves not prepared");
  A2LS_CUDA(cudaMemsetAsync(h->d_counter, 0, sizeof(int), h->st));
  if (v == 0)
    k_local_solve_stream<T, 8, 1><<<sh.ncta, 288, sh.smem, h->st>>>(
        sh.nstages, S.xcap, h->N, S.d_order, h->d_counter, S.d_choff, S.d_meta, S.d_soff,
        static_cast<const T*>(S.d_stream), h->d_off, h->d_nI, h->d_ni, h->d_idx, h->d_D, t, q, z, mode, h->d_status);
  else if (v == 2)
    k_local_solve_stream<T, 8, 2><<<sh.ncta, 288, sh.smem, h->st>>>(
        sh.nstages, S.xcap, h->N, S.d_order, h->d_counter, S.d_choff, S.d_meta, S.d_soff,
        static_cast<const T*>(S.d_stream), h->d_off, h->d_nI, h->d_ni, h->d_idx, h->d_D, t, q, z, mode, h->d_status);
  else
    k_local_solve_stream<T, 4, 2><<<sh.ncta, 160, sh.smem, h->st>>>(
        sh.nstages, S.xcap, h->N, S.d_order, h->d_counter, S.d_choff, S.d_meta, S.d_soff,
        static_cast<const T*>(S.d_stream), h->d_off, h->d_nI, h->d_ni, h->d_idx, h->d_D, t, q, z, mode, h->d_status);
  A2LS_LAUNCH();
}

template void stream_prepare<float>(a2ls_handle*, const float*);
template void stream_prepare<__nv_bfloat16>(a2ls_handle*, const __nv_bfloat16*);
template void launch_local_solve_stream<float>(a2ls_handle*, int, const double*, const double*, double*, int);
template void launch_local_solve_stream<__nv_bfloat16>(a2ls_handle*, int, const double*, const double*, double*,
                                                        int);

}  // namespace a2ls

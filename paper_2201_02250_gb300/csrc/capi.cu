// C ABI of libA2LS: argument checks, setup orchestration, queries.
#include "a2ls_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>

namespace a2ls {

static thread_local std::string g_last_error;

void fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  throw Error(code, buf);
}

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  const char* base = strrchr(file, '/');
  fail(e == cudaErrorMemoryAllocation ? A2LS_ERR_OOM : A2LS_ERR_CUDA, "%s failed: %s (%s:%d)", what,
       cudaGetErrorString(e), base ? base + 1 : file, line);
}

void launched(a2ls_handle* h, cudaError_t e, const char* file, int line) {
  if (h) ++h->launches;
  check_cuda(e, "kernel launch", file, line);
}

static cudaEvent_t pool_event(a2ls_handle* h) {
  if (!h->kt_pool.empty()) {
    cudaEvent_t e = h->kt_pool.back();
    h->kt_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  A2LS_CUDA(cudaEventCreate(&e));
  return e;
}

KTime::KTime(a2ls_handle* hh, int kid, double work) : h(hh), id(kid) {
  if (h && h->opt.timing) {
    h->kt_work[kid] += work;
    b = pool_event(h);
    A2LS_CUDA(cudaEventRecord(b, h->st));
  }
}

KTime::~KTime() {
  if (!b) return;
  cudaEvent_t e = pool_event(h);
  cudaEventRecord(e, h->st);
  h->kt_events[id].push_back({b, e});
}

void collect_kernel_times(a2ls_handle* h) {
  for (int k = 0; k < KT_COUNT; ++k) {
    for (auto& pr : h->kt_events[k]) {
      float ms = 0.f;
      if (cudaEventSynchronize(pr.second) == cudaSuccess && cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
        h->kt_ms[k] += ms;
        h->kt_count[k] += 1;
      }
      h->kt_pool.push_back(pr.first);
      h->kt_pool.push_back(pr.second);
    }
    h->kt_events[k].clear();
  }
}

// ---------------------------------------------------------------------------
// Device memory of the handles comes from one stream-ordered memory pool per device owned by the
// library.  Its release threshold is unbounded: blocks freed by a handle stay mapped for the next
// allocation, so repeated setups of the same size neither map nor unmap gigabytes (a setup of the
// 512x512 problem spends about 10 ms on that with the default pool).  a2ls_trim_memory returns the
// unused blocks.  If the pool cannot be created the default pool of the device is used.
// ---------------------------------------------------------------------------
constexpr int MAX_POOL_DEVICES = 64;
static std::mutex g_pool_mutex;
static cudaMemPool_t g_pools[MAX_POOL_DEVICES] = {};

static cudaMemPool_t library_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_POOL_DEVICES) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_pool_mutex);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
    g_pools[dev] = p;
  }
  return g_pools[dev];
}

void* dalloc_bytes(a2ls_handle* h, size_t bytes) {
  void* p = nullptr;
  const size_t sz = std::max<size_t>(bytes, 16);
  cudaError_t e = h->pool ? cudaMallocFromPoolAsync(&p, sz, h->pool, h->st) : cudaMallocAsync(&p, sz, h->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(A2LS_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  h->allocs.push_back(p);
  return p;
}

void dfree(a2ls_handle* h, void* p) {
  if (!p) return;
  auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
  if (it != h->allocs.end()) {
    h->allocs.erase(it);
    cudaFreeAsync(p, h->st);
  }
}

// ---------------------------------------------------------------------------
// autotune cache: process-wide map, mirrored in the JSON file named by A2LS_AUTOTUNE_CACHE
// ---------------------------------------------------------------------------
static std::mutex g_tune_mutex;
static std::map<std::string, int> g_tune;
static bool g_tune_loaded = false;

static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("A2LS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
  fclose(f);
  // flat JSON object {"key": int, ...}
  size_t p = 0;
  while ((p = text.find('"', p)) != std::string::npos) {
    const size_t q = text.find('"', p + 1);
    if (q == std::string::npos) break;
    const std::string key = text.substr(p + 1, q - p - 1);
    const size_t c = text.find(':', q);
    if (c == std::string::npos) break;
    g_tune[key] = atoi(text.c_str() + c + 1);
    p = text.find_first_of(",}", c);
    if (p == std::string::npos) break;
  }
}

int autotune_lookup(const char* key) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_load_locked();
  auto it = g_tune.find(key);
  return it == g_tune.end() ? 0 : it->second;
}

void autotune_store(const char* key, int value) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_load_locked();
  g_tune[key] = value;
  const char* path = getenv("A2LS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "w");
  if (!f) return;
  fprintf(f, "{");
  bool first = true;
  for (const auto& kv : g_tune) {
    fprintf(f, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
    first = false;
  }
  fprintf(f, "\n}\n");
  fclose(f);
}

static const char* status_name(int c) {
  switch (c) {
    case A2LS_ERR_ARG: return "invalid argument";
    case A2LS_ERR_SINGULAR: return "singular pivot";
    case A2LS_ERR_EIGEN: return "eigensolver";
    case A2LS_ERR_TIMEOUT: return "device wait timed out";
    default: return "device error";
  }
}

void sync_and_check(a2ls_handle* h, const char* phase) {
  A2LS_CUDA(cudaStreamSynchronize(h->st));
  int s[ST_WORDS];
  A2LS_CUDA(cudaMemcpy(s, h->d_status, sizeof(s), cudaMemcpyDeviceToHost));
  h->pivot_boosts = s[ST_BOOSTS];
  if (s[ST_CODE] != 0) {
    const int code = s[ST_CODE];
    int zero[ST_WORDS] = {0};
    A2LS_CUDA(cudaMemcpy(h->d_status, zero, sizeof(zero), cudaMemcpyHostToDevice));
    fail(code, "%s: %s (where=%d, info=%d)", phase, status_name(code), s[ST_WHERE], s[ST_AUX]);
  }
}

static void set_error(const char* msg) { g_last_error = msg ? msg : ""; }

void record_error(const char* msg) { set_error(msg); }

template <class F>
static int guarded(F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    set_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_error(e.what());
    return A2LS_ERR_CUDA;
  } catch (...) {
    set_error("unknown error");
    return A2LS_ERR_CUDA;
  }
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  double stop() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventRecord(a, st);
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

__global__ void k_max_rowlen(int n, const int* rowptr, const int* mrow, int* out) {
  int a = 0, b = 0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    a = max(a, rowptr[r + 1] - rowptr[r]);
    b = max(b, mrow[r + 1] - mrow[r]);
  }
  atomicMax(out, a);
  atomicMax(out + 1, b);
}

static void destroy_handle(a2ls_handle* h) {
  if (!h) return;
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  collect_kernel_times(h);
  for (cudaEvent_t e : h->kt_pool) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFreeAsync(p, h->st);
  h->allocs.clear();
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  cudaStreamSynchronize(h->st);
  delete h;
}

template <class T, class TT>
static void factor_and_coarse(a2ls_handle* h, bool need_coarse, double* times) {
  cudaStream_t st = h->st;
  Timer tm(st);
  const int N = h->N;
  T* fa = dalloc<T>(h, h->fac_elems);
  TT* ft = need_coarse ? dalloc<TT>(h, h->fac_elems) : nullptr;  // A~_ii factors (eigensolve precision)
  double* dscale = dalloc<double>(h, N);
  double* lastp = dalloc<double>(h, N);
  extract_local(h, fa, ft, dscale);
  sync_and_check(h, "local matrix extraction");
  times[Phase::SETUP_EXTRACT] = tm.stop();
  // algorithmic work: the flops of an LU confined to the envelope of the local pattern
  double lu_flops = 0.0, gamma_flops = 0.0;
  for (int i = 0; i < N; ++i) {
    lu_flops += h->h_env[4 * i];
    gamma_flops += h->h_env[4 * i + 1];
  }
  // A_ii and A~_ii share their interior block, so one factorisation of the splitting serves both
  // when it runs in at least the precision of the A_ii factors; only the Schur complement on the
  // overlap rows is factored twice.
  const bool share = need_coarse && Unit<TT>::u <= Unit<T>::u;
  // With a shared factorisation the overlap pivots of A_ii (T) need only the Schur complement copied
  // from the splitting's interior factors: they run on a second stream, alongside the splitting's
  // overlap pivots and the eigensolve, and join the handle's stream at the end (sequential when the
  // per-kernel timing is on, so that each kernel's events see it alone).
  struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    ~SideStream() {
      if (done) cudaEventDestroy(done);
      if (s) {
        // on an error path the handle frees the factors next: nothing may still write them
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    }
  } side;
  const bool overlap_local = share && !h->opt.timing;
  if (!share) {
    KTime kt(h, KT_LU_LOCAL, lu_flops);
    lu_batched<T>(h, fa, 0, nullptr, dscale);
    invert_diag_tiles<T>(h, fa);
  }
  if (need_coarse) {
    {
      KTime kt(h, KT_LU_SPLIT, lu_flops);
      if (share) {
        lu_batched<TT>(h, ft, 1, lastp, dscale, 0);
        schur_copy<TT, T>(h, ft, fa, lastp);
        if (overlap_local) {
          cudaEvent_t copied;
          A2LS_CUDA(cudaEventCreateWithFlags(&copied, cudaEventDisableTiming));
          A2LS_CUDA(cudaEventRecord(copied, st));
          A2LS_CUDA(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking));
          A2LS_CUDA(cudaEventCreateWithFlags(&side.done, cudaEventDisableTiming));
          A2LS_CUDA(cudaStreamWaitEvent(side.s, copied, 0));
          A2LS_CUDA(cudaEventDestroy(copied));
          {
            struct Restore {  // the handle's stream comes back on every exit path
              a2ls_handle* h;
              cudaStream_t st;
              ~Restore() { h->st = st; }
            } restore{h, st};
            h->st = side.s;
            lu_batched<T>(h, fa, 0, nullptr, dscale, 1);
            invert_diag_tiles<T>(h, fa);
          }
          A2LS_CUDA(cudaEventRecord(side.done, side.s));
        }
        lu_batched<TT>(h, ft, 1, lastp, dscale, 1);
      } else {
        lu_batched<TT>(h, ft, 1, lastp, dscale);
      }
      invert_diag_tiles<TT>(h, ft);
    }
    if (share && !overlap_local) {
      KTime kt(h, KT_LU_LOCAL, gamma_flops);
      lu_batched<T>(h, fa, 0, nullptr, dscale, 1);
      invert_diag_tiles<T>(h, fa);
    }
  }
  sync_and_check(h, "LU factorisation of the local matrices and splittings");
  h->d_fac = fa;
  times[Phase::SETUP_LU] = tm.stop();
  if (need_coarse) {
    eigensolve(h, ft, lastp, dscale);  // ends with the coarse operator
    dfree(h, ft);
  }
  if (side.done) A2LS_CUDA(cudaStreamWaitEvent(st, side.done, 0));  // the A_ii factors are complete
  times[Phase::SETUP_EIG] = tm.stop();
  dfree(h, dscale);
  dfree(h, lastp);
}

}  // namespace a2ls

using namespace a2ls;

extern "C" {

void a2ls_default_options(a2ls_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = A2LS_FP64;
  o->variant = A2LS_DEFLATED_RAS;
  o->pou = A2LS_POU_BOOLEAN;
  o->restart = 30;
  o->max_it = 1000;
  o->flexible = -1;
  o->tau = 0.0;
  o->eig_block_steps = 3;
  o->eig_max_cycles = 60;
  o->eig_tol = 0.0;
  o->seed = 12345;
  o->stream = nullptr;
  o->timing = 0;
  o->eig_precision = -1;
  o->graphs = 1;
  o->warm_start = nullptr;
  o->eig_strict = 0;
  o->eig_stall_cycles = 8;
  o->tensor_cores = 1;
  o->eig_thick_restart = 1;
  o->local_solve_kernel = 0;
  o->eig_block_size = 0;
  o->static_pivoting = 0;
}

const char* a2ls_last_error(void) { return g_last_error.c_str(); }

int a2ls_partition(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t nparts, uint64_t seed,
                   int32_t* part) {
  set_error("");
  return guarded([&] {
    partition_graph(n, rowptr, colind, nparts, seed, part);
    return (int)A2LS_OK;
  });
}

int a2ls_trim_memory(void) {
  set_error("");
  std::lock_guard<std::mutex> lk(g_pool_mutex);
  for (int d = 0; d < MAX_POOL_DEVICES; ++d) {
    if (!g_pools[d]) continue;
    const cudaError_t e = cudaMemPoolTrimTo(g_pools[d], 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      char msg[256];
      snprintf(msg, sizeof(msg), "cudaMemPoolTrimTo on device %d: %s", d, cudaGetErrorString(e));
      set_error(msg);
      return A2LS_ERR_CUDA;
    }
  }
  return A2LS_OK;
}

int a2ls_setup(const a2ls_csr* A, const int32_t* partition, int32_t overlap, int32_t nev,
               const a2ls_options* opt, a2ls_handle** out) {
  set_error("");
  if (out) *out = nullptr;
  a2ls_handle* h = nullptr;
  int rc = guarded([&]() -> int {
    if (!A || !out || !partition) fail(A2LS_ERR_ARG, "null argument");
    if (A->n <= 0) fail(A2LS_ERR_ARG, "n must be positive (got %d)", A->n);
    if (A->nnz < A->n) fail(A2LS_ERR_ARG, "nnz = %d is smaller than n = %d (every row needs its diagonal)", A->nnz, A->n);
    if (!A->rowptr || !A->colind || !A->val) fail(A2LS_ERR_ARG, "null CSR array");
    if (overlap < 0) fail(A2LS_ERR_ARG, "overlap must be >= 0");
    if (nev < 0) fail(A2LS_ERR_ARG, "nev must be >= 0");
    a2ls_options o;
    if (opt) o = *opt; else a2ls_default_options(&o);
    if (o.precision != A2LS_FP64 && o.precision != A2LS_FP32 && o.precision != A2LS_BF16)
      fail(A2LS_ERR_ARG, "unknown precision %d", o.precision);
    if (o.variant < 0 || o.variant > A2LS_ONE_LEVEL_ASM) fail(A2LS_ERR_ARG, "unknown variant %d", o.variant);
    if (o.pou != A2LS_POU_BOOLEAN && o.pou != A2LS_POU_MULTIPLICITY) fail(A2LS_ERR_ARG, "unknown partition of unity %d", o.pou);
    if (o.static_pivoting != 0 && o.static_pivoting != 1) fail(A2LS_ERR_ARG, "static_pivoting must be 0 or 1");
    {
      const int k = o.local_solve_kernel;
      if (k != 0 && k != 256 && k != 512 && k != 1024 && k != 1256 && k != 1512 && k != 2256 && k != LS_STREAM &&
          k != LS_STREAM2 && k != LS_STREAM3)
        fail(A2LS_ERR_ARG, "unknown local_solve_kernel %d", k);
      if ((k == LS_STREAM || k == LS_STREAM2 || k == LS_STREAM3) && o.precision == A2LS_FP64)
        fail(A2LS_ERR_ARG, "local_solve_kernel %d needs FP32 or BF16 local factors", k);
    }
    h = new a2ls_handle();
    h->opt = o;
    h->st = static_cast<cudaStream_t>(o.stream);
    h->pool = library_pool();
    h->n = A->n;
    h->nnz = A->nnz;
    h->delta = overlap;
    h->nev = nev;
    cudaStream_t st = h->st;
    Timer total(st), tm(st);
    h->d_status = dalloc<int>(h, ST_WORDS);
    A2LS_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int) * ST_WORDS, st));
    h->rowptr = dalloc<int>(h, h->n + 1);
    h->colind = dalloc<int>(h, h->nnz);
    h->val = dalloc<double>(h, h->nnz);
    h->part = dalloc<int>(h, h->n);
    A2LS_CUDA(cudaMemcpyAsync(h->rowptr, A->rowptr, sizeof(int) * (h->n + 1), cudaMemcpyDeviceToDevice, st));
    A2LS_CUDA(cudaMemcpyAsync(h->colind, A->colind, sizeof(int) * h->nnz, cudaMemcpyDeviceToDevice, st));
    A2LS_CUDA(cudaMemcpyAsync(h->val, A->val, sizeof(double) * h->nnz, cudaMemcpyDeviceToDevice, st));
    A2LS_CUDA(cudaMemcpyAsync(h->part, partition, sizeof(int) * h->n, cudaMemcpyDeviceToDevice, st));
    build_subdomains(h);
    {
      int* mm = dalloc<int>(h, 2);
      A2LS_CUDA(cudaMemsetAsync(mm, 0, sizeof(int) * 2, st));
      k_max_rowlen<<<std::min(1216, ceil_div(h->n, 256)), 256, 0, st>>>(h->n, h->rowptr, h->d_mrow, mm);
      A2LS_LAUNCH();
      int hm[2];
      A2LS_CUDA(cudaMemcpyAsync(hm, mm, sizeof(hm), cudaMemcpyDeviceToHost, st));
      A2LS_CUDA(cudaStreamSynchronize(st));
      h->max_rownnz = hm[0];
      h->max_memb = hm[1];
      dfree(h, mm);
    }
    h->times[Phase::SETUP_GRAPH] = tm.stop();
    h->fac_elems = (size_t)h->h_foff[h->N];
    const int v = o.variant;
    const bool need_coarse = nev > 0 && v != A2LS_ONE_LEVEL_RAS && v != A2LS_ONE_LEVEL_ASM;
    const int ep = (o.eig_precision < 0) ? (o.precision == A2LS_FP64 ? A2LS_FP64 : A2LS_FP32X2) : o.eig_precision;
    if (ep != A2LS_FP64 && ep != A2LS_FP32 && ep != A2LS_FP32X2)
      fail(A2LS_ERR_ARG, "unknown eig_precision %d", o.eig_precision);
    h->opt.eig_precision = ep;
    if (o.precision == A2LS_FP64) {
      if (ep == A2LS_FP64) factor_and_coarse<double, double>(h, need_coarse, h->times);
      else if (ep == A2LS_FP32) factor_and_coarse<double, float>(h, need_coarse, h->times);
      else factor_and_coarse<double, dfloat>(h, need_coarse, h->times);
    } else {
      if (ep == A2LS_FP64) factor_and_coarse<float, double>(h, need_coarse, h->times);
      else if (ep == A2LS_FP32) factor_and_coarse<float, float>(h, need_coarse, h->times);
      else factor_and_coarse<float, dfloat>(h, need_coarse, h->times);
    }
    Timer tprep(st);
    h->h_fld = h->h_ld;
    h->h_ffoff = h->h_foff;
    h->d_fld = h->d_ld;
    h->d_ffoff = h->d_foff;
    if (o.precision == A2LS_BF16) {
      // the FP32 factors rounded to their bfloat16 storage (rows on 16-byte boundaries)
      __nv_bfloat16* fb = factors_to_bf16(h, static_cast<const float*>(h->d_fac));
      dfree(h, h->d_fac);
      h->d_fac = fb;
    }
    // the factors repacked for the streaming local solves
    if (o.precision == A2LS_BF16) stream_prepare<__nv_bfloat16>(h, static_cast<const __nv_bfloat16*>(h->d_fac));
    else if (o.precision == A2LS_FP32) stream_prepare<float>(h, static_cast<const float*>(h->d_fac));
    // apply workspace
    h->d_q = dalloc<double>(h, h->n);
    h->d_t = dalloc<double>(h, h->n);
    h->d_yloc = dalloc<double>(h, h->sum_n);
    // pick the CTA width of the local solves for this problem (timed on its own factors)
    {
      const bool ras = v == A2LS_DEFLATED_RAS || v == A2LS_ADDITIVE_RAS || v == A2LS_ONE_LEVEL_RAS;
      const int mode = ras ? (o.pou == A2LS_POU_BOOLEAN ? 0 : 1) : 2;
      A2LS_CUDA(cudaMemsetAsync(h->d_t, 0, sizeof(double) * h->n, st));
      double* scratch = mode == 0 ? h->d_q : h->d_yloc;
      const int timing = h->opt.timing;
      h->opt.timing = 0;
      if ((o.local_solve_kernel == LS_STREAM && !h->ss.shape[0].ready) ||
          (o.local_solve_kernel == LS_STREAM2 && !h->ss.shape[1].ready) ||
          (o.local_solve_kernel == LS_STREAM3 && !h->ss.shape[2].ready))
        fail(A2LS_ERR_ARG, "the streaming local solves of shape %d do not fit this device's shared memory",
             o.local_solve_kernel);
      if (o.local_solve_kernel > 0) h->ls_width = o.local_solve_kernel;
      else if (o.precision == A2LS_FP64) autotune_local_solves<double>(h, static_cast<double*>(h->d_fac), h->d_t, scratch, mode);
      else if (o.precision == A2LS_BF16)
        autotune_local_solves<__nv_bfloat16>(h, static_cast<__nv_bfloat16*>(h->d_fac), h->d_t, scratch, mode);
      else autotune_local_solves<float>(h, static_cast<float*>(h->d_fac), h->d_t, scratch, mode);
      h->opt.timing = timing;
    }
    // load the module holding a2ls_apply_static's scratch array now, while allocation is allowed
    prime_static_scratch();
    sync_and_check(h, "setup");
    h->times[Phase::SETUP_APPLY_PREP] = tprep.stop();
    h->times[Phase::SETUP_TOTAL] = total.stop();
    *out = h;
    return A2LS_OK;
  });
  if (rc != A2LS_OK && h) {
    destroy_handle(h);
    *out = nullptr;
  }
  return rc;
}

int a2ls_apply(a2ls_handle* h, const double* r, double* z) {
  if (!h || !r || !z) {
    set_error("null argument");
    return A2LS_ERR_ARG;
  }
  if (r == z) {
    set_error("r and z must not alias");
    return A2LS_ERR_ARG;
  }
  return guarded([&]() -> int {
    apply_preconditioner(h, r, z);
    return A2LS_OK;
  });
}

int a2ls_solve(a2ls_handle* h, const double* b, double* x, double rtol, int32_t* iters, double* relres) {
  if (!h || !b || !x) {
    set_error("null argument");
    return A2LS_ERR_ARG;
  }
  if (!(rtol > 0)) {
    set_error("rtol must be positive");
    return A2LS_ERR_ARG;
  }
  return guarded([&]() -> int {
    Timer tm(h->st);
    int it = 0;
    double rr = 0.0;
    int rc = gmres(h, b, x, rtol, &it, &rr);
    sync_and_check(h, "solve");
    h->times[Phase::SOLVE_TOTAL] = tm.stop();
    if (iters) *iters = it;
    if (relres) *relres = rr;
    if (rc == A2LS_ERR_NOT_CONVERGED) set_error("GMRES reached max_it before the tolerance");
    return rc;
  });
}

int a2ls_solve_multi(a2ls_handle* h, int32_t nrhs, const double* B, double* X, double rtol, int32_t* iters,
                     double* relres) {
  if (!h || (nrhs > 0 && (!B || !X))) {
    set_error("null argument");
    return A2LS_ERR_ARG;
  }
  if (nrhs < 0) {
    set_error("nrhs must be >= 0");
    return A2LS_ERR_ARG;
  }
  if (!(rtol > 0)) {
    set_error("rtol must be positive");
    return A2LS_ERR_ARG;
  }
  return guarded([&]() -> int {
    Timer tm(h->st);
    int worst = A2LS_OK;
    for (int k = 0; k < nrhs; ++k) {
      int it = 0;
      double rr = 0.0;
      const int rc = gmres(h, B + (size_t)k * h->n, X + (size_t)k * h->n, rtol, &it, &rr);
      sync_and_check(h, "solve");
      if (iters) iters[k] = it;
      if (relres) relres[k] = rr;
      if (rc != A2LS_OK) worst = rc;
    }
    h->times[Phase::SOLVE_TOTAL] = tm.stop();
    if (worst == A2LS_ERR_NOT_CONVERGED) set_error("GMRES reached max_it before the tolerance for a right-hand side");
    return worst;
  });
}

int a2ls_setup_batch(int32_t nsys, const a2ls_csr* A, const int32_t* const* partition, const int32_t* overlap,
                     const int32_t* nev, const a2ls_options* opt, a2ls_handle** out) {
  set_error("");
  if (nsys < 0 || (nsys > 0 && (!A || !partition || !overlap || !nev || !out))) {
    set_error("null argument");
    return A2LS_ERR_ARG;
  }
  for (int k = 0; k < nsys; ++k) out[k] = nullptr;
  for (int k = 0; k < nsys; ++k) {
    const int rc = a2ls_setup(&A[k], partition[k], overlap[k], nev[k], opt, &out[k]);
    if (rc != A2LS_OK) {
      const std::string msg = std::string("system ") + std::to_string(k) + ": " + a2ls_last_error();
      for (int j = 0; j < k; ++j) {
        destroy_handle(out[j]);
        out[j] = nullptr;
      }
      set_error(msg.c_str());
      return rc;
    }
  }
  return A2LS_OK;
}

void a2ls_destroy(a2ls_handle* h) { destroy_handle(h); }

int a2ls_spmv(a2ls_handle* h, const double* x, double* y) {
  if (!h || !x || !y) {
    set_error("null argument");
    return A2LS_ERR_ARG;
  }
  return guarded([&]() -> int {
    spmv(h, x, y, nullptr, h->st);
    return A2LS_OK;
  });
}

int a2ls_query(a2ls_handle* h, int32_t what, void* out, int64_t capacity, int64_t* needed) {
  if (!h) {
    set_error("null handle");
    return A2LS_ERR_ARG;
  }
  return guarded([&]() -> int {
    A2LS_CUDA(cudaStreamSynchronize(h->st));
    const int N = h->N;
    std::vector<unsigned char> buf;
    auto put = [&](const void* p, size_t bytes) {
      const size_t o = buf.size();
      buf.resize(o + bytes);
      if (bytes) std::memcpy(buf.data() + o, p, bytes);
    };
    auto put_dev = [&](const void* p, size_t bytes) {
      const size_t o = buf.size();
      buf.resize(o + bytes);
      if (bytes) A2LS_CUDA(cudaMemcpy(buf.data() + o, p, bytes, cudaMemcpyDeviceToHost));
    };
    switch (what) {
      case A2LS_Q_SIZES: {
        int64_t s[8] = {h->n, N, h->n0, h->sum_n, h->max_n, h->h_woff.empty() ? 0 : h->h_woff[N],
                        h->opt.precision, h->opt.variant};
        put(s, sizeof(s));
        break;
      }
      case A2LS_Q_SUBDOMAINS:
        put(h->h_off.data(), sizeof(int) * (N + 1));
        put(h->h_nI.data(), sizeof(int) * N);
        put_dev(h->d_idx, sizeof(int) * h->sum_n);
        break;
      case A2LS_Q_LUMP:
        put_dev(h->d_lump, sizeof(double) * h->sum_n);
        break;
      case A2LS_Q_FACTORS: {
        const size_t es = h->opt.precision == A2LS_FP64 ? 8 : (h->opt.precision == A2LS_BF16 ? 2 : 4);
        put_dev(h->d_fac, es * (size_t)h->h_ffoff[N]);
        put(h->h_ffoff.data(), sizeof(int64_t) * (N + 1));
        put(h->h_fld.data(), sizeof(int) * N);
        break;
      }
      case A2LS_Q_COARSE: {
        std::vector<int> m = h->h_m;
        m.resize(N, 0);
        put(m.data(), sizeof(int) * N);
        if (h->d_W && !h->h_woff.empty()) put_dev(h->d_W, sizeof(double) * h->h_woff[N]);
        break;
      }
      case A2LS_Q_EIGVALS:
        put(h->h_eigvals.data(), sizeof(double) * h->h_eigvals.size());
        break;
      case A2LS_Q_TIMES:
        put(h->times, sizeof(h->times));
        break;
      case A2LS_Q_EINV:
        if (h->d_Einv) put_dev(h->d_Einv, sizeof(double) * (size_t)h->n0 * h->n0);
        break;
      case A2LS_Q_EIGSTATS:
        put(h->h_eigstats.data(), sizeof(int) * h->h_eigstats.size());
        break;
      case A2LS_Q_LAUNCHES:
        put(&h->launches, sizeof(int64_t));
        break;
      case A2LS_Q_TUNING: {
        const int32_t v[2] = {h->ls_width, (int32_t)h->graphs.size()};
        put(v, sizeof(v));
        break;
      }
      case A2LS_Q_ENVELOPE:
        put(h->h_env.data(), sizeof(double) * h->h_env.size());
        break;
      case A2LS_Q_EIG_UNCONVERGED: {
        const int32_t v[2] = {h->eig_unconverged, h->eig_stalled};
        put(v, sizeof(v));
        break;
      }
      case A2LS_Q_EIGRES:
        put(h->h_eigres.data(), sizeof(double) * h->h_eigres.size());
        break;
      case A2LS_Q_PIVOT_BOOSTS: {
        const int32_t v = h->pivot_boosts;
        put(&v, sizeof(v));
        break;
      }
      case A2LS_Q_KERNEL_TIMES: {
        collect_kernel_times(h);
        for (int k = 0; k < KT_COUNT; ++k) {
          const double v[3] = {(double)h->kt_count[k], h->kt_ms[k], h->kt_work[k]};
          put(v, sizeof(v));
        }
        break;
      }
      default:
        fail(A2LS_ERR_ARG, "unknown query item %d", what);
    }
    if (needed) *needed = (int64_t)buf.size();
    if (out) {
      if (capacity < (int64_t)buf.size()) fail(A2LS_ERR_ARG, "query buffer too small (%lld < %zu)", (long long)capacity, buf.size());
      std::memcpy(out, buf.data(), buf.size());
    }
    return A2LS_OK;
  });
}

int a2ls_set_coarse_basis(a2ls_handle* h, const int32_t* m, const double* W) {
  if (!h || !m) {
    set_error("null argument");
    return A2LS_ERR_ARG;
  }
  return guarded([&]() -> int {
    std::vector<int> mv(m, m + h->N);
    upload_coarse_layout(h, mv);
    if (h->h_woff[h->N] > 0) {
      if (!W) fail(A2LS_ERR_ARG, "null W");
      A2LS_CUDA(cudaMemcpyAsync(h->d_W, W, sizeof(double) * h->h_woff[h->N], cudaMemcpyHostToDevice, h->st));
    }
    build_coarse_operator(h);
    sync_and_check(h, "coarse operator");
    return A2LS_OK;
  });
}

}  // extern "C"

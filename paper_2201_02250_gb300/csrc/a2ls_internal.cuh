// Internal declarations shared by the a2ls CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/a2ls.h"
#include "dfloat.cuh"

namespace a2ls {

// ---------------------------------------------------------------------------
// Errors: internal code throws, the C ABI converts to a status + message.
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] void fail(int code, const char* fmt, ...);
// host-side k-way partition of the graph of A + A^T (partition.cu); errors through fail()
void partition_graph(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t nparts, uint64_t seed,
                     int32_t* part);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
#define A2LS_CUDA(x) ::a2ls::check_cuda((x), #x, __FILE__, __LINE__)
// every kernel launch of the library goes through this macro: error check and per-handle count
#define A2LS_LAUNCH() ::a2ls::launched(h, cudaGetLastError(), __FILE__, __LINE__)

// Device-side status words written by kernels (never trap): [0] first error
// code, [1] the subdomain or row that raised it, [2] auxiliary information.
// [3] counts the local LU pivots replaced under static pivoting.
enum { ST_CODE = 0, ST_WHERE = 1, ST_AUX = 2, ST_BOOSTS = 3, ST_WORDS = 8 };

__device__ __forceinline__ void raise_status(int* st, int code, int where, int aux) {
  if (atomicCAS(st + ST_CODE, 0, code) == 0) {
    st[ST_WHERE] = where;
    st[ST_AUX] = aux;
  }
}

// Kernels whose launches can be timed with CUDA events (a2ls_options::timing).
enum { KT_LU_LOCAL = 0, KT_LU_SPLIT, KT_EIG_SOLVE, KT_EIG_ORTH, KT_EIG_RR, KT_COARSE_LU, KT_COARSE_INV,
       KT_APPLY_LOCAL, KT_COUNT };

// Tile size of the block-inverted LU format used by all triangular solves.
constexpr int TB = 64;
// Largest number of coarse columns per subdomain.
constexpr int MAXM = 64;
// Largest subdomain size handled by the dense kernels (vector held in shared memory).
constexpr int MAXN_LOCAL = 8192;

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// The handle: every device array the preconditioner owns.
// ---------------------------------------------------------------------------
struct Phase { enum { SETUP_GRAPH, SETUP_EXTRACT, SETUP_LU, SETUP_EIG, SETUP_COARSE, SETUP_TOTAL,
                      SOLVE_TOTAL, SOLVE_APPLY, SETUP_APPLY_PREP, COUNT }; };

// the apply's local factors repacked as one stream in solve order (k_stream.cu)
struct StreamSolve {
  bool ready = false;
  int elem_bytes = 0, nchunks = 0, xcap = 0;
  int64_t stream_elems = 0;
  void* d_stream = nullptr;
  int4* d_meta = nullptr;                    // chunk headers
  int* d_choff = nullptr;                    // chunks of each subdomain
  int* d_order = nullptr;                    // work-queue order of the subdomains (by decreasing cost)
  int64_t* d_soff = nullptr;
  // launch shapes: [0] 8 consumer warps, one CTA per SM; [1] 4 consumer warps, two CTAs per SM; [2] 8
  // consumer warps, two CTAs per SM
  struct Shape {
    bool ready = false;
    int ncta = 0, nstages = 0;
    size_t smem = 0;
  } shape[3];
};
constexpr int LS_STREAM = 3000;   // local-solve configurations of the streaming kernel: shape 0
constexpr int LS_STREAM2 = 3004;  // ... shape 1
constexpr int LS_STREAM3 = 3008;  // ... shape 2

}  // namespace a2ls

struct a2ls_handle {
  // problem
  int n = 0, nnz = 0, N = 0, delta = 0, nev = 0;
  a2ls_options opt{};
  cudaStream_t st = nullptr;
  std::vector<void*> allocs;     // device allocations owned by the handle
  cudaMemPool_t pool = nullptr;  // the library's memory pool of the handle's device (null: default pool)
  int* d_status = nullptr;       // ST_WORDS ints

  // FP64 copy of A and of the partition
  int *rowptr = nullptr, *colind = nullptr;
  double* val = nullptr;
  int* part = nullptr;

  // subdomains: local order = [Omega_I ascending, Omega_Gamma layer by layer, ascending in a layer]
  std::vector<int> h_off, h_nI, h_n, h_ld;   // h_off has N+1 entries
  std::vector<int64_t> h_foff;               // offsets of dense local matrices (elements), N+1
  int *d_off = nullptr, *d_nI = nullptr, *d_ni = nullptr, *d_ld = nullptr;
  int64_t* d_foff = nullptr;
  int* d_idx = nullptr;                      // sum n_i: local -> global
  int* d_ipos = nullptr;                     // n: local index of a node inside its own part
  int* d_gstart = nullptr;                   // N x (delta + 2): local start of the interior, each
                                             // overlap layer, and n_i
  int* d_sched = nullptr;                    // N: subdomains by decreasing size (work order)
  int* d_counter = nullptr;                  // work-queue counter of the persistent kernels
  int ls_width = 0;                          // configuration of the local solves (autotuned)
  a2ls::StreamSolve ss;                      // packed factors of the streaming local solves
  int sum_n = 0, max_n = 0;
  int max_rownnz = 0, max_memb = 0;          // largest row of A, largest membership count
  // node -> memberships (flat local positions off_i + l), sorted by subdomain
  int *d_mrow = nullptr, *d_mpos = nullptr, *d_msub = nullptr;
  double* d_D = nullptr;                     // sum n_i partition-of-unity weights
  double* d_lump = nullptr;                  // sum n_i: s_i on overlap rows, 0 elsewhere
  // local CSR of A restricted to Omega_i (local column or -1 if outside), one row per local row
  int64_t* d_lrow = nullptr;                 // sum n_i + 1
  int* d_lcol = nullptr;
  double* d_lval = nullptr;
  // envelope of the local pattern: first column of each row, first row of each column (local
  // indices, sum n_i each), and their minima per 64-row / 64-column tile (offsets h_toff)
  int *d_pf = nullptr, *d_pg = nullptr;
  std::vector<int> h_toff;
  int *d_toff = nullptr, *d_tf = nullptr, *d_tg = nullptr;
  // per subdomain: envelope LU flops (all pivots, overlap pivots), L and U envelope entries
  std::vector<double> h_env;

  // local factors (block-inverted LU, precision = opt.precision)
  void* d_fac = nullptr;
  size_t fac_elems = 0;
  // layout of d_fac: the factorisation's (ld_i = n_i rounded to 4, offsets h_foff), except for the
  // bfloat16 storage, whose rows start on 16-byte boundaries (ld_i rounded to 8)
  std::vector<int> h_fld;
  std::vector<int64_t> h_ffoff;
  int* d_fld = nullptr;
  int64_t* d_ffoff = nullptr;

  // coarse space
  int n0 = 0;
  int coarse_band = 0;                       // bandwidth of A_00 in its block order
  std::vector<int> h_m, h_coff;              // N, N+1 (coff in the banded block order)
  std::vector<int64_t> h_woff;               // N+1, offsets of W_i (n_i x m_i)
  int *d_m = nullptr, *d_coff = nullptr;
  int64_t* d_woff = nullptr;
  double* d_W = nullptr;
  double* d_Einv = nullptr;                  // n0 x n0 row-major
  std::vector<double> h_eigvals;             // 2*N*(nevmax)
  // eigenvectors selected by the setup, Z_i = [k | V Y] (n_i x zld row-major per subdomain, FP64),
  // kept as training targets of the warm-start network
  double* d_zev = nullptr;
  int64_t* d_zoff = nullptr;                 // N+1
  int zld = 0;
  std::vector<int> h_zcols;                  // N: columns of Z_i in use
  std::vector<int> h_eigstats;               // 2*N
  int eig_unconverged = 0;                   // subdomains whose eigensolve stopped short of eig_tol
  int eig_stalled = 0;                       // ... of them stopped by the stagnation stop
  int pivot_boosts = 0;                      // local LU pivots replaced (static pivoting)
  std::vector<double> h_eigres;              // N: worst relative Ritz residual at the last cycle

  // apply workspace
  double *d_g = nullptr, *d_c = nullptr, *d_q = nullptr, *d_t = nullptr, *d_yloc = nullptr;
  double* d_red = nullptr;                   // reduction scratch

  // GMRES workspace
  int gm_restart = 0;
  double *d_V = nullptr, *d_Z = nullptr, *d_w = nullptr, *d_h = nullptr, *d_part = nullptr;
  double* h_pinned = nullptr;                // pinned host scratch for small readbacks

  double times[16] = {0};
  int64_t launches = 0;                      // kernels launched by this handle
  // CUDA graphs of the apply, one per (input, output) pair used by GMRES
  struct ApplyGraph { const double* r; double* z; cudaGraphExec_t exec; };
  std::vector<ApplyGraph> graphs;
  cudaStream_t cap_st = nullptr;
  // optional per-kernel event timing: pairs of events per tracked kernel
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> kt_events[a2ls::KT_COUNT];
  std::vector<cudaEvent_t> kt_pool;
  double kt_ms[a2ls::KT_COUNT] = {0};
  double kt_work[a2ls::KT_COUNT] = {0};      // algorithmic flops (bytes for the apply local solves)
  int64_t kt_count[a2ls::KT_COUNT] = {0};
};

namespace a2ls {

void launched(a2ls_handle* h, cudaError_t e, const char* file, int line);

// RAII event pair around the launches of one tracked kernel (no-op unless timing is on)
struct KTime {
  a2ls_handle* h;
  int id;
  cudaEvent_t b = nullptr;
  KTime(a2ls_handle* hh, int kid, double work = 0.0);
  ~KTime();
};
void collect_kernel_times(a2ls_handle* h);

// allocation helpers (stream-ordered, owned by the handle)
void* dalloc_bytes(a2ls_handle* h, size_t bytes);
template <class T> T* dalloc(a2ls_handle* h, size_t count) {
  return static_cast<T*>(dalloc_bytes(h, count * sizeof(T) + (count == 0 ? 16 : 0)));
}
void dfree(a2ls_handle* h, void* p);
void sync_and_check(a2ls_handle* h, const char* phase);

// ---------------------------------------------------------------------------
// Launchers implemented in the .cu files.
// ---------------------------------------------------------------------------
// k_graph.cu
void build_subdomains(a2ls_handle* h);                 // validation, overlap, lists, memberships
void extract_local(a2ls_handle* h, void* dense_A, void* dense_At, double* dense_scale);
void exclusive_scan_i64(const int64_t* in, int64_t* out, int n, cudaStream_t st, a2ls_handle* h);

// k_dense.cu
template <class T> void lu_batched(a2ls_handle* h, T* fac, int allow_last_zero, double* last_pivot,
                                   double* diag_scale, int phase = -1);
template <class TS, class TD> void schur_copy(a2ls_handle* h, const TS* src, TD* dst, const double* last_pivot);
template <class T> void invert_diag_tiles(a2ls_handle* h, T* fac);
// y_loc / z output of the RAS/ASM local solves; see k_dense.cu for the modes
template <class T> void local_solves(a2ls_handle* h, const T* fac, const double* t, const double* q,
                                     double* z, int mode);
template <class T> void autotune_local_solves(a2ls_handle* h, const T* fac, const double* t, double* scratch,
                                              int mode);
int autotune_lookup(const char* key);            // 0 if unknown
void autotune_store(const char* key, int value);
void dense_inverse(a2ls_handle* h, double* E, int n, double scale, double* Einv, int band);
// skip_p_le > 0: subdomains with at most that many columns are left to another kernel
template <class T> void block_solve(a2ls_handle* h, const T* fac, T* X, const int64_t* xoff, int col0, int ldx,
                                    const int* pvec, int pmax, const int* active, int forward, int backward,
                                    int skip_p_le = 0);

// k_tcsolve.cu: double-float block triangular solves of the eigensolver on the tensor cores
struct TcSolve {
  bool ready = false;
  int64_t ntiles = 0;
  int64_t *d_ftoff = nullptr, *d_ftab = nullptr, *d_xdoff = nullptr;
  unsigned char *d_fdig = nullptr, *d_xdig = nullptr;
};
void tc_solve_prepare(a2ls_handle* h, const dfloat* fac, TcSolve& ts);   // digits of the factor tiles
void tc_solve_release(a2ls_handle* h, TcSolve& ts);
// one sweep over the subdomains with 1 <= p <= 32 columns (forward: inv(L), else inv(U))
void tc_block_solve(a2ls_handle* h, const TcSolve& ts, dfloat* X, const int64_t* xoff, int col0, int ldx,
                    const int* pvec, const int* active, int forward, unsigned char* xdig = nullptr);
constexpr int TC_SOLVE_MAX_P = 32;

// k_stream.cu: pack the factors (after the diagonal tiles are inverted) into the stream of the
// streaming local solves, and those solves (FP32 or BF16 factors)
template <class T> void stream_prepare(a2ls_handle* h, const T* fac);
template <class T> void launch_local_solve_stream(a2ls_handle* h, int config, const double* t, const double* q,
                                                  double* z, int mode);

// k_dense.cu: FP32 local factors rounded to the bfloat16 storage of A2LS_BF16, in the layout
// h_fld / h_ffoff (which this call sets up); returns the new storage
__nv_bfloat16* factors_to_bf16(a2ls_handle* h, const float* src);
// the apply's local solves with the handle's factor type
void local_solves_any(a2ls_handle* h, const double* t, const double* q, double* z, int mode);

// k_static.cu: loads the module of a2ls_apply_static's static scratch on the current device
void prime_static_scratch();

// k_gnn.cu: the warm-start network's proposal, Y = sum n_i x 16 FP32 on the handle's stream
void gnn_infer(a2ls_handle* h, const a2ls_gnn* model, float* Y);

// k_eig.cu
void eigensolve(a2ls_handle* h, void* fac_tilde, const double* last_pivot, const double* diag_scale);

// k_coarse.cu
void orthonormalize_and_set_W(a2ls_handle* h, double* Z, const int* mcols, int ldz_max);
void upload_coarse_layout(a2ls_handle* h, const std::vector<int>& m);
void build_coarse_operator(a2ls_handle* h);

// k_krylov.cu
void spmv(a2ls_handle* h, const double* x, double* y, const double* b_minus, cudaStream_t st);
void apply_preconditioner(a2ls_handle* h, const double* r, double* z);
void apply_preconditioner_graph(a2ls_handle* h, const double* r, double* z);
double dot(a2ls_handle* h, const double* x, const double* y);
double nrm2(a2ls_handle* h, const double* x);
int gmres(a2ls_handle* h, const double* b, double* x, double rtol, int* iters, double* relres);

}  // namespace a2ls

/*
 * a2ls.h -- C ABI of the GB300 algebraic two-level Schwarz library (libA2LS.so).
 *
 * The library builds and applies the fully algebraic two-level overlapping
 * Schwarz preconditioner of Al Daas, Jolivet and Rees (arXiv 2201.02250) and
 * solves A x = b with it inside restarted GMRES, entirely on one GPU.
 *
 *   setup  : overlap grown from the adjacency graph of A (Section 2), local
 *            matrices A_ii and block splittings A~_ii (Definition 3.1), batched
 *            dense LU of the local matrices, the local generalized eigenproblems
 *            of Eq. 3.1 with the selection of Eq. 3.2, the coarse operator
 *            A_00 = R_0 A R_0^H and its exact LU (Section 4).
 *   apply  : the restricted two-level preconditioner with deflated coarse
 *            correction, Eq. 2.4 (default), or the variants of Section 2.
 *   solve  : right-preconditioned GMRES(restart) with zero-free initial guess
 *            (Section 4); flexible GMRES when the local solves run in FP32.
 *
 * Conventions shared by every entry point:
 *   - Pointers documented as "device" must point to memory of the current CUDA
 *     device; "host" pointers to ordinary host memory.  The caller owns every
 *     buffer it passes; the library copies what it keeps.
 *   - All work is issued on the stream given in a2ls_options::stream (NULL =
 *     the legacy default stream).  Entry points that return results to the
 *     host synchronise that stream; a2ls_apply does not.
 *   - Every function returns an a2ls_status; nothing aborts or traps.  On
 *     failure a human-readable message is available from a2ls_last_error()
 *     (thread-local, valid until the next call on the same thread).
 *   - Indices are 0-based int32; n and nnz must fit in int32.  Only real
 *     (double) matrices are supported.
 */
#ifndef A2LS_H
#define A2LS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  A2LS_OK = 0,
  A2LS_ERR_ARG = 1,           /* invalid argument (sizes, CSR structure, partition) */
  A2LS_ERR_SINGULAR = 2,      /* zero or tiny pivot in a local or coarse LU (the paper's failure mark) */
  A2LS_ERR_NOT_CONVERGED = 3, /* max_it reached; x holds the last iterate */
  A2LS_ERR_EIGEN = 4,         /* local eigenproblem outside what the solver supports or not converged */
  A2LS_ERR_TIMEOUT = 5,       /* a bounded device-side wait expired */
  A2LS_ERR_CUDA = 6,          /* a CUDA runtime error */
  A2LS_ERR_OOM = 7,           /* device allocation failed */
  A2LS_ERR_STATE = 8          /* call not valid in the handle's current state */
} a2ls_status;

/* Precision of the local factors of A_ii and of the local solves of the apply
 * (a2ls_options::precision), and of the factorisation of A~_ii and the local
 * eigensolves (a2ls_options::eig_precision).  The SpMV, the GMRES
 * orthogonalisation, the residual and the coarse operator and its factorisation
 * are always FP64; the small Rayleigh-Ritz problems run in FP64, or in
 * double-float with a double-float eigensolve; the mixed form (precision FP32)
 * forms the explicit inverse of the coarse operator from its FP64 factors in
 * double-float.
 * A2LS_FP32X2 (eigensolve only) is double-float arithmetic: each value is an unevaluated sum
 * of two FP32 numbers (48-bit significand, FP32 exponent range), computed on the FP32 pipe.
 * A2LS_BF16 (local factors only) factors A_ii in FP32 as A2LS_FP32 does and stores the factors in
 * bfloat16 (8-bit significand, half the bytes of the apply's dominant stream); the local solves read
 * them and accumulate in FP32, and flexible GMRES absorbs the rounding of the stored factors. */
enum { A2LS_FP64 = 0, A2LS_FP32 = 1, A2LS_FP32X2 = 2, A2LS_BF16 = 3 };

/* Preconditioner variants (Section 2).  DEFLATED_RAS is Eq. 2.4, the one the
 * paper uses in all experiments. */
enum {
  A2LS_DEFLATED_RAS = 0, /* R0^H A00^-1 R0 + M_RAS^-1 (I - A R0^H A00^-1 R0)  (Eq. 2.4) */
  A2LS_DEFLATED_ASM = 1, /* same with M_ASM^-1 */
  A2LS_ADDITIVE_RAS = 2, /* R0^H A00^-1 R0 + M_RAS^-1 */
  A2LS_ADDITIVE_ASM = 3, /* R0^H A00^-1 R0 + M_ASM^-1                          (Eq. 2.2) */
  A2LS_ONE_LEVEL_RAS = 4,/* M_RAS^-1                                           (Eq. 2.3) */
  A2LS_ONE_LEVEL_ASM = 5 /* M_ASM^-1                                           (Eq. 2.1) */
};

/* Partition of unity D_i (Section 2): BOOLEAN puts 1 on the interior nodes
 * Omega_Ii and 0 on the overlap Omega_Gamma_i; MULTIPLICITY puts 1/k(j) on
 * every node j of Omega_i, k(j) = number of subdomains containing j. */
enum { A2LS_POU_BOOLEAN = 0, A2LS_POU_MULTIPLICITY = 1 };

typedef struct a2ls_handle a2ls_handle;

/* Learned warm start of the local eigensolves (not part of the paper): a message-passing network
 * over each subdomain's local graph, see the a2ls_gnn_* entry points at the end of this header. */
typedef struct a2ls_gnn a2ls_gnn;
typedef struct a2ls_gnn_sample a2ls_gnn_sample;

/* Sparse matrix in CSR form.  All arrays are device pointers owned by the
 * caller and only read during a2ls_setup (the library keeps its own copy).
 * rowptr: n+1 entries, rowptr[0] = 0, non-decreasing, rowptr[n] = nnz.
 * colind: nnz entries in [0, n).  val: nnz doubles. */
typedef struct {
  int32_t n;
  int32_t nnz;
  const int32_t* rowptr;
  const int32_t* colind;
  const double* val;
} a2ls_csr;

typedef struct {
  int32_t precision;        /* A2LS_FP64 (default), A2LS_FP32 or A2LS_BF16 */
  int32_t variant;          /* A2LS_DEFLATED_RAS (default) ... */
  int32_t pou;              /* A2LS_POU_BOOLEAN (default) or A2LS_POU_MULTIPLICITY */
  int32_t restart;          /* GMRES restart length, default 30 (Section 4) */
  int32_t max_it;           /* total inner iterations, default 1000 */
  int32_t flexible;         /* -1: automatic (FGMRES iff precision != FP64), 0: GMRES, 1: FGMRES */
  double tau;               /* <= 0: keep nev eigenpairs per subdomain; > 0: keep |lambda| > 1/tau,
                               at most nev (Eq. 3.2) */
  int32_t eig_block_steps;  /* block Krylov steps per eigen restart cycle, default 3 */
  int32_t eig_max_cycles;   /* eigen restart cycles, default 60 */
  double eig_tol;           /* relative eigen-residual target; 0 = default: 1e-10 when precision is FP64,
                               1e-4 otherwise (a preconditioner's coarse space needs no more) */
  uint64_t seed;            /* seed of the eigensolver's random start blocks */
  void* stream;             /* cudaStream_t for all work; NULL = legacy default stream */
  int32_t timing;           /* 1: record CUDA events around the tracked kernels (A2LS_Q_KERNEL_TIMES) */
  int32_t eig_precision;    /* precision of the factorisation of A~_ii and of the local eigensolves:
                               -1 (default) = FP64 when precision is FP64, else A2LS_FP32X2;
                               A2LS_FP64; A2LS_FP32X2; A2LS_FP32 (only for local splittings whose
                               conditioning FP32 can resolve; high-contrast problems need 48 bits) */
  int32_t graphs;           /* 1 (default): GMRES replays the apply as CUDA graphs captured on first use */
  const a2ls_gnn* warm_start; /* NULL (default): random start blocks for the local eigensolves; otherwise
                                 the network's proposal (a2ls_gnn_forward) starts each subdomain's block
                                 Krylov iteration.  The network is only read; it must outlive a2ls_setup. */
  int32_t eig_strict;       /* 0 (default): a local eigensolve that misses eig_tol after eig_max_cycles keeps
                               the Ritz vectors it reached (still a valid coarse space, possibly a weaker
                               one; counted by A2LS_Q_EIG_UNCONVERGED); 1: a2ls_setup fails with
                               A2LS_ERR_EIGEN instead */
  int32_t eig_stall_cycles; /* stagnation stop of the local eigensolves, default 8: a subdomain whose
                               largest relative residual of the wanted Ritz pairs has not halved over
                               this many cycles stops with the Ritz vectors it has (counted as
                               unconverged, and as stagnated by A2LS_Q_EIG_UNCONVERGED); 0 = off */
  int32_t tensor_cores;     /* 1 (default): the trailing updates of the double-float LU run on the tensor
                               cores (BF16 digit products accumulated exactly in FP32, to double-float
                               accuracy); 0: on the FP32 pipe */
  int32_t eig_thick_restart; /* 1 (default): a restart of the local eigensolves keeps the block of Ritz
                               vectors together with its image under the operator, so that a restarted
                               cycle spans the same block Krylov space with one block application fewer;
                               0: explicit restart from the Ritz vectors alone */
  int32_t local_solve_kernel; /* 0 (default): the apply's local-solve kernel is picked by timing the
                               candidates on the handle's own factors; otherwise that candidate:
                               256, 512, 1024 (one-pass kernel, CTA width), 1256, 1512, 2256
                               (pipelined kernel), 3000 / 3004 / 3008 (streaming kernel on the
                               repacked factors: one CTA of 8 consumer warps, two of 4, two of 8 per
                               SM; FP32 and BF16 factors only) */
  int32_t eig_block_size;   /* columns of the local eigensolves' blocks: 0 (default) = the larger of
                               nev + max(4, nev / 2) and min(2 nev, 24), at most 32; otherwise that many
                               (at least nev + 1, at most 32) */
  int32_t static_pivoting;  /* 0 (default): a pivot of a local LU (A_ii or the splitting A~_ii) at most
                               1e-14 (FP64, double-float) or 1e-12 (FP32) times the subdomain's largest
                               diagonal entry makes a2ls_setup fail with SINGULAR; 1: it is replaced by
                               that largest entry and the factorisation goes on (static pivoting: the
                               factors are those of A_ii plus a diagonal perturbation, which the outer
                               (F)GMRES corrects; for matrices that are not diagonally dominant, whose
                               unpivoted LU can meet a zero pivot).  Replacements are counted by
                               A2LS_Q_PIVOT_BOOSTS.  The coarse LU keeps its SINGULAR check. */
} a2ls_options;

/* Fills *opt with the defaults listed above.  Never fails. */
void a2ls_default_options(a2ls_options* opt);

/*
 * a2ls_setup -- build the preconditioner for A.
 *   A         : CSR matrix (device arrays, see a2ls_csr).
 *   partition : device, n int32 values in [0, N); every part non-empty.  This is
 *               the non-overlapping partition Omega_Ii of Section 2 (the paper
 *               obtains it from ParMETIS; here it is an input, which
 *               a2ls_partition can compute on the host).
 *   overlap   : number of adjacency layers delta >= 0 added around each part
 *               (Section 2 defines one layer; delta layers repeat it).
 *   nev       : eigenpairs kept per subdomain (Eq. 3.2; with tau > 0 an upper bound).
 *   opt       : options, or NULL for the defaults.
 *   out       : receives the new handle on success, NULL on failure.
 * Synchronises opt->stream.  Errors: ARG (bad sizes/CSR/partition), SINGULAR
 * (tiny pivot in a local or the coarse LU), EIGEN, CUDA, OOM.
 */
int a2ls_setup(const a2ls_csr* A, const int32_t* partition, int32_t overlap, int32_t nev,
               const a2ls_options* opt, a2ls_handle** out);

/*
 * a2ls_apply -- z = M^{-1} r for the handle's variant (Eq. 2.4 by default).
 *   r, z : device, n doubles each; they must not alias.
 * Asynchronous on the handle's stream (no host synchronisation).
 */
int a2ls_apply(a2ls_handle* h, const double* r, double* z);

/*
 * a2ls_solve -- right-preconditioned restarted (F)GMRES for A x = b (Section 4).
 *   b      : device, n doubles.
 *   x      : device, n doubles; on entry the initial guess (the paper uses 0),
 *            on exit the last iterate.
 *   rtol   : relative tolerance on the true residual ||b - A x|| / ||b||.
 *   iters  : host, receives the number of inner iterations (may be NULL).
 *   relres : host, receives the final true relative residual (may be NULL).
 * Returns OK or NOT_CONVERGED (x still valid); synchronises the stream.
 */
int a2ls_solve(a2ls_handle* h, const double* b, double* x, double rtol, int32_t* iters,
               double* relres);

/* Releases every device resource of the handle.  NULL is ignored. */
void a2ls_destroy(a2ls_handle* h);

/* Message describing the last failure on this thread ("" if none). */
const char* a2ls_last_error(void);

/*
 * a2ls_trim_memory -- memory management of the implementation (the paper has no counterpart).
 * Handles take their device memory from one stream-ordered memory pool per device, owned by the
 * library, that keeps the blocks a destroyed handle frees for the next setup: repeated setups of
 * similar size then neither map nor unmap device memory.  This call returns the pools' unused
 * blocks to the system (memory of live handles stays).  Call it after destroying handles when other
 * code needs the memory.  Thread-safe; returns OK, or ERR_CUDA if the runtime reports an error.
 */
int a2ls_trim_memory(void);

/*
 * a2ls_partition -- the non-overlapping partition Omega_Ii that a2ls_setup takes (Section 2).  The
 * paper partitions the graph of A^T + A with ParMETIS (Section 4); this is the library's own
 * partitioner of the same graph: multilevel recursive bisection (heavy-edge matching, growing from
 * several starts on the coarsest graph, Fiduccia-Mattheyses refinement on every level).  It runs on
 * the host and needs no GPU.
 *   n, rowptr, colind : HOST CSR pattern of A (n + 1 and rowptr[n] int32 entries; the values are not
 *                       needed).  The graph is the off-diagonal pattern of A + A^T, unit weights.
 *   nparts            : number of parts N, 1 <= N <= n.
 *   seed              : seeds the coarsening's visiting order (the result is a pure function of the
 *                       pattern, nparts and seed).
 *   part              : HOST, n int32 values written in [0, N); every part is non-empty.  Each
 *                       bisection keeps its sides within 2 % of an average final part of their target
 *                       weights, so parts hold n / N vertices to within a few per cent.  Parts of a
 *                       connected graph are connected: a part left in several pieces keeps the
 *                       largest, the others join the neighbouring part they share most edges with
 *                       (connectivity before balance; a subdomain in several floating pieces would
 *                       give its splitting a kernel of dimension above one).  The halves of the top
 *                       recursion levels run on up to 16 host threads; the result does not depend on
 *                       their scheduling.
 * Copy part to the device for a2ls_setup.  Errors: ARG (n < 1, nparts outside [1, n], NULL pointers,
 * rowptr not starting at 0 or decreasing, column index outside [0, n)), OOM (host memory); the
 * caller's buffers are only read, except part.
 */
int a2ls_partition(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t nparts, uint64_t seed,
                   int32_t* part);

/* Items for a2ls_query.  All results are copied to host memory. */
enum {
  A2LS_Q_SIZES = 0,      /* int64[8]: n, N, n0, sum n_i, max n_i, sum m_i rows stored, precision, variant */
  A2LS_Q_SUBDOMAINS = 1, /* int32[(N+1) + N + sum n_i]: offsets, n_I per subdomain, local->global
                            indices (each subdomain: Omega_Ii ascending, then Omega_Gamma_i layer by
                            layer: the nodes of the first overlap step ascending, then the second's, ...) */
  A2LS_Q_LUMP = 2,       /* double[sum n_i]: s_i of Definition 3.1 on overlap rows, 0 on interior rows */
  A2LS_Q_FACTORS = 3,    /* (precision type: double, float or bfloat16)[sum over i of n_i*ld_i] then int64[N+1] offsets and
                            int32[N] ld: LU of A_ii without pivoting, row-major, unit-lower L below
                            the diagonal; each 64x64 diagonal tile holds inv(L_bb) strictly below
                            its diagonal and inv(U_bb) on and above it */
  A2LS_Q_COARSE = 4,     /* int32[N] m_i, then double[sum n_i*m_i]: W_i = orth(D_i Z_i), n_i x m_i
                            row-major per subdomain in the local order of A2LS_Q_SUBDOMAINS */
  A2LS_Q_EIGVALS = 5,    /* double[2*N*nev_max]: per subdomain the kept eigenvalues (re, im),
                            kernel part first as (+inf, 0), unused slots NaN; nev_max = max(nev,1)+1 */
  A2LS_Q_TIMES = 6,      /* double[16]: per-phase milliseconds of the last setup and solve */
  A2LS_Q_EINV = 7,       /* double[n0*n0]: the inverse of A_00 used by the apply, row-major */
  A2LS_Q_EIGSTATS = 8,   /* int32[2*N]: eigen cycles run and kernel dimension per subdomain */
  A2LS_Q_LAUNCHES = 9,   /* int64[1]: kernels this handle has launched so far */
  A2LS_Q_TUNING = 11,    /* int32[2]: CTA width chosen for the local solves, CUDA graphs held */
  A2LS_Q_EIG_UNCONVERGED = 12, /* int32[2]: subdomains whose eigensolve stopped short of eig_tol, and how
                                  many of them by the stagnation stop (the others ran eig_max_cycles) */
  A2LS_Q_PIVOT_BOOSTS = 15, /* int32[1]: local LU pivots replaced under a2ls_options::static_pivoting */
  A2LS_Q_EIGRES = 14,    /* double[N]: per subdomain the largest residual ||T u - lambda u|| / |lambda| of
                            the wanted Ritz pairs at its last eigen cycle (0 without a Krylov part) */
  A2LS_Q_ENVELOPE = 13,  /* double[4*N]: per subdomain the flops of an LU confined to the envelope of the
                            local pattern (all pivots; overlap pivots only), and the entries of L's row
                            envelope and U's column envelope (sum_r r - f_r + 1, sum_c c - g_c + 1), f_r / g_c
                            being the first nonzero column of row r / row of column c; the factors are
                            zero outside these envelopes and the kernels skip the 64x64 tiles there */
  A2LS_Q_KERNEL_TIMES = 10 /* double[3*8]: (launches, total ms, algorithmic work) of the tracked kernels;
                              work is flops, or bytes moved for the apply local solves; in the order
                              local LU, splitting LU, eigen triangular solves, eigen orthogonalisation,
                              Rayleigh-Ritz, coarse LU, coarse inverse, apply local solves;
                              populated only with a2ls_options::timing = 1 */
};

/*
 * a2ls_solve_multi -- solve A X = B for nrhs right-hand sides with the same preconditioner.
 *   B, X     : device, n x nrhs doubles, column k at offset k*n (X holds the initial guesses on input).
 *   iters    : host, nrhs int32 (may be NULL); relres: host, nrhs doubles (may be NULL).
 * Each column runs its own (F)GMRES as a2ls_solve does, one after another on the handle's stream,
 * sharing the setup.  Returns OK when every column converged, NOT_CONVERGED if any did not (its X
 * column holds the last iterate), or the first other error.
 */
int a2ls_solve_multi(a2ls_handle* h, int32_t nrhs, const double* B, double* X, double rtol, int32_t* iters,
                     double* relres);

/*
 * a2ls_setup_batch -- set up nsys independent systems with one call.
 *   A[k], partition[k], overlap[k], nev[k] : as for a2ls_setup, per system; opt shared (may be NULL).
 *   out      : host array of nsys handles, filled on success (all NULL on failure; every handle
 *              created before the failing system is destroyed again).
 * The systems are set up one after another on the options' stream; each setup batches all of its
 * subdomains into single launches.  Each handle is used and destroyed on its own.
 */
int a2ls_setup_batch(int32_t nsys, const a2ls_csr* A, const int32_t* const* partition, const int32_t* overlap,
                     const int32_t* nev, const a2ls_options* opt, a2ls_handle** out);

/*
 * a2ls_query -- copy one internal quantity to host memory (inspection and tests).
 *   what     : an A2LS_Q_* item.
 *   out      : host buffer of at least `capacity` bytes, or NULL to only ask the size.
 *   needed   : host, receives the bytes the item needs (may be NULL).
 * Returns ARG if capacity is too small.  Synchronises the stream.
 */
int a2ls_query(a2ls_handle* h, int32_t what, void* out, int64_t capacity, int64_t* needed);

/*
 * a2ls_set_coarse_basis -- replace the coarse space by a given one.
 *   m : host, N int32, columns per subdomain.
 *   W : host, doubles, for each subdomain in order an n_i x m_i row-major block in
 *       the local order of A2LS_Q_SUBDOMAINS (rows on Omega_Gamma_i are used as given).
 * Rebuilds A_00 = R_0 A R_0^H with R_0^H = [R_1^T W_1 ... R_N^T W_N] and its inverse.
 * Used to compare the apply against another implementation with the same basis
 * (the apply is invariant to the choice of basis of the coarse space).
 */
int a2ls_set_coarse_basis(a2ls_handle* h, const int32_t* m, const double* W);

/*
 * a2ls_apply_static -- the same z = M^{-1} r as a2ls_apply, for callers that must not have device
 * memory allocated on their behalf: applications whose device memory is fully reserved by their
 * own pool allocator, or latency-critical loops in which an allocation (which may synchronise the
 * device) is not allowed.  The paper has no counterpart; this is an interface convenience.
 *   r, z : device, n doubles each, owned by the caller; they must not alias.
 * The call allocates nothing.  Its scratch vectors (2n + 2 n0 doubles, plus sum of the subdomain
 * sizes for the ASM variants or the multiplicity partition of unity) come from a fixed array of
 * 1,048,576 doubles (8 MiB) in the library's static device memory, which every GPU on which a
 * handle is set up holds until the process exits; larger problems get A2LS_ERR_ARG.  a2ls_setup loads the
 * array on its device (the one allocation it needs, made while setup allocates anyway); each call
 * then looks up the array's device address (cudaGetSymbolAddress) with the handle's device current,
 * which allocates nothing once the array is loaded.  The handle must have been set up on the current
 * device (A2LS_ERR_STATE otherwise).  All calls on a device share the one array and overwrite every
 * scratch value they read, so no clearing is needed, but calls whose work overlaps on the GPU
 * (other streams, handles or threads) race on it.  Asynchronous on the handle's stream.
 */
int a2ls_apply_static(a2ls_handle* h, const double* r, double* z);

/*
 * a2ls_spmv -- y = A x with the handle's FP64 copy of A (x, y: device, n doubles).
 * Asynchronous on the handle's stream.
 */
int a2ls_spmv(a2ls_handle* h, const double* x, double* y);

/* ---------------------------------------------------------------------------------------------
 * Learned warm start (not part of the paper; an addition of this library).
 *
 * The local eigenproblems of Eq. 3.1 are solved by a restarted block Krylov iteration whose
 * starting block is random unless a2ls_options::warm_start names a network.  The network reads
 * each subdomain's local matrix A_ii and lumped sums s_i (Definition 3.1) and proposes 16 columns:
 *   edge weights  w_lk = (|a_lk| + |a_kl|) / (2 sqrt(|a_ll a_kk|)) on entries with a_lk, a_kl != 0;
 *   features      x_l = [1, d_l / max d, clip(log(d_l / mean d) / 10, -1, 1), [l in Omega_Gamma_i],
 *                        s_l / d_l, sum_k w_lk / 4], d_l = |a_ll|;
 *   three message-passing layers of width 64, h_t = relu(h_{t-1} W_s + (W h_{t-1}) W_n + b),
 *   an output layer to 16 columns and 32 steps of p <- 0.9 D^-1/2 W D^-1/2 p + 0.1 p_0.
 * Weights are held in bfloat16 for the forward pass (FP32 master copy for training); all sums
 * accumulate in FP32.  Training minimises, per subdomain, L_i = min_C ||Z_i - Y C||^2 / m_i (plus
 * 1e-6 ||C||^2 / m_i) against the eigenvectors Z_i (n_i x m_i) that the setup selected, averaged over
 * the subdomains with a target, with Adam (beta 0.9 / 0.999, eps 1e-8).
 * Parameters are one float vector of a2ls_gnn_num_params() entries in this order, each matrix
 * row-major (rows = inputs): W_in 6x64, b_in 64, then for t = 1..3: W_s,t 64x64, W_n,t 64x64,
 * b_t 64, then W_out 64x16.
 * All a2ls_gnn_* calls return an a2ls_status and synchronise their stream; a network must not be
 * used by two calls at once.
 * --------------------------------------------------------------------------------------------- */

/* Number of float parameters of the network (26240). */
int64_t a2ls_gnn_num_params(void);

/* New network with He-normal weights (std sqrt(2 / inputs)) drawn from `seed`, zero biases.
 * stream: cudaStream_t for the network's own work (NULL = legacy default stream). */
int a2ls_gnn_create(uint64_t seed, void* stream, a2ls_gnn** out);
int a2ls_gnn_destroy(a2ls_gnn* g);

/* host: count = a2ls_gnn_num_params() floats.  set_params also clears the Adam state and the
 * gradient accumulator. */
int a2ls_gnn_get_params(a2ls_gnn* g, float* host, int64_t count);
int a2ls_gnn_set_params(a2ls_gnn* g, const float* host, int64_t count);

/* Mean of the gradients accumulated by a2ls_gnn_loss_grad since the last Adam step (zeros if none). */
int a2ls_gnn_get_grads(a2ls_gnn* g, float* host, int64_t count);

/* A training or inference sample: the local graphs and features of a set-up handle's subdomains
 * and, as target, the eigenvectors its setup selected (none for one-level variants or nev = 0).
 * The sample copies what it needs; the handle may be destroyed afterwards.  Its work runs on the
 * handle's stream. */
int a2ls_gnn_sample_create(a2ls_handle* h, a2ls_gnn_sample** out);
/* Replace the target.  m: host, N int32 in [0, 32]; Z: host doubles, for each subdomain an
 * n_i x m_i row-major block in the local order of A2LS_Q_SUBDOMAINS. */
int a2ls_gnn_sample_set_target(a2ls_gnn_sample* s, const int32_t* m, const double* Z);
int a2ls_gnn_sample_destroy(a2ls_gnn_sample* s);

/* Items for a2ls_gnn_sample_query (copied to host; rows in the local order of A2LS_Q_SUBDOMAINS). */
enum {
  A2LS_GQ_FEATURES = 0,    /* float[sum n_i * 8]: the 6 features per row, then two zeros */
  A2LS_GQ_ROWPTR = 1,      /* int64[sum n_i + 1]: entries of each row (one per entry of the row of A) */
  A2LS_GQ_COLS = 2,        /* int32[entries]: flat row index off_i + k of the neighbour, or -1 */
  A2LS_GQ_WEIGHTS = 3,     /* float[entries]: w_lk (0 where the column is -1) */
  A2LS_GQ_SWEIGHTS = 4,    /* float[entries]: w_lk / sqrt(deg_l deg_k) */
  A2LS_GQ_TARGET_COLS = 5  /* int32[N]: m_i of the target */
};
int a2ls_gnn_sample_query(a2ls_gnn_sample* s, int32_t what, void* out, int64_t capacity, int64_t* needed);

/* Y: host, sum n_i x 16 floats, the network's proposal for every subdomain. */
int a2ls_gnn_forward(a2ls_gnn* g, a2ls_gnn_sample* s, float* Y);

/* Forward pass, loss and backward pass on one sample; adds the sample's gradient to the
 * accumulator.  loss: host, receives the sample's mean loss (may be NULL).  STATE if the sample
 * has no target. */
int a2ls_gnn_loss_grad(a2ls_gnn* g, a2ls_gnn_sample* s, double* loss);

/* One Adam step (Kingma and Ba, 2015) with the mean accumulated gradient; clears the accumulator.
 * STATE if nothing was accumulated. */
int a2ls_gnn_adam_step(a2ls_gnn* g, double lr);

/* Kernels the network's own calls have launched so far. */
int64_t a2ls_gnn_launches(const a2ls_gnn* g);

#ifdef __cplusplus
}
#endif

#endif /* A2LS_H */

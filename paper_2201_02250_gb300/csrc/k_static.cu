// a2ls_apply_static: the apply of a2ls_apply with its scratch vectors taken
// from a fixed array in the library's static device memory instead of the
// handle's workspace, so that the call allocates nothing at all.
//
// Scratch layout (doubles, each piece padded to 256 bytes):
//   q: n | t: n | g: n0 | c: n0 | yloc: sum n_i (only ASM variants or the multiplicity PoU)
// Every piece is completely overwritten by each call before it is read, so
// nothing has to be cleared between calls.  The array is shared by all calls
// on a device: two calls whose work overlaps on the GPU (different streams,
// different handles, or other threads) race on it.
#include "a2ls_internal.cuh"

#include <algorithm>

namespace a2ls {

// kernels of the apply, defined in k_krylov.cu
__global__ void k_restrict(const int* ni, const int* nI, const int* off, const int* idx, const int* m,
                           const int* coff, const int64_t* woff, const double* __restrict__ W,
                           const double* __restrict__ r, double* g, int boolean_pou);
__global__ void k_gemv(int n0, const double* __restrict__ Einv, const double* __restrict__ g,
                       double* __restrict__ c);
__global__ void k_prolong(int n, const int* mrow, const int* mpos, const int* msub, const int* off, const int* m,
                          const int* coff, const int64_t* woff, const double* D, const double* __restrict__ W,
                          const double* __restrict__ c, double* q);
__global__ void k_combine(int n, const int* mrow, const int* mpos, const double* __restrict__ yloc,
                          const double* __restrict__ q, double* z);

// 1 Mi doubles = 8 MiB per device, held from the first a2ls_setup on that device until process exit
constexpr size_t STATIC_SCRATCH_DOUBLES = size_t(1) << 20;
static __device__ __align__(256) double g_static_scratch[STATIC_SCRATCH_DOUBLES];

void record_error(const char* msg);  // capi.cu: sets the message a2ls_last_error() returns

static int fail_status(int code, const char* msg) {
  record_error(msg);
  return code;
}

template <class F>
static int guarded_call(F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    record_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    record_error(e.what());
    return A2LS_ERR_CUDA;
  }
}

// Device address of the static scratch on the current device.  Looked up on every call, so that a
// context the caller recreated (cudaDeviceReset) is never written through a stale address.  The
// lookup loads the module that holds the array the first time it runs in a context; with CUDA's lazy
// module loading that load maps the array's 8 MiB, so a2ls_setup performs it (prime_static_scratch)
// and the apply itself then only reads the address of an already loaded module.
static double* static_scratch_address() {
  void* p = nullptr;
  A2LS_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
  return static_cast<double*>(p);
}

void prime_static_scratch() { (void)static_scratch_address(); }

static size_t pad32(size_t v) { return (v + 31) / 32 * 32; }

static void apply_static(a2ls_handle* h, const double* r, double* z) {
  const int v = h->opt.variant;
  const bool ras = (v == A2LS_DEFLATED_RAS || v == A2LS_ADDITIVE_RAS || v == A2LS_ONE_LEVEL_RAS);
  const bool coarse = (v != A2LS_ONE_LEVEL_RAS && v != A2LS_ONE_LEVEL_ASM) && h->n0 > 0;
  const bool deflated = (v == A2LS_DEFLATED_RAS || v == A2LS_DEFLATED_ASM);
  const bool boolean = h->opt.pou == A2LS_POU_BOOLEAN;
  const int mode = ras ? (boolean ? 0 : 1) : 2;
  const size_t need = 2 * pad32(h->n) + (coarse ? 2 * pad32(h->n0) : 0) + (mode != 0 ? pad32(h->sum_n) : 0);
  if (need > STATIC_SCRATCH_DOUBLES)
    fail(A2LS_ERR_ARG,
         "a2ls_apply_static needs %zu scratch doubles for this problem; the static scratch holds %zu "
         "(2n + 2 n0, plus sum n_i for ASM or the multiplicity partition of unity)",
         need, STATIC_SCRATCH_DOUBLES);
  // the handle's data must live on the current device, the one whose static array is used
  int dev = 0;
  A2LS_CUDA(cudaGetDevice(&dev));
  cudaPointerAttributes attr{};
  A2LS_CUDA(cudaPointerGetAttributes(&attr, h->rowptr));
  if (attr.device != dev)
    fail(A2LS_ERR_STATE, "the handle was set up on device %d but device %d is current", attr.device, dev);
  double* base = static_scratch_address();
  double* q = base;
  double* t = q + pad32(h->n);
  double* g = t + pad32(h->n);
  double* c = g + (coarse ? pad32(h->n0) : 0);
  double* yloc = c + (coarse ? pad32(h->n0) : 0);
  cudaStream_t st = h->st;
  const int grid_n = (int)std::max<int64_t>(1, std::min<int64_t>(152 * 8, ((int64_t)h->n + 255) / 256));

  auto local = [&](const double* tin, const double* qin) {
    double* out = (mode == 0) ? z : yloc;
    local_solves_any(h, tin, qin, out, mode);
    if (mode != 0) {
      k_combine<<<grid_n, 256, 0, st>>>(h->n, h->d_mrow, h->d_mpos, yloc, qin, z);
      A2LS_LAUNCH();
    }
  };
  if (!coarse) {
    local(r, nullptr);
    return;
  }
  k_restrict<<<h->N, 256, 0, st>>>(h->d_ni, h->d_nI, h->d_off, h->d_idx, h->d_m, h->d_coff, h->d_woff, h->d_W, r,
                                   g, boolean);
  A2LS_LAUNCH();
  k_gemv<<<std::min(152 * 8, ceil_div((int64_t)h->n0 * 32, 256)), 256, 0, st>>>(h->n0, h->d_Einv, g, c);
  A2LS_LAUNCH();
  k_prolong<<<grid_n, 256, 0, st>>>(h->n, h->d_mrow, h->d_mpos, h->d_msub, h->d_off, h->d_m, h->d_coff,
                                    h->d_woff, h->d_D, h->d_W, c, q);
  A2LS_LAUNCH();
  if (deflated) {
    spmv(h, q, t, r, st);  // t = r - A q
    local(t, q);
  } else {
    local(r, q);
  }
}

}  // namespace a2ls

extern "C" int a2ls_apply_static(a2ls_handle* h, const double* r, double* z) {
  using namespace a2ls;
  if (!h || !r || !z) return fail_status(A2LS_ERR_ARG, "null argument");
  if (r == z) return fail_status(A2LS_ERR_ARG, "r and z must not alias");
  return guarded_call([&]() -> int {
    apply_static(h, r, z);
    return A2LS_OK;
  });
}

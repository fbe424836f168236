// nslct_backward_noalloc: nslct_backward for callers that cannot allocate.
//
// nslct_backward needs two scratch buffers and, when the caller does not pass
// them, allocates them on its first call (cudaMalloc): a field-sized buffer for
// the value path and a small buffer of per-CTA partial sums. Some callers cannot
// allow that -- code running while a CUDA graph is being captured, code under a
// caching allocator that must see every device allocation, or code with a fixed
// memory budget. This entry point allocates nothing:
//   * the per-CTA partial sums live in the file-scope device array below, of a
//     fixed size that covers every supported field (any Nx, Ny <= 4096); every
//     GPU that loads the library keeps it (about 196 KB) until the process exits;
//   * the value path runs in the caller's y buffer, which on return holds
//     L^{-1} y (the reconstructed forward input) instead of y.
// The array's host-side name is not a device address: the device address is
// looked up with cudaGetSymbolAddress, with the plan's device current, on the
// first call in each CUDA context of that device (the first call after a
// cudaDeviceReset looks it up again). That first call should therefore come
// before any stream capture.
#include <mutex>

#include "internal.h"

// defined in backward.cu
int nslct_backward_impl(nslct_plan_t p, const void* grad_out, const void* y, void* grad_in, double* grad_theta,
                        double* grad_chirp, void* ws, double* partials, int stride, cudaStream_t s, int nbatch,
                        long long fstride, int only_pass);

namespace {

// Rows of partial sums per accumulating pass: one per CTA of a dual pass, at
// most max(Nx, Ny) / 2 + 1 = 2049 for the largest supported field.
constexpr int kNoallocRows = 2049;
static __device__ __align__(256) double g_noalloc_partials[4 * kNoallocRows * 3];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
// per device: the context the address was looked up in, and the address
void* g_partials_ctx[kMaxDevices] = {};
double* g_partials_addr[kMaxDevices] = {};

typedef int (*CtxGetCurrentFn)(void**);

// The driver's current context (cuCtxGetCurrent, through the runtime's entry
// point query, so no link against libcuda); null if it cannot be had.
void* current_context() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(ptr);
  });
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

// Device address of g_noalloc_partials on the current device, looked up once
// per (device, context).
int partials_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return NSLCT_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  void* ctx = current_context();
  if (!g_partials_addr[device] || !ctx || ctx != g_partials_ctx[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_partials) != cudaSuccess || !ptr) return NSLCT_E_CUDA;
    g_partials_addr[device] = static_cast<double*>(ptr);
    g_partials_ctx[device] = ctx;
  }
  *out = g_partials_addr[device];
  return NSLCT_OK;
}

}  // namespace

extern "C" int nslct_backward_noalloc(nslct_plan_t p, const void* grad_out, void* y_inout, void* grad_in,
                                      double* grad_theta, double* grad_chirp, nslct_stream_t stream) {
  if (!p || !grad_out || !y_inout || !grad_in) return NSLCT_E_ARG;
  if (p->padded || p->type2) return NSLCT_E_UNSUPPORTED;
  if (grad_theta && !p->has_theta) return NSLCT_E_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(grad_out) | reinterpret_cast<uintptr_t>(y_inout) |
       reinterpret_cast<uintptr_t>(grad_in)) & 15u)
    return NSLCT_E_ARG;
  // y_inout is the value path's input and output at once; grad_in must not
  // overlap it, or the two paths would overwrite each other
  {
    const size_t bytes = (size_t)p->Nx * p->Ny * (p->prec ? 16u : 8u);
    const uintptr_t y0 = reinterpret_cast<uintptr_t>(y_inout), g0 = reinterpret_cast<uintptr_t>(grad_in);
    if (y0 < g0 + bytes && g0 < y0 + bytes) return NSLCT_E_ARG;
  }
  const int rows = (p->Nx > p->Ny ? p->Nx : p->Ny) / 2 + 1;
  if (rows > kNoallocRows) return NSLCT_E_SIZE;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return NSLCT_E_CUDA;
  if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess) return NSLCT_E_CUDA;
  double* partials = nullptr;
  int rc = partials_address(p->device, &partials);
  if (rc == NSLCT_OK)
    rc = nslct_backward_impl(p, grad_out, y_inout, grad_in, grad_theta, grad_chirp, y_inout, partials, kNoallocRows,
                             reinterpret_cast<cudaStream_t>(stream), 1, 0, -1);
  if (prev != p->device) cudaSetDevice(prev);
  return rc;
}

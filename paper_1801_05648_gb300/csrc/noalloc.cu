// fsi_mass_solve_noalloc: the solid-mass Chebyshev solve (block inverse 4 of
// fsi_apply_block) for callers that cannot allocate device memory at call time,
// e.g. code that runs while a stream is being captured into a CUDA graph (where
// cudaMalloc is not permitted), or code living under a device-memory budget that
// another framework's allocator owns.  Its two scratch vectors live in a
// file-scope device array, fixed at load time, instead of in memory the context
// allocated; the caller passes only the input and output vectors.
#include "../../include/fsi.h"
#include "solver.cuh"

namespace {

// Scratch of the entry point: two FP64 vectors (ping-pong iterate and Chebyshev
// direction) of at most kNoAllocMaxRows entries each, 16 MiB in total.  Every
// GPU that loads the library holds this array until the process exits.
constexpr int64_t kNoAllocMaxRows = int64_t(1) << 20;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxRows];

// Device address of g_noalloc_scratch on the context's device (which the caller
// has made current).  In host code the array's name is only a host-side stand-in,
// not a device address.  The address is looked up on the first call on a context
// and kept with that context: a context lives inside one CUDA context of one
// device, so the address stays valid for as long as the context does (a device
// reset invalidates both together, and contexts made afterwards look it up anew).
int scratch_address(fsi::Context& C, double** out, std::string& err) {
  if (!C.noalloc_scratch) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) { err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e); return FSI_ECUDA; }
    C.noalloc_scratch = p;
  }
  *out = static_cast<double*>(C.noalloc_scratch);
  return FSI_OK;
}

}  // namespace

struct fsi_ctx {
  fsi::Context C;
};

extern "C" int fsi_mass_solve_noalloc(fsi_ctx* ctx, const double* in_dev, double* out_dev) {
  if (!ctx) return FSI_EINVAL;
  fsi::Context& C = ctx->C;
  try {
    if (!C.built) { C.err = "fsi_mass_solve_noalloc before fsi_precond_build"; return FSI_EINVAL; }
    if (!in_dev || !out_dev) { C.err = "null vector"; return FSI_EINVAL; }
    const int64_t n = C.mass.A.rows();
    if (n > kNoAllocMaxRows) {
      C.err = "fsi_mass_solve_noalloc: the solid block has " + std::to_string(n) +
              " displacement DOFs, more than the static scratch holds (" + std::to_string(kNoAllocMaxRows) + ")";
      return FSI_EINVAL;
    }
    fsi::DeviceGuard on_device(C.device);
    double* scratch = nullptr;
    std::string err;
    const int rc = scratch_address(C, &scratch, err);
    if (rc != FSI_OK) { C.err = err; return rc; }
    // xb = scratch[0, n), d = scratch[max, max + n); the first Chebyshev step
    // overwrites both, so nothing needs clearing between calls.
    fsi::cheb_apply_scratch(C.mass, in_dev, out_dev, scratch, scratch + kNoAllocMaxRows, C.s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { C.err = cudaGetErrorString(e); return FSI_ECUDA; }
    C.err.clear();
    return FSI_OK;
  } catch (const fsi::Error& e) {
    C.err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    C.err = e.what();
    return FSI_ECUDA;
  }
}

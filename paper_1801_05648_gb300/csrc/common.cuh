// Shared device-side definitions of the FSI solver library: error handling,
// device buffers, the block-sparse-row (BSR) matrix type and small helpers.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <stdexcept>
#include <utility>

namespace fsi {

// Error raised inside the library; converted to a status code at the C ABI.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

enum Status { OK = 0, EINVAL_ = -1, ENOMEM_ = -2, ECUDA_ = -3, ENOTCONV_ = -4, EBREAKDOWN_ = -5, ENONFINITE_ = -6 };

#define FSI_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      if (e_ == cudaErrorMemoryAllocation)                                                      \
        throw ::fsi::Error(::fsi::ENOMEM_, std::string("out of device memory at ") + #call);    \
      throw ::fsi::Error(::fsi::ECUDA_, std::string(cudaGetErrorString(e_)) + " at " + #call);  \
    }                                                                                           \
  } while (0)

// Kernel launches issued by the library (captured launches are re-counted per
// graph replay by the solver).
inline int64_t g_kernel_launches = 0;

#define FSI_CHECK_LAUNCH()        \
  do {                            \
    ++::fsi::g_kernel_launches;   \
    FSI_CUDA(cudaGetLastError()); \
  } while (0)

// Programmatic dependent launch (sm_90 and later).  A kernel started with
// launch_k() may be scheduled while the previous kernel of its stream drains
// (its blocks become resident during that kernel's tail); it executes
// dep_wait() before its first global-memory access, which returns once the
// previous kernel has completed and its writes are visible.  Every kernel
// launched through launch_k() therefore starts with dep_wait().  Off for the
// whole process when a context was set up with FSI_NO_PDL.
__device__ __forceinline__ void dep_wait() {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 900)
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

// Launch knobs (programmatic dependent launch here; the SpMV shape and the coarse
// V-cycle threshold below) are per thread: every entry point that takes a context
// applies that context's values for the duration of the call (KnobScope in
// fsi_api.cu), so contexts with different parameters do not interfere.
inline bool& pdl_enabled() {
  thread_local bool on = true;
  return on;
}
// Learned-stage MLP on the tensor cores (else on the CUDA cores).
inline bool& mlp_tensor_cores() {
  thread_local bool on = true;
  return on;
}
// Host-side fault injection for the tests of the bounded waits (0 in normal use):
// kInjectCoarseBarrier: the coarse V-cycle's grid barrier waits for one CTA more than
// the launch has; kInjectMlpCommit: the tensor-core MLP does not commit its first
// layer's MMAs to the barrier it then waits on.  Either wait then runs out.
enum { kInjectCoarseBarrier = 1, kInjectMlpCommit = 2 };
inline int& fault_inject() {
  thread_local int v = 0;
  return v;
}

// Streaming multiprocessors of the current device (looked up once per device).
inline int device_sms() {
  constexpr int kMaxDev = 64;
  static int cache[kMaxDev] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 152;
  int v = __atomic_load_n(&cache[dev], __ATOMIC_RELAXED);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    __atomic_store_n(&cache[dev], v, __ATOMIC_RELAXED);
  }
  return v;
}

template <class... KArgs, class... Args>
void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args);

inline void require(bool ok, const std::string& msg) {
  if (!ok) throw Error(EINVAL_, msg);
}

// Makes `dev` the calling thread's current CUDA device while the guard lives and
// restores the previous device afterwards (nothing to do when dev < 0 or when it
// is current already).  A context's streams and memory belong to the device that
// was current at fsi_setup; every entry point runs under a guard for it, so a
// caller whose thread has since switched devices still launches on the right one.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (dev < 0) return;
    int cur = -1;
    FSI_CUDA(cudaGetDevice(&cur));
    if (cur == dev) return;
    FSI_CUDA(cudaSetDevice(dev));
    prev = cur;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Runs setup(dev) once per device dev, on the current one: a kernel's function attributes
// and a __device__ variable's address belong to the copy of the module that each
// device loads, so what was set up on one device does not hold on another.  `done`
// is the call site's set of devices already set up (bit d for device d).  Two
// threads may both run it for the same device; it must be idempotent.
template <class F>
void once_per_device(std::atomic<unsigned long long>& done, F&& setup) {
  int dev = 0;
  FSI_CUDA(cudaGetDevice(&dev));
  require(dev >= 0 && dev < 64, "device ordinal above 63");
  const unsigned long long bit = 1ull << dev;
  if (done.load(std::memory_order_acquire) & bit) return;
  setup(dev);
  done.fetch_or(bit, std::memory_order_release);
}

// Owning device buffer.
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    n = count;
    if (count) FSI_CUDA(cudaMalloc(&p, count * sizeof(T)));
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr; n = 0;
  }
  T* get() const { return p; }
};

// Block sparse row matrix on the device: nbr x nbc blocks of br x bc values,
// block values row-major, blocks of a row stored consecutively with sorted
// block-column indices.  Values may exist in FP64, FP32 or both.
struct Bsr {
  int nbr = 0, nbc = 0, br = 1, bc = 1;
  int64_t nnzb = 0;
  DBuf<int> rowptr;     // nbr + 1
  DBuf<int> colind;     // nnzb
  DBuf<double> v64;     // nnzb * br * bc
  DBuf<float> v32;      // optional FP32 copy
  DBuf<int16_t> cd16;   // optional, square matrices: block column minus block row as int16 (read by the
                        // FP32 Chebyshev steps when every offset fits; 2 bytes per block instead of 4)
  DBuf<int4> ord2;      // optional: the slot table of the two-matrix SpMV with the partner whose row
  const int* ord2_rp2 = nullptr;   // pointers these are: block rows sorted by (length here, length
                        // there) within 32-row windows, {row | length << 24, first block, first
                        // partner block, partner length} per slot (k_pair_order)
  int stage_rows = 0;   // 2 x 2 FP32 with cd16: block rows per CTA the staged Chebyshev kernel was sized for
  int stage_max = 0;    // ... and the largest CTA slice in blocks, from the 8-entry boundary below it
  int tpr = 32;         // threads per block row of the FP32 SpMV, from the mean row length
  int tpr64 = 2;        // ... of the FP64 SpMV (fewer lanes: FP64 issue slots are scarce)
  int64_t rows() const { return (int64_t)nbr * br; }
  int64_t cols() const { return (int64_t)nbc * bc; }
  template <class T> const T* vals() const;
  // algorithmic bytes of one SpMV: values + column indices + row pointers + x + y
  // (FP32 products of a matrix with 16-bit column offsets read 2 bytes per block index)
  double spmv_bytes(int value_bytes) const {
    const int ib = (value_bytes == 4 && cd16.p) ? 2 : 4;
    return (double)nnzb * (br * bc * value_bytes + ib) + 4.0 * (nbr + 1) + (double)value_bytes * (cols() + rows());
  }
};
// FP32 copies of blocks with 9 values (3 x 3) are stored planar (values 0-3 of
// every block, then 4-7, then 8; see load_block in spmv.cuh); all other copies are
// row-major blocks.
__host__ __device__ constexpr bool planar_fp32_shape(int br, int bc) { return br * bc == 9; }

template <> inline const double* Bsr::vals<double>() const { return v64.p; }
template <> inline const float* Bsr::vals<float>() const { return v32.p; }

// Lanes per block row: the most lanes (a power of two, at most 32) that leave
// each lane at least `min_per_lane` blocks of an average row, so a row's blocks
// are read by neighbouring lanes (coalesced) in about one pass per lane,
// whatever the number of rows.  FP32 rows keep two blocks per lane.  FP64 rows
// keep at least eight: the FP64 pipe of this GPU retires a small fraction of the
// FP32 rate, and the shuffle reduction across a wide lane group would cost more
// FP64 instructions than the products themselves.
inline int lanes_for(int64_t nnzb, int nbr, double min_per_lane) {
  const double mean = nbr ? (double)nnzb / nbr : 0.0;
  int t = 1;
  while (t < 32 && mean / (2 * t) >= min_per_lane) t *= 2;
  return t;
}

// SpMV launch shape knobs (fsi_params: spmv_unroll, spmv_prefetch).
struct SpmvTuning {
  int unroll = 4;      // blocks each lane loads before multiplying: 4 or 8 (8 only for small blocks)
  int prefetch = 1;    // 0 none, 1 L2 bulk prefetch of each CTA's matrix slice, 2 also persistent CTAs
  int ctas_per_sm = 5; // persistent grid size per SM (prefetch 2)
  int lane_shift = 0;  // FP32 launches: lanes per block row divided by 2^lane_shift (at least 1)
  int keep_x64 = 1;    // FP64 launches gather x with the L2 evict-last policy (see OuterOperatorScope)
  int stage = 0;       // 2 x 2 FP32 Chebyshev steps with the column offsets staged in shared memory
  int order = 1;       // two-matrix launches take their rows in the order of Bsr::ord2 when it is built
  int setup_depth = 0; // > 0 while matrices are being built: no reads before the dependency wait
};
inline SpmvTuning& spmv_tuning() {
  thread_local SpmvTuning t;
  return t;
}

// Marks the set-up phase (context set-up, preconditioner build): an SpMV may then
// be launched right after the kernel that writes its matrix, so it reads no matrix
// memory before its dependency wait.
struct SetupPhase {
  SetupPhase() { ++spmv_tuning().setup_depth; }
  ~SetupPhase() { --spmv_tuning().setup_depth; }
  SetupPhase(const SetupPhase&) = delete;
  SetupPhase& operator=(const SetupPhase&) = delete;
};

// The outer FP64 operator gathers x with the default L2 policy: measured on the
// 1024x512 system, evict-last gathers cut its DRAM traffic from 7.5 to 6.4 GB but
// made it 5% slower (it is bound by the FP64 pipe), while the FP64 V-cycles, bound
// by memory, ran 8% faster with them.
struct OuterOperatorScope {
  int saved;
  OuterOperatorScope() : saved(spmv_tuning().keep_x64) { spmv_tuning().keep_x64 = 0; }
  ~OuterOperatorScope() { spmv_tuning().keep_x64 = saved; }
  OuterOperatorScope(const OuterOperatorScope&) = delete;
  OuterOperatorScope& operator=(const OuterOperatorScope&) = delete;
};

inline void set_tpr(Bsr& A) {
  A.tpr = lanes_for(A.nnzb, A.nbr, 2.0);
  A.tpr64 = lanes_for(A.nnzb, A.nbr, 8.0);
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

template <class... KArgs, class... Args>
void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  FSI_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
  ++g_kernel_launches;
}


}  // namespace fsi

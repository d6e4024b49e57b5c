#include "vec.cuh"

namespace fsi {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b > device_sms() * 16) b = device_sms() * 16;
  return (int)(b < 1 ? 1 : b);
}

template <class T>
__global__ void k_axpby(int64_t n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  dep_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T v = a * x[i];
    if (b != T(0)) v += b * y[i];
    y[i] = v;
  }
}

template <class T>
__global__ void k_axpbyz(int64_t n, T a, const T* __restrict__ x, T b, const T* __restrict__ y, T* __restrict__ z) {
  dep_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = a * x[i] + b * y[i];
}

template <class T>
__global__ void k_vmul(int64_t n, const T* __restrict__ x, const T* __restrict__ w, T* __restrict__ y) {
  dep_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * w[i];
}

template <class T>
__global__ void k_vfma(int64_t n, const T* __restrict__ w, const T* __restrict__ x, T* __restrict__ y) {
  dep_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += w[i] * x[i];
}

template <class Ti, class To>
__global__ void k_cast(int64_t n, const Ti* __restrict__ x, To* __restrict__ y) {
  dep_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (To)x[i];
}

// Block-wide sum of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (threadIdx.x < (blockDim.x >> 5)) v = sh[threadIdx.x];
  if (w == 0)
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// partials[blockIdx] = sum over this block's contiguous chunk of x*y
template <class T>
__global__ void __launch_bounds__(kRedThreads) k_dot_partial(int64_t n, const T* __restrict__ x,
                                                              const T* __restrict__ y, double* __restrict__ partials) {
  dep_wait();
  __shared__ double sh[32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += (double)x[i] * (double)y[i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// out[c] = (sqrt?) sum_k partials[c * np + k], one block per column c
// (out[c] = 0 instead when *skip != 0)
__global__ void __launch_bounds__(kRedThreads) k_reduce_cols(const double* __restrict__ partials, int np,
                                                             const int* jcount, int joff, double* out, int take_sqrt,
                                                             const int* skip) {
  dep_wait();
  __shared__ double sh[32];
  const int c = blockIdx.x;
  const int J = jcount ? (*jcount + joff) : joff;
  if (c >= J) return;
  if (skip && *skip) {
    if (threadIdx.x == 0) out[c] = 0.0;
    return;
  }
  double acc = 0.0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) acc += partials[(size_t)c * np + k];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[c] = take_sqrt ? sqrt(acc) : acc;
}

// Multi-dot: partials[i * gridDim + block] = <V_i, w> over the block's chunk, i < J.
// Four basis vectors per pass over the chunk of w.
__global__ void __launch_bounds__(kRedThreads) k_mdot_partial(int64_t n, const double* __restrict__ V, int64_t ldv,
                                                              const int* __restrict__ jcount, int joff,
                                                              const double* __restrict__ w,
                                                              double* __restrict__ partials,
                                                              const int* __restrict__ skip) {
  dep_wait();
  if (skip && *skip) return;
  __shared__ double sh[32];
  const int J = *jcount + joff;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  for (int i0 = 0; i0 < J; i0 += 4) {
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const int ni = J - i0 < 4 ? J - i0 : 4;
    const double* v0 = V + (size_t)i0 * ldv;
    for (int64_t r = lo + threadIdx.x; r < hi; r += blockDim.x) {
      const double wr = __ldg(w + r);
      a0 += __ldcs(v0 + r) * wr;
      if (ni > 1) a1 += __ldcs(v0 + ldv + r) * wr;
      if (ni > 2) a2 += __ldcs(v0 + 2 * ldv + r) * wr;
      if (ni > 3) a3 += __ldcs(v0 + 3 * ldv + r) * wr;
    }
    double s0 = block_sum(a0, sh);
    if (threadIdx.x == 0) partials[(size_t)i0 * gridDim.x + blockIdx.x] = s0;
    if (ni > 1) { double s = block_sum(a1, sh); if (threadIdx.x == 0) partials[(size_t)(i0 + 1) * gridDim.x + blockIdx.x] = s; }
    if (ni > 2) { double s = block_sum(a2, sh); if (threadIdx.x == 0) partials[(size_t)(i0 + 2) * gridDim.x + blockIdx.x] = s; }
    if (ni > 3) { double s = block_sum(a3, sh); if (threadIdx.x == 0) partials[(size_t)(i0 + 3) * gridDim.x + blockIdx.x] = s; }
  }
}

// w -= sign * sum_i h[i] V_i  over the block's chunk; optional per-block sum of w^2
__global__ void __launch_bounds__(kRedThreads) k_maxpy(int64_t n, const double* __restrict__ V, int64_t ldv,
                                                       const int* __restrict__ jcount, int joff,
                                                       const double* __restrict__ h, double sign,
                                                       double* __restrict__ w, double* __restrict__ nrm_partials,
                                                       const int* __restrict__ skip) {
  dep_wait();
  if (skip && *skip) return;
  __shared__ double hs[256];
  __shared__ double sh[32];
  const int J = *jcount + joff;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double nacc = 0.0;
  for (int i0 = 0; i0 < J || i0 == 0; i0 += 256) {
    const int cnt = J - i0 < 256 ? J - i0 : 256;
    __syncthreads();
    if (threadIdx.x < cnt) hs[threadIdx.x] = sign * h[i0 + threadIdx.x];
    __syncthreads();
    const bool last = i0 + 256 >= J;
    for (int64_t r = lo + threadIdx.x; r < hi; r += blockDim.x) {
      double acc = w[r];
      const double* vp = V + (size_t)i0 * ldv + r;
      for (int i = 0; i < cnt; ++i) acc -= hs[i] * __ldcs(vp + (size_t)i * ldv);
      w[r] = acc;
      if (last) nacc += acc * acc;
    }
    if (J <= 0) break;
  }
  if (nrm_partials) {
    nacc = block_sum(nacc, sh);
    if (threadIdx.x == 0) nrm_partials[blockIdx.x] = nacc;
  }
}

// ---- 16-byte variants of the Gram-Schmidt products (basis columns, w and the
// chunk starts 16-byte aligned): the FP64 products are issue-bound, so each thread
// takes two consecutive elements per load instruction and the multi-dot eight
// basis vectors per pass over its chunk, cutting the load, address and loop
// instructions per FMA.  A block's chunk starts at an even element.
constexpr int kDotCols = 8;

__device__ __forceinline__ void chunk_of(int64_t n, int64_t& lo, int64_t& hi) {
  int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  chunk = (chunk + 1) & ~(int64_t)1;
  lo = blockIdx.x * chunk;
  hi = lo + chunk < n ? lo + chunk : n;
}

__global__ void __launch_bounds__(kRedThreads, 4) k_mdot_partial_v2(int64_t n, const double* __restrict__ V,
                                                                 int64_t ldv, const int* __restrict__ jcount,
                                                                 int joff, const double* __restrict__ w,
                                                                 double* __restrict__ partials,
                                                                 const int* __restrict__ skip) {
  dep_wait();
  if (skip && *skip) return;
  __shared__ double sh[kDotCols][kRedThreads / 32];
  const int J = *jcount + joff;
  int64_t lo, hi;
  chunk_of(n, lo, hi);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 < J; i0 += kDotCols) {
    const int ni = J - i0 < kDotCols ? J - i0 : kDotCols;
    const double* v0 = V + (size_t)i0 * ldv;
    double acc[kDotCols];
#pragma unroll
    for (int u = 0; u < kDotCols; ++u) acc[u] = 0.0;
    for (int64_t r = lo + 2 * threadIdx.x; r < hi; r += 2 * blockDim.x) {
      if (r + 1 < hi) {
        const double2 wr = __ldg(reinterpret_cast<const double2*>(w + r));
#pragma unroll
        for (int u = 0; u < kDotCols; ++u)
          if (u < ni) {
            const double2 v = __ldcs(reinterpret_cast<const double2*>(v0 + (size_t)u * ldv + r));
            acc[u] = fma(v.y, wr.y, fma(v.x, wr.x, acc[u]));
          }
      } else {
        const double wr = __ldg(w + r);
#pragma unroll
        for (int u = 0; u < kDotCols; ++u)
          if (u < ni) acc[u] = fma(__ldcs(v0 + (size_t)u * ldv + r), wr, acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kDotCols; ++u) {
      double a = acc[u];
      for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
      if (lane == 0) sh[u][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < ni) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[threadIdx.x][q];
      partials[(size_t)(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// w -= sign * sum_i h[i] V_i over the block's chunk, two elements per thread and
// load; each element sums the basis vectors in increasing order (as k_maxpy).
__global__ void __launch_bounds__(kRedThreads) k_maxpy_v2(int64_t n, const double* __restrict__ V, int64_t ldv,
                                                          const int* __restrict__ jcount, int joff,
                                                          const double* __restrict__ h, double sign,
                                                          double* __restrict__ w, double* __restrict__ nrm_partials,
                                                          const int* __restrict__ skip) {
  dep_wait();
  if (skip && *skip) return;
  extern __shared__ double hs[];
  __shared__ double sh[32];
  const int J = *jcount + joff;
  int64_t lo, hi;
  chunk_of(n, lo, hi);
  for (int i = threadIdx.x; i < J; i += blockDim.x) hs[i] = sign * h[i];
  __syncthreads();
  double nacc = 0.0;
  for (int64_t r = lo + 2 * threadIdx.x; r < hi; r += 2 * blockDim.x) {
    if (r + 1 < hi) {
      double2 acc = *reinterpret_cast<const double2*>(w + r);
      const double* vp = V + r;
      for (int i = 0; i < J; ++i) {
        const double hv = hs[i];
        const double2 v = __ldcs(reinterpret_cast<const double2*>(vp + (size_t)i * ldv));
        acc.x -= hv * v.x;
        acc.y -= hv * v.y;
      }
      *reinterpret_cast<double2*>(w + r) = acc;
      nacc += acc.x * acc.x + acc.y * acc.y;
    } else {
      double acc = w[r];
      for (int i = 0; i < J; ++i) acc -= hs[i] * __ldcs(V + (size_t)i * ldv + r);
      w[r] = acc;
      nacc += acc * acc;
    }
  }
  if (nrm_partials) {
    nacc = block_sum(nacc, sh);
    if (threadIdx.x == 0) nrm_partials[blockIdx.x] = nacc;
  }
}

// Arnoldi defect: w = V_j - w over the block's chunk (j = *jcount), per-block sums of w^2.
__global__ void __launch_bounds__(kRedThreads) k_defect(int64_t n, const double* __restrict__ V, int64_t ldv,
                                                        const int* __restrict__ jcount, double* __restrict__ w,
                                                        double* __restrict__ partials) {
  dep_wait();
  __shared__ double sh[32];
  const double* vj = V + (size_t)(*jcount) * ldv;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double acc = 0.0;
  for (int64_t r = lo + threadIdx.x; r < hi; r += blockDim.x) {
    const double d = vj[r] - w[r];
    w[r] = d;
    acc = fma(d, d, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// A second Gram-Schmidt pass is needed when the first kept less than eta of the
// vector's norm (a: its partial sums of squares after the pass, b: before):
// flag[0] = 1 when it is not (the skip flag of the second pass), flag[1] += passes needed
__global__ void __launch_bounds__(kRedThreads) k_reorth_flag(const double* __restrict__ pa,
                                                             const double* __restrict__ pb, int np, double eta2,
                                                             int* __restrict__ flag) {
  dep_wait();
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) { a += pa[k]; b += pb[k]; }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    const int need = (a < eta2 * b) ? 1 : 0;
    flag[0] = 1 - need;
    flag[1] += need;
  }
}

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

template <class T>
void axpby(int64_t n, T a, const T* x, T b, T* y, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(k_axpby<T>, grid_for(n), kThreads, 0, s, n, a, x, b, y);
}
template <class T>
void axpbyz(int64_t n, T a, const T* x, T b, const T* y, T* z, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(k_axpbyz<T>, grid_for(n), kThreads, 0, s, n, a, x, b, y, z);
}
template <class T>
void vmul(int64_t n, const T* x, const T* w, T* y, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(k_vmul<T>, grid_for(n), kThreads, 0, s, n, x, w, y);
}
template <class T>
void vfma(int64_t n, const T* w, const T* x, T* y, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(k_vfma<T>, grid_for(n), kThreads, 0, s, n, w, x, y);
}
template <class Ti, class To>
void cast(int64_t n, const Ti* x, To* y, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(k_cast<Ti, To>, grid_for(n), kThreads, 0, s, n, x, y);
}
template <class T>
void dot_dev(int64_t n, const T* x, const T* y, double* partials, double* out, cudaStream_t s) {
  launch_k(k_dot_partial<T>, kRedBlocks, kRedThreads, 0, s, n, x, y, partials);
  launch_k(k_reduce_cols, 1, kRedThreads, 0, s, partials, kRedBlocks, (const int*)nullptr, 1, out, 0,
           (const int*)nullptr);
}
template <class T>
double dot_host(int64_t n, const T* x, const T* y, double* partials, double* out, cudaStream_t s) {
  dot_dev<T>(n, x, y, partials, out, s);
  double h = 0.0;
  FSI_CUDA(cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  return h;
}

void mdot(int64_t n, const double* V, int64_t ldv, const int* jcount, int joff, const double* w, double* partials,
          double* h, int maxcols, cudaStream_t s, const int* skip) {
  if (ldv % 2 == 0 && aligned16(V) && aligned16(w))
    launch_k(k_mdot_partial_v2, kRedBlocks, kRedThreads, 0, s, n, V, ldv, jcount, joff, w, partials, skip);
  else
    launch_k(k_mdot_partial, kRedBlocks, kRedThreads, 0, s, n, V, ldv, jcount, joff, w, partials, skip);
  launch_k(k_reduce_cols, maxcols, kRedThreads, 0, s, partials, kRedBlocks, jcount, joff, h, 0, skip);
}

void maxpy(int64_t n, const double* V, int64_t ldv, const int* jcount, int joff, const double* h, double sign,
           double* w, double* nrm_partials, int maxcols, cudaStream_t s, const int* skip) {
  if (maxcols > 0 && ldv % 2 == 0 && aligned16(V) && aligned16(w))
    launch_k(k_maxpy_v2, kRedBlocks, kRedThreads, sizeof(double) * maxcols, s, n, V, ldv, jcount, joff, h, sign, w,
             nrm_partials, skip);
  else
    launch_k(k_maxpy, kRedBlocks, kRedThreads, 0, s, n, V, ldv, jcount, joff, h, sign, w, nrm_partials, skip);
}

void finish_norm(const double* partials, double* out, cudaStream_t s) {
  launch_k(k_reduce_cols, 1, kRedThreads, 0, s, partials, kRedBlocks, (const int*)nullptr, 1, out, 1,
           (const int*)nullptr);
}

void arnoldi_defect(int64_t n, const double* V, int64_t ldv, const int* jcount, double* w, double* partials,
                    cudaStream_t s) {
  launch_k(k_defect, kRedBlocks, kRedThreads, 0, s, n, V, ldv, jcount, w, partials);
}

void reorth_flag(const double* after, const double* before, double eta, int* flag, cudaStream_t s) {
  launch_k(k_reorth_flag, 1, kRedThreads, 0, s, after, before, kRedBlocks, eta * eta, flag);
}

template void axpby<double>(int64_t, double, const double*, double, double*, cudaStream_t);
template void axpby<float>(int64_t, float, const float*, float, float*, cudaStream_t);
template void axpbyz<double>(int64_t, double, const double*, double, const double*, double*, cudaStream_t);
template void axpbyz<float>(int64_t, float, const float*, float, const float*, float*, cudaStream_t);
template void vmul<double>(int64_t, const double*, const double*, double*, cudaStream_t);
template void vmul<float>(int64_t, const float*, const float*, float*, cudaStream_t);
template void vfma<double>(int64_t, const double*, const double*, double*, cudaStream_t);
template void vfma<float>(int64_t, const float*, const float*, float*, cudaStream_t);
template void cast<double, float>(int64_t, const double*, float*, cudaStream_t);
template void cast<float, double>(int64_t, const float*, double*, cudaStream_t);
template void dot_dev<double>(int64_t, const double*, const double*, double*, double*, cudaStream_t);
template void dot_dev<float>(int64_t, const float*, const float*, double*, double*, cudaStream_t);
template double dot_host<double>(int64_t, const double*, const double*, double*, double*, cudaStream_t);
template double dot_host<float>(int64_t, const float*, const float*, double*, double*, cudaStream_t);

}  // namespace fsi

// The coarse end of a V-cycle in one launch.
//
// Levels whose matrices are small (a few MB) leave most of the GPU idle and
// cost a kernel launch per smoothing step, residual, restriction and
// prolongation.  Here every level from `first` down to the dense coarsest solve
// and back up runs inside one launch whose CTAs share the rows of each step and
// meet at a barrier between dependent steps: either one thread-block cluster
// (hardware cluster barrier), or a cooperative grid over half the GPU's
// co-resident CTAs (software grid barrier; half, so that the two concurrent
// sub-solve branches of Alg. 2 can both be resident).  The arithmetic is that of
// the per-level path (Chebyshev steps with the same coefficients, residual, R,
// coarsest dense solve, P correction); only the launch granularity differs.
//
// Memory ordering: vectors written in one step are read by other CTAs in the
// next.  Those loads go through L2 (ld.global.cg) after the barrier; read-only
// data (matrices, D^-1, the coarse inverse) uses the read-only path.  Every
// barrier sits in control flow that is uniform across the CTAs (loop bounds come
// from the plan).  The grid barrier's wait is bounded: a CTA that waits too long
// sets the run's error flag and leaves the kernel (the solve then reports the
// failure), so the kernel cannot hang.
#include "amg.cuh"
#include "spmv.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace fsi {

namespace {

template <class T>
__device__ __forceinline__ T ldv(const T* p) { return __ldcg(p); }

// Per-row group product over a BSR row with lanes `lane` of `tpr`; x read via L2.
template <class T, int BR, int BC>
__device__ __forceinline__ void row_prod(const CoarseMat& M, const T* x, int row, int lane, int tpr, T* acc) {
  const T* v = static_cast<const T*>(M.v);
  const int kb = __ldg(M.rp + row), ke = __ldg(M.rp + row + 1);
  for (int k = kb + lane; k < ke; k += tpr) {
    const int c = __ldg(M.ci + k);
    const T* xc = x + (size_t)c * BC;
    T xv[BC], blk[BR * BC];
#pragma unroll
    for (int j = 0; j < BC; ++j) xv[j] = ldv(xc + j);
    if constexpr (planar_blocks<T, BR, BC>()) {
      // planar FP32 3 x 3 blocks (see load_block in spmv.cuh)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        blk[t] = __ldg(v + 4 * (int64_t)k + t);
        blk[4 + t] = __ldg(v + 4 * M.nnzb + 4 * (int64_t)k + t);
      }
      blk[8] = __ldg(v + 8 * M.nnzb + k);
    } else {
#pragma unroll
      for (int t = 0; t < BR * BC; ++t) blk[t] = __ldg(v + (size_t)k * (BR * BC) + t);
    }
#pragma unroll
    for (int i = 0; i < BR; ++i)
#pragma unroll
      for (int j = 0; j < BC; ++j) acc[i] += blk[i * BC + j] * xv[j];
  }
}

enum StepKind { kCheb = 0, kResid = 1, kAxpy = 2 };

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Spins (with ~64 ns sleeps) a CTA waits at a grid barrier before it gives up.
constexpr unsigned kBarrierSpins = 1u << 22;

// Grid-wide barrier over `nblocks` co-resident CTAs: bar[0] counts arrivals,
// bar[1] is the generation the last arrival advances.  Returns false (in every
// thread of the CTA) when the wait gave up; err is then set.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* err, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = ld_acquire(bar + 1);
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned spins = 0;
      while (ld_acquire(bar + 1) == g) {
        if (++spins > kBarrierSpins) {
          ok = 0;
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// One pass over the rows of M: acc = M x, then per row
//   kCheb : r = dinv (b - acc); d = c1 d + c2 r; xo = xin + d   (xin = x, the gathered vector)
//   kResid: out = b - acc
//   kAxpy : out = alpha * acc + beta * out
template <class T, int BR, int BC>
__device__ void pass(const CoarseMat& M, const T* x, int kind, const T* b, const T* dinv, T* d, T* out, T c1, T c2,
                     T alpha, T beta, int gwarp, int nwarps, int lane32) {
  const int tpr = M.tpr;
  const int rows_per_warp = 32 / tpr;
  const int sub = lane32 / tpr, lane = lane32 & (tpr - 1);
  for (int row0 = gwarp * rows_per_warp; row0 < M.nbr; row0 += nwarps * rows_per_warp) {
    const int row = row0 + sub;
    const bool valid = row < M.nbr;
    T acc[BR];
#pragma unroll
    for (int i = 0; i < BR; ++i) acc[i] = T(0);
    if (valid) row_prod<T, BR, BC>(M, x, row, lane, tpr, acc);
    for (int off = tpr >> 1; off > 0; off >>= 1)
#pragma unroll
      for (int i = 0; i < BR; ++i) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], off, tpr);
    if (valid && lane == 0) {
#pragma unroll
      for (int i = 0; i < BR; ++i) {
        const size_t k = (size_t)row * BR + i;
        if (kind == kCheb) {
          const T r = __ldg(dinv + k) * (ldv(b + k) - acc[i]);
          T dn = c2 * r;
          if (c1 != T(0)) dn += c1 * ldv(d + k);
          d[k] = dn;
          out[k] = ldv(x + k) + dn;
        } else if (kind == kResid) {
          out[k] = ldv(b + k) - acc[i];
        } else {
          T v = alpha * acc[i];
          if (beta != T(0)) v += beta * ldv(out + k);
          out[k] = v;
        }
      }
    }
  }
}

template <class T>
__device__ void pass_any(const CoarseMat& M, const T* x, int kind, const T* b, const T* dinv, T* d, T* out, T c1,
                         T c2, T alpha, T beta, int gwarp, int nwarps, int lane32) {
#define FSI_P(a, c) if (M.br == a && M.bc == c) { pass<T, a, c>(M, x, kind, b, dinv, d, out, c1, c2, alpha, beta, gwarp, nwarps, lane32); return; }
  FSI_P(1, 1) FSI_P(2, 2) FSI_P(3, 3) FSI_P(6, 6) FSI_P(2, 3) FSI_P(3, 2) FSI_P(3, 6) FSI_P(6, 3)
#undef FSI_P
}

template <class T, bool GRID>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse_vcycle(const CoarsePlan* __restrict__ plan, const T* b0,
                                                                  T* x0, unsigned* bar, int* err, int extra) {
  __shared__ int s_ok;
  int nblk, rank;
  if constexpr (GRID) {
    nblk = (int)gridDim.x + extra;   // extra > 0 only under fault injection (tests)
    rank = (int)blockIdx.x;
  } else {
    cg::cluster_group cluster = cg::this_cluster();
    nblk = (int)cluster.num_blocks();
    rank = (int)cluster.block_rank();
  }
  auto sync = [&]() -> bool {
    if constexpr (GRID) {
      return grid_barrier(bar, (unsigned)nblk, err, &s_ok);
    } else {
      cg::this_cluster().sync();
      return true;
    }
  };
  const int lane32 = threadIdx.x & 31;
  const int gwarp = rank * (kCoarseThreads / 32) + (threadIdx.x >> 5);
  const int nwarps = nblk * (kCoarseThreads / 32);
  const int gtid = rank * kCoarseThreads + threadIdx.x;
  const int nth = nblk * kCoarseThreads;
  const int L = plan->nlev;
  // ------------------------------------------------ descend
  for (int li = 0; li + 1 < L; ++li) {
    const CoarseLevel& lv = plan->lev[li];
    const T* b = li == 0 ? b0 : static_cast<const T*>(lv.b);
    T* x = li == 0 ? x0 : static_cast<T*>(lv.x);
    T* xb = static_cast<T*>(lv.xb);
    T* d = static_cast<T*>(lv.d);
    const T* dinv = static_cast<const T*>(lv.dinv);
    const int n = lv.A.nbr * lv.A.br;
    const int deg = lv.deg;
    for (int sw = 0; sw < plan->presmooth; ++sw) {
      const bool zero = sw == 0;
      const int nsp = zero ? deg - 1 : deg;
      T* cur = x;
      T* oth = xb;
      if (zero) {
        T* first = (nsp % 2 == 0) ? x : xb;
        for (int i = gtid; i < n; i += nth) {
          const T v = __ldg(dinv + i) * ldv(b + i) * (T)lv.inv_theta;
          d[i] = v;
          first[i] = v;
        }
        cur = first;
        oth = (first == x) ? xb : x;
        if (!sync()) return;
      }
      for (int st = 0; st < nsp; ++st) {
        T c1, c2;
        if (!zero && st == 0) { c1 = T(0); c2 = (T)lv.inv_theta; }
        else { const int r = zero ? st : st - 1; c1 = (T)lv.c1[r]; c2 = (T)lv.c2[r]; }
        pass_any<T>(lv.A, cur, kCheb, b, dinv, d, oth, c1, c2, T(0), T(0), gwarp, nwarps, lane32);
        T* t = cur; cur = oth; oth = t;
        if (!sync()) return;
      }
      if (cur != x) {
        for (int i = gtid; i < n; i += nth) x[i] = ldv(cur + i);
        if (!sync()) return;
      }
    }
    pass_any<T>(lv.A, x, kResid, b, nullptr, nullptr, static_cast<T*>(lv.r), T(0), T(0), T(0), T(0), gwarp, nwarps,
                lane32);
    if (!sync()) return;
    pass_any<T>(lv.R, static_cast<const T*>(lv.r), kAxpy, nullptr, nullptr, nullptr,
                static_cast<T*>(plan->lev[li + 1].b), T(0), T(0), T(1), T(0), gwarp, nwarps, lane32);
    if (!sync()) return;
  }
  // ------------------------------------------------ coarsest: x = Cinv b
  {
    const CoarseLevel& lv = plan->lev[L - 1];
    const T* b = L == 1 ? b0 : static_cast<const T*>(lv.b);
    T* x = L == 1 ? x0 : static_cast<T*>(lv.x);
    const T* M = static_cast<const T*>(plan->cinv);
    const int nc = plan->ncoarse;
    for (int row = gwarp; row < nc; row += nwarps) {
      T acc = T(0);
      for (int c = lane32; c < nc; c += 32) acc += __ldg(M + (size_t)row * nc + c) * ldv(b + c);
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
      if (lane32 == 0) x[row] = acc;
    }
    if (!sync()) return;
  }
  // ------------------------------------------------ ascend
  for (int li = L - 2; li >= 0; --li) {
    const CoarseLevel& lv = plan->lev[li];
    const T* b = li == 0 ? b0 : static_cast<const T*>(lv.b);
    T* x = li == 0 ? x0 : static_cast<T*>(lv.x);
    T* xb = static_cast<T*>(lv.xb);
    T* d = static_cast<T*>(lv.d);
    const T* dinv = static_cast<const T*>(lv.dinv);
    const int n = lv.A.nbr * lv.A.br;
    const int deg = lv.deg;
    pass_any<T>(lv.P, static_cast<const T*>(plan->lev[li + 1].x), kAxpy, nullptr, nullptr, nullptr, x, T(0), T(0),
                T(1), T(1), gwarp, nwarps, lane32);
    if (!sync()) return;
    for (int sw = 0; sw < plan->postsmooth; ++sw) {
      T* cur = x;
      T* oth = xb;
      for (int st = 0; st < deg; ++st) {
        T c1, c2;
        if (st == 0) { c1 = T(0); c2 = (T)lv.inv_theta; }
        else { c1 = (T)lv.c1[st - 1]; c2 = (T)lv.c2[st - 1]; }
        pass_any<T>(lv.A, cur, kCheb, b, dinv, d, oth, c1, c2, T(0), T(0), gwarp, nwarps, lane32);
        T* t = cur; cur = oth; oth = t;
        if (!sync()) return;
      }
      if (cur != x) {
        for (int i = gtid; i < n; i += nth) x[i] = ldv(cur + i);
        if (!sync()) return;
      }
    }
  }
}

int lanes_for_rows(const Bsr& A, int threads) {
  const double mean = A.nbr ? (double)A.nnzb / A.nbr : 0.0;
  int t = 1;
  while (t < 32 && (double)A.nbr * t < threads && mean / (2 * t) >= 1.0) t *= 2;
  return t;
}

template <class T> const T* vals_of(const Bsr& A);
template <> const double* vals_of<double>(const Bsr& A) { return A.v64.p; }
template <> const float* vals_of<float>(const Bsr& A) { return A.v32.p; }

template <class T>
CoarseMat mat_of(const Bsr& A, int threads) {
  CoarseMat m;
  m.nbr = A.nbr; m.br = A.br; m.bc = A.bc; m.nnzb = A.nnzb;
  m.rp = A.rowptr.p; m.ci = A.colind.p; m.v = vals_of<T>(A);
  m.tpr = lanes_for_rows(A, threads);
  return m;
}

bool shape_ok(const Bsr& A) {
  const int a = A.br, c = A.bc;
  return (a == c && (a == 1 || a == 2 || a == 3 || a == 6)) || (a == 2 && c == 3) || (a == 3 && c == 2) ||
         (a == 3 && c == 6) || (a == 6 && c == 3);
}

template <class T>
void launch(const CoarseRun<T>& run, const T* b0, T* x0, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(run.ctas, 1, 1);
  cfg.blockDim = dim3(kCoarseThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (run.mode == COARSE_GRID) {
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
  } else {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = run.ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (run.mode == COARSE_GRID)
    FSI_CUDA(cudaLaunchKernelEx(&cfg, k_coarse_vcycle<T, true>, run.plan.p, b0, x0, run.bar.p, run.err.p,
                                (fault_inject() & kInjectCoarseBarrier) ? 1 : 0));
  else
    FSI_CUDA(cudaLaunchKernelEx(&cfg, k_coarse_vcycle<T, false>, run.plan.p, b0, x0, (unsigned*)nullptr,
                                (int*)nullptr, 0));
  ++g_kernel_launches;
}

// Cooperative grid: half of the CTAs the whole GPU holds at once (0 when none fit);
// found once per device.
template <class T>
int choose_grid() {
  static std::atomic<int> cached[64];
  static std::atomic<unsigned long long> done{0};
  once_per_device(done, [](int dev) {
    int nsm = 0, per_sm = 0, coop = 0;
    FSI_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FSI_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    FSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_vcycle<T, true>, kCoarseThreads, 0));
    cached[dev].store(coop ? (per_sm * nsm) / 2 : 0, std::memory_order_relaxed);
  });
  int dev = 0;
  FSI_CUDA(cudaGetDevice(&dev));
  return cached[dev].load(std::memory_order_relaxed);
}

template <class T>
int find_cluster();

// Cluster size of the one-launch coarse V-cycle: 16 (non-portable, which the kernel
// then allows on this device) or 8 when a cluster of that size fits, else 0; found
// once per device.
template <class T>
int choose_cluster() {
  static std::atomic<int> cached[64];
  static std::atomic<unsigned long long> done{0};
  once_per_device(done, [](int dev) { cached[dev].store(find_cluster<T>(), std::memory_order_relaxed); });
  int dev = 0;
  FSI_CUDA(cudaGetDevice(&dev));
  return cached[dev].load(std::memory_order_relaxed);
}

template <class T>
int find_cluster() {
  int best = 0;
  for (int c : {16, 8}) {
    if (c == 16 && cudaFuncSetAttribute(k_coarse_vcycle<T, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                       cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c, 1, 1);
    cfg.blockDim = dim3(kCoarseThreads, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_vcycle<T, false>, &cfg) == cudaSuccess && nclusters > 0) {
      best = c;
      break;
    }
    cudaGetLastError();
  }
  return best;
}

}  // namespace

template <class T>
void coarse_plan_build(Hierarchy& H, int first, CoarseRun<T>& run, cudaStream_t s) {
  run = CoarseRun<T>();
  const int L = (int)H.levels.size();
  require(first >= 0 && first < L, "coarse plan: bad first level");
  require(L - first <= kCoarseMaxLevels, "coarse plan: too many levels");
  run.mode = H.coarse_mode;
  run.ctas = run.mode == COARSE_GRID ? choose_grid<T>() : choose_cluster<T>();
  if (run.ctas == 0) return;             // no such launch possible: caller keeps the per-level path
  const int threads = run.ctas * kCoarseThreads;
  CoarsePlan p = {};
  p.nlev = L - first;
  p.presmooth = H.prm.presmooth;
  p.postsmooth = H.prm.postsmooth;
  for (int li = 0; li < p.nlev; ++li) {
    AmgLevel& Lv = H.levels[first + li];
    CoarseLevel& c = p.lev[li];
    const bool last = li + 1 == p.nlev;
    if (!last) {
      require(shape_ok(Lv.A) && shape_ok(Lv.P) && shape_ok(Lv.R), "coarse plan: unsupported block shape");
      c.A = mat_of<T>(Lv.A, threads);
      c.P = mat_of<T>(Lv.P, threads);
      c.R = mat_of<T>(Lv.R, threads);
    }
    LevelWork<T>& W = [&]() -> LevelWork<T>& {
      if constexpr (sizeof(T) == 8) return Lv.w64; else return Lv.w32;
    }();
    c.b = W.b.p; c.x = W.x.p; c.xb = W.xb.p; c.r = W.r.p; c.d = W.d.p;
    if constexpr (sizeof(T) == 8) c.dinv = Lv.dinv64.p; else c.dinv = Lv.dinv32.p;
    // Chebyshev coefficients of the level (Saad Alg. 12.1 recurrence)
    const double beta = H.prm.cheb_upper * Lv.lam, alpha = Lv.lam / H.prm.cheb_ratio;
    const double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha), sigma = theta / delta;
    double rho = 1.0 / sigma;
    c.inv_theta = 1.0 / theta;
    c.deg = H.prm.degree(first + li);
    require(c.deg >= 1 && c.deg - 1 <= kCoarseMaxDeg, "coarse plan: Chebyshev degree out of range");
    for (int k = 0; k + 1 < c.deg; ++k) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      c.c1[k] = rn * rho;
      c.c2[k] = 2.0 * rn / delta;
      rho = rn;
    }
  }
  if constexpr (sizeof(T) == 8) p.cinv = H.cinv64.p; else p.cinv = H.cinv32.p;
  p.ncoarse = H.ncoarse;
  run.plan.alloc(1);
  FSI_CUDA(cudaMemcpyAsync(run.plan.p, &p, sizeof(CoarsePlan), cudaMemcpyHostToDevice, s));
  if (run.mode == COARSE_GRID) {
    run.bar.alloc(2);
    run.err.alloc(1);
    FSI_CUDA(cudaMemsetAsync(run.bar.p, 0, 2 * sizeof(unsigned), s));
    FSI_CUDA(cudaMemsetAsync(run.err.p, 0, sizeof(int), s));
  }
  FSI_CUDA(cudaStreamSynchronize(s));
  run.first = first;
}

namespace {
template <class T>
bool run_failed(CoarseRun<T>& run, cudaStream_t s) {
  if (run.mode != COARSE_GRID || !run.err.p) return false;
  int h = 0;
  FSI_CUDA(cudaMemcpyAsync(&h, run.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  if (h == 0) return false;
  FSI_CUDA(cudaMemsetAsync(run.bar.p, 0, 2 * sizeof(unsigned), s));
  FSI_CUDA(cudaMemsetAsync(run.err.p, 0, sizeof(int), s));
  FSI_CUDA(cudaStreamSynchronize(s));
  return true;
}
}  // namespace

bool coarse_failed(Hierarchy& H, cudaStream_t s) {
  const bool a = run_failed(H.crun64, s);
  const bool b = run_failed(H.crun32, s);
  return a || b;
}

template <class T>
void coarse_vcycle(const CoarseRun<T>& run, const T* b, T* x, cudaStream_t s) {
  launch<T>(run, b, x, s);
}

template void coarse_plan_build<double>(Hierarchy&, int, CoarseRun<double>&, cudaStream_t);
template void coarse_plan_build<float>(Hierarchy&, int, CoarseRun<float>&, cudaStream_t);
template void coarse_vcycle<double>(const CoarseRun<double>&, const double*, double*, cudaStream_t);
template void coarse_vcycle<float>(const CoarseRun<float>&, const float*, float*, cudaStream_t);

}  // namespace fsi

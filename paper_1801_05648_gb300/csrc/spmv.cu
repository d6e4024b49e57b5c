// Host-side dispatch of the BSR SpMV kernels over the block shapes the solver
// uses: d x d vector blocks (d = 2, 3), the d x 1 / 1 x d velocity-pressure
// couplings, scalar blocks, and the k x k / b x k / k x b blocks of the AMG
// levels (k = 3 or 6 rigid-body modes for the solid block).
#include "spmv.cuh"

namespace fsi {

namespace {

// L2 prefetch per CTA and matrix: at most this many bytes from the head of its slice.
constexpr int kPrefetchCap = 32768;

// Staged 2 x 2 Chebyshev steps: at most this much dynamic shared memory per CTA.
constexpr int kStageSmemMax = 100 * 1024;

// Set by a staged kernel whose wait for its copies gave up (see spmv_stage_failed).
__device__ int g_stage_err = 0;

// The flag's device address on the current device (looked up once per device).
int* stage_err_ptr() {
  static std::atomic<int*> addr[64];
  static std::atomic<unsigned long long> done{0};
  once_per_device(done, [](int dev) {
    int* a = nullptr;
    FSI_CUDA(cudaGetSymbolAddress((void**)&a, g_stage_err));
    addr[dev].store(a, std::memory_order_relaxed);
  });
  int dev = 0;
  FSI_CUDA(cudaGetDevice(&dev));
  return addr[dev].load(std::memory_order_relaxed);
}

// Persistent grid of the staged kernel: up to eight 256-thread CTAs per SM (its
// register limit), fewer if shared memory runs out.
inline int staged_grid(int nchunks, int smax) {
  const size_t per_cta = staged_smem_bytes(smax) + 1024;
  int c = (int)((200 * 1024) / per_cta);
  c = c < 1 ? 1 : (c > 8 ? 8 : c);
  const int g = device_sms() * c;
  return nchunks < g ? nchunks : g;
}

template <class Epi, class G1, int UREQ>
void launch_staged(const Bsr& A1, const G1& g1, const Epi& epi, int tpr, int rows_per_cta, int nchunks, int grid,
                   int pre_wait, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};   // the opt-in above 48 KB, per instantiation and device
  once_per_device(attr, [](int) {
    FSI_CUDA(cudaFuncSetAttribute(k_bsr_cheb_staged<Epi, G1, UREQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kStageSmemMax));
  });
  launch_k(k_bsr_cheb_staged<Epi, G1, UREQ>, grid, 256, staged_smem_bytes(A1.stage_max), s, A1.nbr, tpr,
           rows_per_cta, nchunks, pre_wait, A1.rowptr.p, (const int16_t*)A1.cd16.p, A1.vals<float>(), g1, epi,
           A1.stage_max, stage_err_ptr());
}

// ALLOW16: the first matrix's 16-bit column offsets are read when present (FP32
// Chebyshev steps on the square level matrices).
template <class T, int BR, int BC1, int BC2, class Epi, class G1, bool ALLOW16 = false>
void launch_g(const Bsr& A1, const G1& g1, const Bsr* A2, const T* x2, const Epi& epi, cudaStream_t s) {
  if (A1.nbr == 0) return;
  const SpmvTuning& tu = spmv_tuning();
  int tpr = sizeof(T) == 8 ? A1.tpr64 : A1.tpr;
  if (sizeof(T) == 4) tpr = (tpr >> tu.lane_shift) > 0 ? (tpr >> tu.lane_shift) : 1;
  const int threads = 256;
  const int per_pass = threads / tpr;
  int rows_per_cta = per_pass;
  int blocks = div_up(A1.nbr, per_pass);
  if (tu.prefetch >= 2 && blocks > device_sms() * tu.ctas_per_sm) {
    // persistent: at most ctas_per_sm CTAs per SM, each over a longer contiguous slice
    const int passes = div_up(blocks, device_sms() * tu.ctas_per_sm);
    rows_per_cta = passes * per_pass;
    blocks = div_up(A1.nbr, rows_per_cta);
  }
  const T* v2 = nullptr; const int* rp2 = nullptr; const int* ci2 = nullptr;
  int64_t nnzb2 = 0;
  if (A2) { v2 = A2->vals<T>(); rp2 = A2->rowptr.p; ci2 = A2->colind.p; nnzb2 = A2->nnzb; }
  const int pre_wait = tu.setup_depth == 0 ? 1 : 0;
  const int pf = tu.prefetch > 0 ? kPrefetchCap : 0;
  const int4* ord2 = BC2 > 0 && tu.order && A2 && A1.ord2.p && A1.ord2_rp2 == A2->rowptr.p ? A1.ord2.p : nullptr;
  if constexpr (ALLOW16 && sizeof(T) == 4 && BC2 == 0) {
    if constexpr (BR == 2 && BC1 == 2) {
      // staged for matrices with at least two chunks per CTA of the persistent grid
      if (A1.cd16.p && tu.stage && A1.stage_rows == rows_per_cta && A1.stage_max > 0 &&
          staged_smem_bytes(A1.stage_max) <= (size_t)kStageSmemMax) {
        const int grid = staged_grid(blocks, A1.stage_max);
        if (blocks >= 2 * grid) {
          launch_staged<Epi, G1, 4>(A1, g1, epi, tpr, rows_per_cta, blocks, grid, pre_wait, s);
          return;
        }
      }
    }
    if (A1.cd16.p) {
      if (tu.unroll >= 8 && unroll_for<T, BR, BC1, 8>() == 8)
        launch_k(k_bsr_spmv<T, BR, BC1, BC2, Epi, G1, 8, int16_t>, blocks, threads, 0, s, A1.nbr, tpr, rows_per_cta,
                 pf, pre_wait, ord2, A1.rowptr.p, (const int16_t*)A1.cd16.p, A1.vals<T>(), A1.nnzb, g1, rp2, ci2, v2, nnzb2,
                 x2, epi);
      else
        launch_k(k_bsr_spmv<T, BR, BC1, BC2, Epi, G1, 4, int16_t>, blocks, threads, 0, s, A1.nbr, tpr, rows_per_cta,
                 pf, pre_wait, ord2, A1.rowptr.p, (const int16_t*)A1.cd16.p, A1.vals<T>(), A1.nnzb, g1, rp2, ci2, v2, nnzb2,
                 x2, epi);
      return;
    }
  }
  if (tu.unroll >= 8 && unroll_for<T, BR, BC1, 8>() == 8)
    launch_k(k_bsr_spmv<T, BR, BC1, BC2, Epi, G1, 8>, blocks, threads, 0, s, A1.nbr, tpr, rows_per_cta, pf, pre_wait,
             ord2, A1.rowptr.p, A1.colind.p, A1.vals<T>(), A1.nnzb, g1, rp2, ci2, v2, nnzb2, x2, epi);
  else
    launch_k(k_bsr_spmv<T, BR, BC1, BC2, Epi, G1, 4>, blocks, threads, 0, s, A1.nbr, tpr, rows_per_cta, pf, pre_wait,
             ord2, A1.rowptr.p, A1.colind.p, A1.vals<T>(), A1.nnzb, g1, rp2, ci2, v2, nnzb2, x2, epi);
}

template <class T, int BR, int BC1, int BC2, class Epi, bool ALLOW16 = false>
void launch(const Bsr& A1, const T* x1, const Bsr* A2, const T* x2, const Epi& epi, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    if (spmv_tuning().keep_x64) {
      launch_g<T, BR, BC1, BC2, Epi, GatherX<T, BC1, true>, ALLOW16>(A1, GatherX<T, BC1, true>{x1}, A2, x2, epi, s);
      return;
    }
  }
  launch_g<T, BR, BC1, BC2, Epi, GatherX<T, BC1>, ALLOW16>(A1, GatherX<T, BC1>{x1}, A2, x2, epi, s);
}

// Calls f.template operator()<BR, BC1, BC2>() for the runtime shape.
template <class F>
void dispatch(int br, int bc1, int bc2, F&& f) {
#define FSI_SHAPE(a, b, c) if (br == a && bc1 == b && bc2 == c) { f.template operator()<a, b, c>(); return; }
  FSI_SHAPE(1, 1, 0) FSI_SHAPE(2, 2, 0) FSI_SHAPE(3, 3, 0) FSI_SHAPE(6, 6, 0)
  FSI_SHAPE(2, 3, 0) FSI_SHAPE(3, 2, 0) FSI_SHAPE(3, 6, 0) FSI_SHAPE(6, 3, 0)
  FSI_SHAPE(2, 1, 0) FSI_SHAPE(3, 1, 0) FSI_SHAPE(1, 2, 0) FSI_SHAPE(1, 3, 0)
  FSI_SHAPE(2, 2, 1) FSI_SHAPE(3, 3, 1) FSI_SHAPE(1, 2, 1) FSI_SHAPE(1, 3, 1)
#undef FSI_SHAPE
  throw Error(EINVAL_, "unsupported BSR block shape " + std::to_string(br) + "x" + std::to_string(bc1) + "+" +
                           std::to_string(bc2));
}

inline void check_pair(const Bsr& A1, const Bsr* A2) {
  if (A2 && A2->nbr != 0)
    require(A2->nbr == A1.nbr && A2->br == A1.br, "fused SpMV: matrices with different block rows");
}

}  // namespace

bool spmv_stage_failed(cudaStream_t s) {
  int h = 0;
  FSI_CUDA(cudaMemcpyAsync(&h, stage_err_ptr(), sizeof(int), cudaMemcpyDeviceToHost, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  if (h) FSI_CUDA(cudaMemsetAsync(stage_err_ptr(), 0, sizeof(int), s));
  return h != 0;
}

template <class T>
void spmv_axpby(const Bsr& A, const T* x, T alpha, T beta, T* y, cudaStream_t s) {
  dispatch(A.br, A.bc, 0, [&]<int BR, int BC1, int BC2>() {
    launch<T, BR, BC1, 0>(A, x, nullptr, nullptr, EpiAxpby<T, BR>{y, alpha, beta}, s);
  });
}

template <class T>
void spmv2_axpby(const Bsr& A1, const T* x1, const Bsr* A2, const T* x2, T alpha, T beta, T* y, cudaStream_t s) {
  if (A2 && A2->nbr == 0) A2 = nullptr;
  check_pair(A1, A2);
  dispatch(A1.br, A1.bc, A2 ? A2->bc : 0, [&]<int BR, int BC1, int BC2>() {
    launch<T, BR, BC1, BC2>(A1, x1, A2, x2, EpiAxpby<T, BR>{y, alpha, beta}, s);
  });
}

template <class T>
void spmv2_resid(const Bsr& A1, const T* x1, const Bsr* A2, const T* x2, const T* b, T* r, cudaStream_t s) {
  if (A2 && A2->nbr == 0) A2 = nullptr;
  check_pair(A1, A2);
  dispatch(A1.br, A1.bc, A2 ? A2->bc : 0, [&]<int BR, int BC1, int BC2>() {
    launch<T, BR, BC1, BC2>(A1, x1, A2, x2, EpiResid<T, BR>{b, r}, s);
  });
}

template <class T>
void spmv_restrict(const Bsr& R, const T* b, const Bsr& RAn, const T* x, T* y, cudaStream_t s) {
  require(RAn.nbr == R.nbr && RAn.br == R.br && RAn.bc == R.bc, "spmv_restrict: R and -(R A) shapes differ");
  // coarse block k x fine block b: translations (k = b = 1, 2, 3), rigid-body modes
  // on the first solid level (3 x 2, 6 x 3) and below it (3 x 3, 6 x 6)
  // RAn leads (its lane count is set from both matrices' row lengths), R b follows
  auto run = [&]<int BR, int BC>() {
    launch<T, BR, BC, BC>(RAn, x, &R, b, EpiAxpby<T, BR>{y, T(1), T(0)}, s);
  };
  const int br = R.br, bc = R.bc;
  if (br == 1 && bc == 1) run.template operator()<1, 1>();
  else if (br == 2 && bc == 2) run.template operator()<2, 2>();
  else if (br == 3 && bc == 3) run.template operator()<3, 3>();
  else if (br == 6 && bc == 6) run.template operator()<6, 6>();
  else if (br == 3 && bc == 2) run.template operator()<3, 2>();
  else if (br == 6 && bc == 3) run.template operator()<6, 3>();
  else throw Error(EINVAL_, "spmv_restrict: unsupported block shape " + std::to_string(br) + "x" + std::to_string(bc));
}

template <class T>
void spmv_cheb(const Bsr& A, const T* x, const T* b, const T* dinv, T* d, T* xo, T c1, T c2, cudaStream_t s) {
  require(A.br == A.bc, "spmv_cheb: square blocks only");
  dispatch(A.br, A.bc, 0, [&]<int BR, int BC1, int BC2>() {
    if constexpr (BR == BC1)
      launch<T, BR, BC1, 0, EpiCheb<T, BR>, true>(A, x, nullptr, nullptr, EpiCheb<T, BR>{b, dinv, x, d, xo, c1, c2}, s);
  });
}

template <class T>
void spmv_dinv(const Bsr& A, const T* x, const T* dinv, T* y, cudaStream_t s) {
  dispatch(A.br, A.bc, 0, [&]<int BR, int BC1, int BC2>() {
    launch<T, BR, BC1, 0>(A, x, nullptr, nullptr, EpiDinv<T, BR>{dinv, y}, s);
  });
}

template <class T>
void spmv_cheb_from_zero(const Bsr& A, const T* b, const T* dinv, T* d, T* xo, T inv_theta, T c1, T c2,
                         cudaStream_t s) {
  require(A.br == A.bc, "spmv_cheb_from_zero: square blocks only");
  dispatch(A.br, A.bc, 0, [&]<int BR, int BC1, int BC2>() {
    if constexpr (BR == BC1) {
      launch_g<T, BR, BC1, 0, EpiChebFromZero<T, BR>, GatherScaled<T, BC1>, true>(
          A, GatherScaled<T, BC1>{b, dinv, inv_theta}, nullptr, (const T*)nullptr,
          EpiChebFromZero<T, BR>{b, dinv, d, xo, inv_theta, c1, c2}, s);
    }
  });
}

#define FSI_INST(T)                                                                                         \
  template void spmv_axpby<T>(const Bsr&, const T*, T, T, T*, cudaStream_t);                                \
  template void spmv2_axpby<T>(const Bsr&, const T*, const Bsr*, const T*, T, T, T*, cudaStream_t);         \
  template void spmv2_resid<T>(const Bsr&, const T*, const Bsr*, const T*, const T*, T*, cudaStream_t);     \
  template void spmv_cheb<T>(const Bsr&, const T*, const T*, const T*, T*, T*, T, T, cudaStream_t);         \
  template void spmv_restrict<T>(const Bsr&, const T*, const Bsr&, const T*, T*, cudaStream_t);             \
  template void spmv_dinv<T>(const Bsr&, const T*, const T*, T*, cudaStream_t);                             \
  template void spmv_cheb_from_zero<T>(const Bsr&, const T*, const T*, T*, T*, T, T, T, cudaStream_t);
FSI_INST(double)
FSI_INST(float)
#undef FSI_INST

}  // namespace fsi

#include "amg.cuh"
#include "spmv.cuh"
#include "sparse_util.cuh"
#include "vec.cuh"

#include <cmath>

namespace fsi {

namespace {

constexpr int kIdxBits = 27;
constexpr int kStateShift = 59;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int lbound(const int* a, int lo, int hi, int key) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Frobenius norm per block: squares summed in row-major order, no FMA contraction.
__global__ void k_block_fro(int64_t nnzb, int bsz, const double* __restrict__ v, double* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnzb) return;
  const double* p = v + k * bsz;
  double s = __dmul_rn(p[0], p[0]);
  for (int t = 1; t < bsz; ++t) s = __dadd_rn(s, __dmul_rn(p[t], p[t]));
  out[k] = __dsqrt_rn(s);
}

__device__ __forceinline__ double block_norm_at(const int* rp, const int* ci, const double* fro, int row, int col) {
  const int pos = lbound(ci, rp[row], rp[row + 1], col);
  return (pos < rp[row + 1] && ci[pos] == col) ? fro[pos] : 0.0;
}

template <bool FILL>
__global__ void k_strength(int nbr, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ fro, double theta, int* __restrict__ cnt,
                           const int* __restrict__ grp, int* __restrict__ gci) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  const double dii = block_norm_at(rp, ci, fro, i, i);
  int c = 0;
  int pos = FILL ? grp[i] : 0;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = ci[k];
    if (j == i) continue;
    const double fij = fro[k];
    const double fji = block_norm_at(rp, ci, fro, j, i);
    const double djj = block_norm_at(rp, ci, fro, j, j);
    const double m = fij > fji ? fij : fji;
    const double thr = __dmul_rn(theta, __dsqrt_rn(__dmul_rn(dii, djj)));
    if (m > 0.0 && m >= thr) {
      if (FILL) gci[pos++] = j;
      ++c;
    }
  }
  if (!FILL) cnt[i] = c;
}

__global__ void k_mis_init(int n, const int* __restrict__ grp, int level, int* __restrict__ state,
                           long long* __restrict__ base) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long pr = splitmix64((unsigned long long)i + ((unsigned long long)level << 32)) >> 32;
  base[i] = (long long)((pr << kIdxBits) | (unsigned long long)i);
  state[i] = (grp[i + 1] == grp[i]) ? 0 : 1;
}

__global__ void k_mis_key(int n, const int* __restrict__ state, const long long* __restrict__ base,
                          long long* __restrict__ key) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = ((long long)state[i] << kStateShift) | base[i];
}

// out[i] = max(in[i], max over strong neighbours j of in[j])
__global__ void k_rowmax(int n, const int* __restrict__ grp, const int* __restrict__ gci,
                         const long long* __restrict__ in, long long* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long m = in[i];
  for (int k = grp[i]; k < grp[i + 1]; ++k) {
    const long long v = in[gci[k]];
    if (v > m) m = v;
  }
  out[i] = m;
}

__global__ void k_mis_update(int n, int* __restrict__ state, const long long* __restrict__ key,
                             const long long* __restrict__ t2, int* __restrict__ undecided) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int still = 0;
  if (i < n && state[i] == 1) {
    if (t2[i] == key[i]) state[i] = 2;
    else if ((t2[i] >> kStateShift) == 2) state[i] = 0;
    else still = 1;
  }
  still = __syncthreads_count(still);
  if (threadIdx.x == 0 && still) atomicAdd(undecided, still);
}

__global__ void k_root_flag(int n, const int* __restrict__ state, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = state[i] == 2 ? 1 : 0;
}

__global__ void k_agg_roots(int n, const int* __restrict__ state, const int* __restrict__ rid, int* __restrict__ agg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) agg[i] = state[i] == 2 ? rid[i] : -1;
}

__global__ void k_agg_phase1(int n, const int* __restrict__ grp, const int* __restrict__ gci,
                             const int* __restrict__ state, int* __restrict__ agg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || state[i] == 2) return;
  for (int k = grp[i]; k < grp[i + 1]; ++k) {
    const int j = gci[k];
    if (state[j] == 2) { agg[i] = agg[j]; return; }
  }
}

__global__ void k_agg_phase2(int n, const int* __restrict__ grp, const int* __restrict__ gci,
                             const long long* __restrict__ base, const int* __restrict__ agg1, int* __restrict__ agg2,
                             int* __restrict__ fail) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = agg1[i];
  if (a < 0 && grp[i + 1] > grp[i]) {
    long long best = -1;
    for (int k = grp[i]; k < grp[i + 1]; ++k) {
      const int j = gci[k];
      if (agg1[j] >= 0 && base[j] > best) best = base[j];
    }
    if (best < 0) atomicExch(fail, 1);
    else a = agg1[(int)(best & ((1ll << kIdxBits) - 1))];
  }
  agg2[i] = a;
}

__global__ void k_count_agg(int n, const int* __restrict__ agg, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) atomicAdd(cnt + agg[i], 1);
}
__global__ void k_fill_members(int n, const int* __restrict__ agg, const int* __restrict__ off, int* __restrict__ cur,
                               int* __restrict__ mem) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) mem[off[agg[i]] + atomicAdd(cur + agg[i], 1)] = i;
}
__global__ void k_has_agg(int n, const int* __restrict__ agg, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = agg[i] >= 0 ? 1 : 0;
}
__global__ void k_ptent_cols(int n, const int* __restrict__ agg, const int* __restrict__ prp, int* __restrict__ pci) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) pci[prp[i]] = agg[i];
}

// One thread per aggregate: modified Gram-Schmidt on the near-nullspace rows of
// its members, Q written into P_tent's blocks, R into the coarse near-nullspace.
__global__ void k_tentative(int nagg, int b, int k, const int* __restrict__ off, const int* __restrict__ mem,
                            const int* __restrict__ prp, const double* __restrict__ B, double drop_tol,
                            double* __restrict__ Q, double* __restrict__ Bc) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= nagg) return;
  const int lo = off[J], hi = off[J + 1];
  for (int e = lo; e < hi; ++e) {
    const int m = mem[e];
    for (int r = 0; r < b; ++r)
      for (int c = 0; c < k; ++c) Q[((int64_t)prp[m] * b + r) * k + c] = B[((int64_t)m * b + r) * k + c];
  }
  double* R = Bc + (int64_t)J * k * k;
  for (int t = 0; t < k * k; ++t) R[t] = 0.0;
  for (int c = 0; c < k; ++c) {
    double s = 0.0;
    for (int e = lo; e < hi; ++e)
      for (int r = 0; r < b; ++r) { const double q = Q[((int64_t)prp[mem[e]] * b + r) * k + c]; s += q * q; }
    const double orig = sqrt(s);
    for (int j = 0; j < c; ++j) {
      double rjc = 0.0;
      for (int e = lo; e < hi; ++e)
        for (int r = 0; r < b; ++r) {
          const int64_t row = ((int64_t)prp[mem[e]] * b + r) * k;
          rjc += Q[row + j] * Q[row + c];
        }
      R[j * k + c] = rjc;
      for (int e = lo; e < hi; ++e)
        for (int r = 0; r < b; ++r) {
          const int64_t row = ((int64_t)prp[mem[e]] * b + r) * k;
          Q[row + c] = Q[row + c] - rjc * Q[row + j];
        }
    }
    s = 0.0;
    for (int e = lo; e < hi; ++e)
      for (int r = 0; r < b; ++r) { const double q = Q[((int64_t)prp[mem[e]] * b + r) * k + c]; s += q * q; }
    const double nrm = sqrt(s);
    const bool drop = (orig == 0.0) || (nrm <= drop_tol * orig);
    for (int e = lo; e < hi; ++e)
      for (int r = 0; r < b; ++r) {
        const int64_t row = ((int64_t)prp[mem[e]] * b + r) * k;
        Q[row + c] = drop ? 0.0 : Q[row + c] / nrm;
      }
    R[c * k + c] = drop ? 0.0 : nrm;
  }
}

// P = P_tent - (omega * dinv) * AP on the pattern of AP (which contains P_tent's).
__global__ void k_smooth_p(int nbr, int b, int k, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ ap, const int* __restrict__ agg, const int* __restrict__ prp,
                           const double* __restrict__ Q, const double* __restrict__ dinv, double omega,
                           double* __restrict__ p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const bool tent = agg[i] >= 0 && ci[e] == agg[i];
    for (int r = 0; r < b; ++r) {
      const double w = omega * dinv[(int64_t)i * b + r];
      for (int c = 0; c < k; ++c) {
        const int64_t o = ((int64_t)e * b + r) * k + c;
        const double t = tent ? Q[((int64_t)prp[i] * b + r) * k + c] : 0.0;
        p[o] = t - w * ap[o];
      }
    }
  }
}

__global__ void k_power_init(int64_t n, int stream_id, double* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long z = splitmix64((unsigned long long)i + ((unsigned long long)stream_id << 32));
  x[i] = 1.0 + (double)(z >> 11) * 0x1.0p-53;
}

// d = dinv * b / theta; x = d   (first Chebyshev step from x = 0)
template <class T>
__global__ void k_cheb_first(int64_t n, const T* __restrict__ b, const T* __restrict__ dinv, T inv_theta,
                             T* __restrict__ d, T* __restrict__ x) {
  dep_wait();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T v = dinv[i] * b[i] * inv_theta;
  d[i] = v;
  x[i] = v;
}

// x = M b, M dense row-major n x n; one warp per row
template <class T>
__global__ void k_dense_gemv(int n, const T* __restrict__ M, const T* __restrict__ b, T* __restrict__ x) {
  dep_wait();
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  T acc = 0;
  for (int c = lane; c < n; c += 32) acc += M[(int64_t)row * n + c] * b[c];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) x[row] = acc;
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

template <class T> LevelWork<T>& work(AmgLevel& L);
template <> LevelWork<double>& work<double>(AmgLevel& L) { return L.w64; }
template <> LevelWork<float>& work<float>(AmgLevel& L) { return L.w32; }
template <class T> const T* dinv_of(const AmgLevel& L);
template <> const double* dinv_of<double>(const AmgLevel& L) { return L.dinv64.p; }
template <> const float* dinv_of<float>(const AmgLevel& L) { return L.dinv32.p; }
template <class T> const T* cinv_of(const Hierarchy& H);
template <> const double* cinv_of<double>(const Hierarchy& H) { return H.cinv64.p; }
template <> const float* cinv_of<float>(const Hierarchy& H) { return H.cinv32.p; }

template <class T>
void alloc_work(LevelWork<T>& W, int64_t n) {
  W.b.alloc(n); W.x.alloc(n); W.xb.alloc(n); W.r.alloc(n); W.d.alloc(n);
}

void to_f32(const double* a, DBuf<float>& b, int64_t n, cudaStream_t s) {
  b.alloc(n > 0 ? n : 1);
  if (n > 0) {
    k_f64_to_f32<<<div_up(n, 256), 256, 0, s>>>(n, a, b.p);
    FSI_CHECK_LAUNCH();
  }
}

// One Chebyshev sweep of `deg` steps (Saad Alg. 12.1) on D^-1 A over
// [lam/ratio, upper*lam]; the result ends in x (xb is the ping-pong buffer).
template <class T>
void cheb_sweep(const Bsr& A, const T* dinv, double lam, int deg, double ratio, double upper, const T* b, T* x, T* xb,
                T* d, bool zero_start, cudaStream_t s) {
  const int64_t n = A.rows();
  const double beta = upper * lam, alpha = lam / ratio;
  const double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const int nsp = zero_start ? deg - 1 : deg;
  T* cur;
  T* oth;
  int step0 = 0;
  if (zero_start && nsp >= 1) {
    // steps 1 and 2 in one pass: the first iterate dinv b / theta is gathered on the fly
    T* first = ((nsp - 1) % 2 == 0) ? x : xb;
    const double rn = 1.0 / (2.0 * sigma - rho);
    spmv_cheb_from_zero<T>(A, b, dinv, d, first, (T)(1.0 / theta), (T)(rn * rho), (T)(2.0 * rn / delta), s);
    rho = rn;
    cur = first;
    oth = (first == x) ? xb : x;
    step0 = 1;
  } else if (zero_start) {
    launch_k(k_cheb_first<T>, div_up(n, 256), 256, 0, s, n, b, dinv, (T)(1.0 / theta), d, x);
    cur = x;
    oth = xb;
  } else {
    cur = x;
    oth = xb;
  }
  for (int step = step0; step < nsp; ++step) {
    double c1, c2;
    if (!zero_start && step == 0) {
      c1 = 0.0; c2 = 1.0 / theta;
    } else {
      const double rn = 1.0 / (2.0 * sigma - rho);
      c1 = rn * rho; c2 = 2.0 * rn / delta;
      rho = rn;
    }
    spmv_cheb<T>(A, cur, b, dinv, d, oth, (T)c1, (T)c2, s);
    T* t = cur; cur = oth; oth = t;
  }
  if (cur != x) FSI_CUDA(cudaMemcpyAsync(x, cur, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
}

template <class T>
void vcycle_level(Hierarchy& H, int l, const T* b, T* x, cudaStream_t s) {
  const int last = (int)H.levels.size() - 1;
  if (l == last) {
    const int n = H.ncoarse;
    if (n == 0) return;
    launch_k(k_dense_gemv<T>, div_up((int64_t)n * 32, 256), 256, 0, s, n, cinv_of<T>(H), b, x);
    return;
  }
  {
    const CoarseRun<T>& run = [&]() -> const CoarseRun<T>& {
      if constexpr (sizeof(T) == 8) return H.crun64; else return H.crun32;
    }();
    if (H.coarse_mode != COARSE_PER_LEVEL && run.first == l && run.ctas > 0) {
      coarse_vcycle<T>(run, b, x, s);
      return;
    }
  }
  AmgLevel& L = H.levels[l];
  LevelWork<T>& W = work<T>(L);
  const AmgParams& p = H.prm;
  for (int sw = 0; sw < p.presmooth; ++sw)
    cheb_sweep<T>(L.A, dinv_of<T>(L), L.lam, p.degree(l), p.cheb_ratio, p.cheb_upper, b, x, W.xb.p, W.d.p, sw == 0, s);
  AmgLevel& C = H.levels[l + 1];
  LevelWork<T>& WC = work<T>(C);
  if (L.RAn.nbr) {
    spmv_restrict<T>(L.R, b, L.RAn, x, WC.b.p, s);                 // b_c = R b - (R A) x = R (b - A x)
  } else {
    spmv2_resid<T>(L.A, x, nullptr, nullptr, b, W.r.p, s);         // r = b - A x
    spmv_axpby<T>(L.R, W.r.p, T(1), T(0), WC.b.p, s);              // b_c = R r
  }
  vcycle_level<T>(H, l + 1, WC.b.p, WC.x.p, s);
  spmv_axpby<T>(L.P, WC.x.p, T(1), T(1), x, s);
  for (int sw = 0; sw < p.postsmooth; ++sw)
    cheb_sweep<T>(L.A, dinv_of<T>(L), L.lam, p.degree(l), p.cheb_ratio, p.cheb_upper, b, x, W.xb.p, W.d.p, false, s);
}

int sync_read_int(const int* dev, cudaStream_t s) {
  int h = 0;
  FSI_CUDA(cudaMemcpyAsync(&h, dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  return h;
}

}  // namespace

double power_lambda(const Bsr& A, const double* dinv, int iters, int stream_id, cudaStream_t s) {
  const int64_t n = A.rows();
  if (n == 0) return 0.0;
  DBuf<double> x(n), y(n), part(kRedBlocks), out(1);
  k_power_init<<<div_up(n, 256), 256, 0, s>>>(n, stream_id, x.p);
  FSI_CHECK_LAUNCH();
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    spmv_dinv<double>(A, x.p, dinv, y.p, s);
    const double ny = std::sqrt(dot_host<double>(n, y.p, y.p, part.p, out.p, s));
    const double nx = std::sqrt(dot_host<double>(n, x.p, x.p, part.p, out.p, s));
    lam = ny / nx;
    if (ny == 0.0) break;
    axpby<double>(n, 1.0 / ny, y.p, 0.0, x.p, s);
  }
  return lam;
}

double Hierarchy::operator_complexity() const {
  if (levels.empty()) return 0.0;
  double tot = 0.0;
  for (auto& L : levels) tot += (double)L.A.nnzb * L.A.br * L.A.bc;
  return tot / ((double)levels[0].A.nnzb * levels[0].A.br * levels[0].A.bc);
}

double Hierarchy::vcycle_bytes(int vb) const {
  double tot = 0.0;
  const int nl = (int)levels.size();
  for (int l = 0; l + 1 < nl; ++l) {
    const AmgLevel& L = levels[l];
    // smoother SpMVs (the first two steps from zero share one pass), the restricted
    // residual R b + RAn x (one pass over both, one output) and the prolongation
    const int sweeps = prm.presmooth * prm.degree(l) - 1 + prm.postsmooth * prm.degree(l);
    tot += sweeps * L.A.spmv_bytes(vb) + L.P.spmv_bytes(vb);
    if (L.RAn.nbr)
      tot += L.R.spmv_bytes(vb) + L.RAn.spmv_bytes(vb) - (double)vb * L.R.rows();
    else
      tot += L.A.spmv_bytes(vb) + (double)vb * L.A.rows() + L.R.spmv_bytes(vb);
  }
  tot += (double)ncoarse * ncoarse * vb;
  return tot;
}

void amg_setup(Hierarchy& H, Bsr&& A0, const double* B0, int k0, const AmgParams& prm, cudaStream_t s) {
  require(A0.br == A0.bc && A0.nbr == A0.nbc, "amg_setup: square matrix with square blocks required");
  H.levels.clear();
  H.prm = prm;
  if (A0.nbr == 0) {   // empty block (e.g. no solid): a single empty level, nothing to solve
    H.levels.emplace_back();
    H.levels.back().A = std::move(A0);
    H.ncoarse = 0;
    H.cinv64.alloc(1);
    return;
  }
  DBuf<double> Bcur;
  const double* B = B0;
  int k = k0;
  Bsr A = std::move(A0);
  for (int lvl = 0;; ++lvl) {
    H.levels.emplace_back();
    AmgLevel& L = H.levels.back();
    L.A = std::move(A);
    const int b = L.A.br;
    const int nbr = L.A.nbr;
    const int64_t n = L.A.rows();
    DBuf<double> diag(n > 0 ? n : 1);
    L.dinv64.alloc(n > 0 ? n : 1);
    bsr_point_diagonal(L.A, diag.p, s);
    invert_nonzero(n, diag.p, L.dinv64.p, s);
    L.lam = power_lambda(L.A, L.dinv64.p, prm.power_iters, 256 + lvl, s);
    alloc_work(L.w64, n);
    if (n <= prm.coarse_max || lvl + 1 >= prm.max_levels) break;
    require(nbr < (1 << kIdxBits), "amg_setup: too many nodes for the aggregation key");
    // ---- strength graph
    DBuf<double> fro(L.A.nnzb > 0 ? L.A.nnzb : 1);
    if (L.A.nnzb > 0) {
      k_block_fro<<<div_up(L.A.nnzb, 256), 256, 0, s>>>(L.A.nnzb, b * b, L.A.v64.p, fro.p);
      FSI_CHECK_LAUNCH();
    }
    DBuf<int> gcnt(nbr), grp(nbr + 1);
    k_strength<false><<<div_up(nbr, 128), 128, 0, s>>>(nbr, L.A.rowptr.p, L.A.colind.p, fro.p, prm.theta, gcnt.p,
                                                      nullptr, nullptr);
    FSI_CHECK_LAUNCH();
    const int64_t gnnz = exclusive_scan(gcnt.p, grp.p, nbr, s);
    DBuf<int> gci(gnnz > 0 ? gnnz : 1);
    k_strength<true><<<div_up(nbr, 128), 128, 0, s>>>(nbr, L.A.rowptr.p, L.A.colind.p, fro.p, prm.theta, nullptr,
                                                     grp.p, gci.p);
    FSI_CHECK_LAUNCH();
    // ---- distance-2 MIS
    DBuf<int> state(nbr), und(1);
    DBuf<long long> base(nbr), key(nbr), t1(nbr), t2(nbr);
    const int g = div_up(nbr, 256);
    k_mis_init<<<g, 256, 0, s>>>(nbr, grp.p, lvl, state.p, base.p);
    FSI_CHECK_LAUNCH();
    for (int it = 0;; ++it) {
      require(it < 10000, "amg_setup: MIS iteration did not terminate");
      FSI_CUDA(cudaMemsetAsync(und.p, 0, sizeof(int), s));
      k_mis_key<<<g, 256, 0, s>>>(nbr, state.p, base.p, key.p);
      k_rowmax<<<g, 256, 0, s>>>(nbr, grp.p, gci.p, key.p, t1.p);
      k_rowmax<<<g, 256, 0, s>>>(nbr, grp.p, gci.p, t1.p, t2.p);
      k_mis_update<<<g, 256, 0, s>>>(nbr, state.p, key.p, t2.p, und.p);
      FSI_CHECK_LAUNCH();
      if (sync_read_int(und.p, s) == 0) break;
    }
    // ---- aggregates
    DBuf<int> flag(nbr), rid(nbr + 1), agg1(nbr), fail(1);
    L.agg.alloc(nbr);
    k_root_flag<<<g, 256, 0, s>>>(nbr, state.p, flag.p);
    FSI_CHECK_LAUNCH();
    const int nagg = (int)exclusive_scan(flag.p, rid.p, nbr, s);
    k_agg_roots<<<g, 256, 0, s>>>(nbr, state.p, rid.p, agg1.p);
    k_agg_phase1<<<g, 256, 0, s>>>(nbr, grp.p, gci.p, state.p, agg1.p);
    FSI_CUDA(cudaMemsetAsync(fail.p, 0, sizeof(int), s));
    k_agg_phase2<<<g, 256, 0, s>>>(nbr, grp.p, gci.p, base.p, agg1.p, L.agg.p, fail.p);
    FSI_CHECK_LAUNCH();
    require(sync_read_int(fail.p, s) == 0, "amg_setup: aggregation left a node without an aggregated neighbour");
    L.nagg = nagg;
    if (nagg == 0 || (int64_t)nagg * k >= n) break;   // coarsening stalled: this level is the coarsest
    // ---- member lists (sorted by node index)
    DBuf<int> acnt(nagg), aoff(nagg + 1), acur(nagg), mem(nbr);
    FSI_CUDA(cudaMemsetAsync(acnt.p, 0, sizeof(int) * nagg, s));
    FSI_CUDA(cudaMemsetAsync(acur.p, 0, sizeof(int) * nagg, s));
    k_count_agg<<<g, 256, 0, s>>>(nbr, L.agg.p, acnt.p);
    FSI_CHECK_LAUNCH();
    exclusive_scan(acnt.p, aoff.p, nagg, s);
    k_fill_members<<<g, 256, 0, s>>>(nbr, L.agg.p, aoff.p, acur.p, mem.p);
    FSI_CHECK_LAUNCH();
    sort_segments(nagg, aoff.p, mem.p, nullptr, s);
    // ---- tentative prolongator
    Bsr Pt;
    Pt.nbr = nbr; Pt.nbc = nagg; Pt.br = b; Pt.bc = k;
    Pt.rowptr.alloc(nbr + 1);
    k_has_agg<<<g, 256, 0, s>>>(nbr, L.agg.p, flag.p);
    FSI_CHECK_LAUNCH();
    Pt.nnzb = exclusive_scan(flag.p, Pt.rowptr.p, nbr, s);
    Pt.colind.alloc(Pt.nnzb > 0 ? Pt.nnzb : 1);
    Pt.v64.alloc(Pt.nnzb > 0 ? Pt.nnzb * b * k : 1);
    k_ptent_cols<<<g, 256, 0, s>>>(nbr, L.agg.p, Pt.rowptr.p, Pt.colind.p);
    FSI_CHECK_LAUNCH();
    DBuf<double> Bc((int64_t)nagg * k * k);
    k_tentative<<<div_up(nagg, 64), 64, 0, s>>>(nagg, b, k, aoff.p, mem.p, Pt.rowptr.p, B, prm.drop_tol, Pt.v64.p,
                                                Bc.p);
    FSI_CHECK_LAUNCH();
    set_tpr(Pt);
    // ---- smoothed prolongator
    const double omega = 4.0 / (3.0 * L.lam);
    Bsr AP;
    bsr_spgemm(L.A, Pt, AP, s);
    L.P.nbr = AP.nbr; L.P.nbc = AP.nbc; L.P.br = AP.br; L.P.bc = AP.bc; L.P.nnzb = AP.nnzb;
    L.P.rowptr = std::move(AP.rowptr);
    L.P.colind = std::move(AP.colind);
    L.P.v64.alloc(AP.nnzb > 0 ? AP.nnzb * b * k : 1);
    k_smooth_p<<<div_up(nbr, 128), 128, 0, s>>>(nbr, b, k, L.P.rowptr.p, L.P.colind.p, AP.v64.p, L.agg.p,
                                                Pt.rowptr.p, Pt.v64.p, L.dinv64.p, omega, L.P.v64.p);
    FSI_CHECK_LAUNCH();
    set_tpr(L.P);
    bsr_transpose(L.P, L.R, s);
    Bsr AP2, Ac;
    bsr_spgemm(L.A, L.P, AP2, s);
    bsr_spgemm(L.R, AP2, Ac, s);
    // -(R A) where it pays: one pass over R and R A against b and x instead of the
    // residual (A, x, b read, r written) and its restriction (R, r read); kept when
    // that moves fewer bytes (in FP32) and the product's rows fit the SpGEMM table
    if (bsr_spgemm_if_fits(L.R, L.A, L.RAn, s)) {
      const double fused = L.R.spmv_bytes(4) + L.RAn.spmv_bytes(4) - 4.0 * L.R.rows();
      const double split = L.A.spmv_bytes(4) + 4.0 * L.A.rows() + L.R.spmv_bytes(4);
      if (fused < 0.95 * split) {
        bsr_scale(L.RAn, -1.0, s);
        L.RAn.tpr = lanes_for(L.RAn.nnzb + L.R.nnzb, L.RAn.nbr, 2.0);   // one lane group reads both rows
        L.RAn.tpr64 = lanes_for(L.RAn.nnzb + L.R.nnzb, L.RAn.nbr, 8.0);
      } else {
        L.RAn = Bsr();
      }
    }
    A = std::move(Ac);
    Bcur = std::move(Bc);
    B = Bcur.p;
    k = k;   // coarse block size equals the near-nullspace dimension
    FSI_CUDA(cudaStreamSynchronize(s));
  }
  // ---- coarsest level: dense inverse
  AmgLevel& C = H.levels.back();
  const int64_t nc = C.A.rows();
  require(nc <= 8192, "amg_setup: coarsest level too large for a dense inverse");
  H.ncoarse = (int)nc;
  DBuf<double> dense(nc * nc > 0 ? nc * nc : 1);
  H.cinv64.alloc(nc * nc > 0 ? nc * nc : 1);
  bsr_to_dense(C.A, dense.p, s);
  require(dense_inverse((int)nc, dense.p, H.cinv64.p, s), "amg_setup: singular coarsest matrix");
  FSI_CUDA(cudaStreamSynchronize(s));
  const int first = coarse_first_level(H, 8);
  if (first >= 0 && H.coarse_mode != COARSE_PER_LEVEL) coarse_plan_build<double>(H, first, H.crun64, s);
}

int coarse_first_level(const Hierarchy& H, int value_bytes) {
  const int L = (int)H.levels.size();
  if (L > kCoarseMaxLevels + 64) return -1;
  int first = L - 1;
  while (first - 1 >= 0) {
    const Bsr& A = H.levels[first - 1].A;
    const double bytes = (double)A.nnzb * A.br * A.bc * value_bytes;
    if (bytes > coarse_max_bytes()) break;
    --first;
  }
  if (first >= L - 1) return -1;                  // only the coarsest: nothing to merge
  if (L - first > kCoarseMaxLevels) first = L - kCoarseMaxLevels;
  return first;
}

void amg_make_fp32(Hierarchy& H, cudaStream_t s) {
  for (auto& L : H.levels) {
    const int64_t n = L.A.rows();
    bsr_make_fp32(L.A, s);
    bsr_make_delta16(L.A, s);
    if (L.P.nbr) { bsr_make_fp32(L.P, s); bsr_make_fp32(L.R, s); }
    if (L.RAn.nbr) bsr_make_fp32(L.RAn, s);
    to_f32(L.dinv64.p, L.dinv32, n, s);
    alloc_work(L.w32, n);
  }
  to_f32(H.cinv64.p, H.cinv32, (int64_t)H.ncoarse * H.ncoarse, s);
  H.has_fp32 = true;
  FSI_CUDA(cudaStreamSynchronize(s));
  const int first = coarse_first_level(H, 4);
  if (first >= 0 && H.coarse_mode != COARSE_PER_LEVEL) coarse_plan_build<float>(H, first, H.crun32, s);
}

template <class T>
void amg_vcycle(Hierarchy& H, const T* b, T* x, cudaStream_t s) {
  vcycle_level<T>(H, 0, b, x, s);
}

void cheb_setup(ChebSolver& C, Bsr&& A, int degree, double ratio, double upper, int power_iters, cudaStream_t s) {
  C.A = std::move(A);
  C.degree = degree; C.ratio = ratio; C.upper = upper;
  const int64_t n = C.A.rows();
  DBuf<double> diag(n > 0 ? n : 1);
  C.dinv64.alloc(n > 0 ? n : 1);
  bsr_point_diagonal(C.A, diag.p, s);
  invert_nonzero(n, diag.p, C.dinv64.p, s);
  C.lam = n > 0 ? power_lambda(C.A, C.dinv64.p, power_iters, 256, s) : 0.0;
  alloc_work(C.w64, n);
  FSI_CUDA(cudaStreamSynchronize(s));
}

void cheb_make_fp32(ChebSolver& C, cudaStream_t s) {
  bsr_make_fp32(C.A, s);
  bsr_make_delta16(C.A, s);
  to_f32(C.dinv64.p, C.dinv32, C.A.rows(), s);
  alloc_work(C.w32, C.A.rows());
  FSI_CUDA(cudaStreamSynchronize(s));
}

template <class T>
void cheb_apply(ChebSolver& C, const T* b, T* x, cudaStream_t s) {
  if (C.A.nbr == 0) return;
  LevelWork<T>& W = [&]() -> LevelWork<T>& {
    if constexpr (sizeof(T) == 8) return C.w64; else return C.w32;
  }();
  const T* dinv;
  if constexpr (sizeof(T) == 8) dinv = C.dinv64.p; else dinv = C.dinv32.p;
  cheb_sweep<T>(C.A, dinv, C.lam, C.degree, C.ratio, C.upper, b, x, W.xb.p, W.d.p, true, s);
}

template <class T>
double amg_smoother_steps(Hierarchy& H, int level, int reps, cudaStream_t s) {
  require(level >= 0 && level + 1 < (int)H.levels.size(), "smoother level must have a coarser level");
  AmgLevel& L = H.levels[level];
  LevelWork<T>& W = work<T>(L);
  const int64_t n = L.A.rows();
  if (!W.zeroed) {
    for (DBuf<T>* v : {&W.b, &W.x, &W.xb, &W.d}) FSI_CUDA(cudaMemsetAsync(v->p, 0, sizeof(T) * n, s));
    W.zeroed = true;
  }
  T* cur = W.x.p;
  T* oth = W.xb.p;
  for (int r = 0; r < reps; ++r) {
    spmv_cheb<T>(L.A, cur, W.b.p, dinv_of<T>(L), W.d.p, oth, T(0.5), T(0.5), s);
    T* t = cur; cur = oth; oth = t;
  }
  return cheb_step_bytes(L.A, (int)sizeof(T));
}

template double amg_smoother_steps<double>(Hierarchy&, int, int, cudaStream_t);
template double amg_smoother_steps<float>(Hierarchy&, int, int, cudaStream_t);
void cheb_apply_scratch(const ChebSolver& C, const double* b, double* x, double* xb, double* d, cudaStream_t s) {
  if (C.A.nbr == 0) return;
  cheb_sweep<double>(C.A, C.dinv64.p, C.lam, C.degree, C.ratio, C.upper, b, x, xb, d, true, s);
}

template void amg_vcycle<double>(Hierarchy&, const double*, double*, cudaStream_t);
template void amg_vcycle<float>(Hierarchy&, const float*, float*, cudaStream_t);
template void cheb_apply<double>(ChebSolver&, const double*, double*, cudaStream_t);
template void cheb_apply<float>(ChebSolver&, const float*, float*, cudaStream_t);

}  // namespace fsi

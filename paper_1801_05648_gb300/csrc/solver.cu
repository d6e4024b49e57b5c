// Block-LDU preconditioned FGMRES for the monolithic FSI Jacobian.
//
// Block structure (Eq. mat:small): DOFs in the class order m | s_v | s_u | f_v | f_p,
//   A = [[M, C_ms, 0], [C_sm, S, C_sf], [C_fm, C_fs, F]],  s = (s_v, s_u), f = (f_v, f_p).
// P^-1 r (Alg. 2, Sec. 4.1):
//   x_m = M^-1 r_m;  x_s = S^-1 r_s;  x_f = F^-1 (r_f - C_fm x_m - C_fs x_s);
//   x_s -= S^-1 C_sf x_f;  x_m -= M^-1 C_ms x_s.
// S^-1 (Alg. 3, Sec. 4.3): y = A_uu^-1 r_u;  x_v = S_hat^-1 (r_v - A_vu y), S_hat = A_vv + dt*theta*A_vu;
//   x_u = A_uu^-1 (r_u - A_uv x_v) = y + dt*theta x_v on the free s_u rows (A_uv = -dt*theta A_uu
//   there; fixed rows keep y), so one mass solve serves both steps of Alg. 3.
// F^-1 (Sec. 4.4, pressure Schur complement S_p = C_pp - B_pv diag(A_ff)^-1 B_vp):
//   y = A_ff^-1 r_v;  x_p = S_p^-1 (r_p - B_pv y);  x_v = A_ff^-1 (r_v - B_vp x_p).
// Inverses: smoothed-aggregation V-cycles (M, S_hat, A_ff, S_p) and a Chebyshev
// polynomial for the solid mass matrix A_uu.  The outer iteration is
// right-preconditioned FGMRES (Saad Alg. 9.6) with classical Gram-Schmidt applied
// twice and Givens rotations kept on the device.
#include "solver.cuh"
#include "spmv.cuh"
#include "vec.cuh"

#include <chrono>
#include <cmath>
#include <cstring>

namespace fsi {

namespace {

using clk = std::chrono::steady_clock;
inline double secs(clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); }

template <class T> PrecWork<T>& pwork(Context& C);
template <> PrecWork<double>& pwork<double>(Context& C) { return C.pw64; }
template <> PrecWork<float>& pwork<float>(Context& C) { return C.pw32; }

template <class T>
void alloc_pw(PrecWork<T>& W, int64_t n) {
  if (W.ready) return;
  W.in.alloc(n); W.out.alloc(n); W.a2_t.alloc(n); W.a2_u.alloc(n);
  W.s3_y.alloc(n); W.s3_t.alloc(n);
  W.ready = true;
}

void bsr_clone(const Bsr& A, Bsr& B, cudaStream_t s) {
  B = Bsr();
  B.nbr = A.nbr; B.nbc = A.nbc; B.br = A.br; B.bc = A.bc; B.nnzb = A.nnzb; B.tpr = A.tpr; B.tpr64 = A.tpr64;
  B.rowptr.alloc(A.nbr + 1);
  B.colind.alloc(A.nnzb > 0 ? A.nnzb : 1);
  B.v64.alloc(A.nnzb > 0 ? A.nnzb * A.br * A.bc : 1);
  FSI_CUDA(cudaMemcpyAsync(B.rowptr.p, A.rowptr.p, sizeof(int) * (A.nbr + 1), cudaMemcpyDeviceToDevice, s));
  if (A.nnzb) {
    FSI_CUDA(cudaMemcpyAsync(B.colind.p, A.colind.p, sizeof(int) * A.nnzb, cudaMemcpyDeviceToDevice, s));
    FSI_CUDA(cudaMemcpyAsync(B.v64.p, A.v64.p, sizeof(double) * A.nnzb * A.br * A.bc, cudaMemcpyDeviceToDevice, s));
  }
}

// ------------------------------------------------------------------ kernels
template <class Ti, class To>
__global__ void k_col_in(int64_t n, const Ti* __restrict__ V, int64_t ldv, const int* __restrict__ jdev, int joff,
                         To* __restrict__ out) {
  dep_wait();
  const int j = *jdev + joff;
  const Ti* src = V + (size_t)j * ldv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (To)src[i];
}
// zfix = (double) in; Z_j = zfix
template <class T>
__global__ void k_col_out(int64_t n, const T* __restrict__ in, double* __restrict__ zfix, double* __restrict__ Z,
                          int64_t ldz, const int* __restrict__ jdev) {
  dep_wait();
  double* dst = Z + (size_t)(*jdev) * ldz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)in[i];
    zfix[i] = v;
    dst[i] = v;
  }
}
// V_{j+1} = sign * w / h  (left zero when h == 0)
__global__ void k_scale_col(int64_t n, const double* __restrict__ w, const double* __restrict__ h,
                            double* __restrict__ V, int64_t ldv, const int* __restrict__ jdev, double sign) {
  dep_wait();
  const double hv = *h;
  double* dst = V + (size_t)(*jdev + 1) * ldv;
  const double inv = hv > 0.0 ? sign / hv : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = w[i] * inv;
}

// Hessenberg column j = h1 + h2 (two Gram-Schmidt passes on w), or, with defect != 0,
// e_j - (h1 + h2) (the passes ran on the defect v_j - w), h_{j+1,j} = ||w||; apply the
// previous rotations, form the new one, update g.  Writes |g_{j+1}|/||b|| and a
// breakdown flag to host-mapped memory.  One thread.
__global__ void k_givens(int ldh, const int* __restrict__ jdev, const double* __restrict__ h1,
                         const double* __restrict__ h2, const double* __restrict__ hnorm, double* __restrict__ H,
                         double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                         const double* __restrict__ inv_bnorm_p, double* __restrict__ out, int defect) {
  dep_wait();
  const double inv_bnorm = *inv_bnorm_p;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int j = *jdev;
  double* col = H + (size_t)j * ldh;
  double w0 = 0.0;
  for (int i = 0; i <= j; ++i) {
    col[i] = defect ? (i == j ? 1.0 : 0.0) - (h1[i] + h2[i]) : h1[i] + h2[i];
    w0 += col[i] * col[i];
  }
  const double hn = *hnorm;
  col[j + 1] = hn;
  w0 = sqrt(w0 + hn * hn);
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[j], col[j + 1]);
  double c = 1.0, sv = 0.0;
  if (den > 0.0) { c = col[j] / den; sv = col[j + 1] / den; }
  cs[j] = c; sn[j] = sv;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -sv * g[j];
  g[j] = c * g[j];
  out[0] = fabs(g[j + 1]) * inv_bnorm;
  out[1] = (hn <= 1e-14 * w0) ? 1.0 : 0.0;
  out[2] = hn;
  out[3] = (isfinite(g[j + 1]) && isfinite(hn)) ? 0.0 : 1.0;
}

// H y = g, k x k upper triangular (column-major, leading dimension ldh); one thread
__global__ void k_backsolve(int ldh, const int* __restrict__ kdev, const double* __restrict__ H,
                            const double* __restrict__ g, double* __restrict__ y) {
  dep_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = *kdev;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * ldh + i] * y[l];
    y[i] = s / H[(size_t)i * ldh + i];
  }
}

__global__ void k_set_first(double* __restrict__ g, int len, double beta) {
  dep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) g[i] = (i == 0) ? beta : 0.0;
}

inline int grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > device_sms() * 8) b = device_sms() * 8;
  return (int)(b < 1 ? 1 : b);
}

// near-nullspaces (host-built, node-major rows, row-major columns)
std::vector<double> translations(int64_t nodes, int d) {
  std::vector<double> B((size_t)nodes * d * d, 0.0);
  for (int64_t i = 0; i < nodes; ++i)
    for (int r = 0; r < d; ++r) B[((size_t)i * d + r) * d + r] = 1.0;
  return B;
}

std::vector<double> rigid_modes(const double* X, int64_t nodes, int d) {
  const int k = d == 2 ? 3 : 6;
  std::vector<double> B((size_t)nodes * d * k, 0.0);
  for (int64_t i = 0; i < nodes; ++i) {
    auto at = [&](int r, int c) -> double& { return B[((size_t)i * d + r) * k + c]; };
    for (int r = 0; r < d; ++r) at(r, r) = 1.0;
    const double x = X[i * d], y = X[i * d + 1];
    if (d == 2) {
      at(0, 2) = -y; at(1, 2) = x;
    } else {
      const double z = X[i * d + 2];
      at(0, 3) = -y; at(1, 3) = x;
      at(1, 4) = -z; at(2, 4) = y;
      at(2, 5) = -x; at(0, 5) = z;
    }
  }
  return B;
}

void upload(DBuf<double>& dst, const std::vector<double>& src, cudaStream_t s) {
  dst.alloc(src.size() > 0 ? src.size() : 1);
  if (!src.empty())
    FSI_CUDA(cudaMemcpyAsync(dst.p, src.data(), sizeof(double) * src.size(), cudaMemcpyHostToDevice, s));
  FSI_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ sub-solves
// x = inverse of hierarchy h applied with `nc` V-cycles: x = V(b); x += V(b - A x) ...
// The residual and correction of the repeated cycles use the level-0 work vectors
// b and x of that hierarchy (a V-cycle leaves them untouched on level 0), so
// sub-solves on different hierarchies can run concurrently.
template <class T>
void amg_solve(Context& C, int h, int nc, const T* b, T* x, cudaStream_t st) {
  Hierarchy& H = C.H[h];
  amg_vcycle<T>(H, b, x, st);
  if (nc <= 1) return;
  const Bsr& A = H.levels[0].A;
  const int64_t nn = A.rows();
  LevelWork<T>& W = [&]() -> LevelWork<T>& {
    if constexpr (sizeof(T) == 8) return H.levels[0].w64; else return H.levels[0].w32;
  }();
  for (int c = 1; c < nc; ++c) {
    spmv2_resid<T>(A, x, nullptr, nullptr, b, W.b.p, st);
    amg_vcycle<T>(H, W.b.p, W.x.p, st);
    axpby<T>(nn, T(1), W.x.p, T(1), x, st);
  }
}

template <class T>
void mesh_solve(Context& C, const T* r, T* x, cudaStream_t st) { amg_solve<T>(C, 0, C.prm.vc_mesh, r, x, st); }

// Alg. 3: solid sub-solve on (r_v, r_u) -> (x_v, x_u)
template <class T> const T* uv_weight(const Context& C);
template <> const double* uv_weight<double>(const Context& C) { return C.uv_w64.p; }
template <> const float* uv_weight<float>(const Context& C) { return C.uv_w32.p; }

// w[i] = c where scalar row i of A (block rows of br) has entries, else 0
__global__ void k_row_weight(int nbr, int br, const int* __restrict__ rowptr, double c, double* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr * br) return;
  const int r = i / br;
  w[i] = rowptr[r + 1] > rowptr[r] ? c : 0.0;
}

// r_u_zero: the caller's r_u is zero by structure; y = A_uu^-1 0 = 0 and t = r_v
// exactly, so the mass solve and the A_vu product are skipped (same result).
template <class T>
void solid_solve(Context& C, const T* r, T* x, cudaStream_t st, bool r_u_zero = false) {
  PrecWork<T>& W = pwork<T>(C);
  const int64_t nsv = C.off[2] - C.off[1];
  const T* r_v = r;
  const T* r_u = r + nsv;
  T* x_v = x;
  T* x_u = x + nsv;
  const int64_t nsu = C.off[3] - C.off[2];
  if (r_u_zero) {
    amg_solve<T>(C, 1, C.prm.vc_solid, r_v, x_v, st);                          // x_v = S_hat^-1 r_v
    vmul<T>(nsu, x_v, uv_weight<T>(C), x_u, st);                                // x_u = dt*theta x_v
    return;
  }
  cheb_apply<T>(C.mass, r_u, x_u, st);                                        // y = A_uu^-1 r_u (in x_u)
  spmv2_resid<T>(C.A_vu, x_u, nullptr, nullptr, r_v, W.s3_t.p, st);           // t = r_v - A_vu y
  amg_solve<T>(C, 1, C.prm.vc_solid, W.s3_t.p, x_v, st);                      // x_v = S_hat^-1 t
  vfma<T>(nsu, uv_weight<T>(C), x_v, x_u, st);                                // x_u = y + dt*theta x_v
}

// ---- Sec. 4.4 inner solver for A_ff^-1: k steps of GMRES on A_ff from x = 0,
// right-preconditioned by the A_ff V-cycle(s).  Arnoldi in FP64 with classical
// Gram-Schmidt applied twice; the (k+1) x k least-squares problem by Givens
// rotations in one device thread; x = Z y.  k is fixed (no stopping test), so the
// whole sequence is enqueued once and can be captured into the iteration graph.

// out = w / a with a = nrm[0] (sqrt(nrm[0]) when squared); out = 0 when a == 0
__global__ void k_unit_scale(int64_t n, const double* __restrict__ w, const double* __restrict__ nrm, int squared,
                             double* __restrict__ out) {
  dep_wait();
  const double a = squared ? sqrt(nrm[0]) : nrm[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a > 0.0 ? w[i] / a : 0.0;
}

// y = argmin || beta e_1 - H y ||, H the (k+1) x k Hessenberg matrix of the Arnoldi
// step: H(i, j) = h1[j ld + i] + h2[j ld + i] for i <= j (the two Gram-Schmidt
// passes), H(j+1, j) = nrm[j]; beta = sqrt(beta2[0]).  A zero pivot (exact
// breakdown) gives y_i = 0 for that column.
__global__ void k_inner_ls(int k, const double* __restrict__ h1, const double* __restrict__ h2, int ld,
                           const double* __restrict__ nrm, const double* __restrict__ beta2, double* __restrict__ y) {
  __shared__ double R[kFluidGmresMax + 1][kFluidGmresMax];   // shared, not local: no stack frame
  __shared__ double g[kFluidGmresMax + 1], cs[kFluidGmresMax], sn[kFluidGmresMax];
  dep_wait();
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i <= k; ++i) R[i][j] = 0.0;
    for (int i = 0; i <= j; ++i) R[i][j] = h1[(size_t)j * ld + i] + h2[(size_t)j * ld + i];
    R[j + 1][j] = nrm[j];
  }
  for (int i = 0; i <= k; ++i) g[i] = 0.0;
  g[0] = sqrt(beta2[0]);
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * R[i][j] + sn[i] * R[i + 1][j];
      R[i + 1][j] = -sn[i] * R[i][j] + cs[i] * R[i + 1][j];
      R[i][j] = t;
    }
    const double den = hypot(R[j][j], R[j + 1][j]);
    cs[j] = den > 0.0 ? R[j][j] / den : 1.0;
    sn[j] = den > 0.0 ? R[j + 1][j] / den : 0.0;
    R[j][j] = den;
    R[j + 1][j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
  }
  for (int i = k - 1; i >= 0; --i) {
    double acc = g[i];
    for (int l = i + 1; l < k; ++l) acc -= R[i][l] * y[l];
    y[i] = R[i][i] != 0.0 ? acc / R[i][i] : 0.0;
  }
}

template <class Ti, class To>
void copy_as(int64_t n, const Ti* x, To* y, cudaStream_t st) {
  if constexpr (sizeof(Ti) == sizeof(To)) axpby<To>(n, To(1), x, To(0), y, st);
  else cast<Ti, To>(n, x, y, st);
}

template <class T>
void aff_gmres(Context& C, const T* r, T* x, cudaStream_t st) {
  FluidGmres& F = C.fg;
  const int k = F.k;
  const int64_t n = F.n;
  const int ld = k + 1;
  const Bsr& A = C.H[2].levels[0].A;
  double* V = F.V.p;
  double* Z = F.Z.p;
  copy_as<T, double>(n, r, F.w.p, st);                                          // v_0 = r / ||r||
  dot_dev<double>(n, F.w.p, F.w.p, F.part.p, F.beta.p, st);
  launch_k(k_unit_scale, grid_n(n), 256, 0, st, n, (const double*)F.w.p, (const double*)F.beta.p, 1, V);
  for (int j = 0; j < k; ++j) {
    double* vj = V + (size_t)j * n;
    double* zj = Z + (size_t)j * n;
    if constexpr (sizeof(T) == 4) {                                             // z_j = V-cycle(v_j)
      cast<double, float>(n, vj, F.t32a.p, st);
      amg_solve<float>(C, 2, C.prm.vc_fluid, F.t32a.p, F.t32b.p, st);
      cast<float, double>(n, F.t32b.p, zj, st);
    } else {
      amg_solve<double>(C, 2, C.prm.vc_fluid, vj, zj, st);
    }
    spmv_axpby<double>(A, zj, 1.0, 0.0, F.w.p, st);                             // w = A_ff z_j
    double* hj1 = F.h1.p + (size_t)j * ld;
    double* hj2 = F.h2.p + (size_t)j * ld;
    mdot(n, V, n, F.zero.p, j + 1, F.w.p, F.part.p, hj1, ld, st);              // CGS, twice
    maxpy(n, V, n, F.zero.p, j + 1, hj1, 1.0, F.w.p, nullptr, k + 1, st);
    mdot(n, V, n, F.zero.p, j + 1, F.w.p, F.part.p, hj2, ld, st);
    maxpy(n, V, n, F.zero.p, j + 1, hj2, 1.0, F.w.p, F.npart.p, k + 1, st);
    finish_norm(F.npart.p, F.nrm.p + j, st);                                    // h_{j+1,j} = ||w||
    if (j + 1 < k)
      launch_k(k_unit_scale, grid_n(n), 256, 0, st, n, (const double*)F.w.p, (const double*)(F.nrm.p + j), 0,
               V + (size_t)(j + 1) * n);
  }
  launch_k(k_inner_ls, 1, 32, 0, st, k, (const double*)F.h1.p, (const double*)F.h2.p, ld, (const double*)F.nrm.p,
           (const double*)F.beta.p, F.y.p);
  FSI_CUDA(cudaMemsetAsync(F.w.p, 0, sizeof(double) * n, st));
  maxpy(n, Z, n, F.zero.p, k, F.y.p, -1.0, F.w.p, nullptr, k, st);              // x = Z y
  copy_as<double, T>(n, F.w.p, x, st);
}

// Workspace of the inner GMRES for the current flags and k (allocated outside any
// stream capture: at preconditioner build, before a solve, before a block apply).
void ensure_fluid_gmres(Context& C) {
  if (!(C.prm.flags & FLUID_GMRES)) return;
  FluidGmres& F = C.fg;
  const int k = C.prm.fluid_gmres_iters;
  const int64_t n = C.off[4] - C.off[3];
  if (F.k == k && F.n == n) return;
  F.k = k;
  F.n = n;
  if (n == 0) return;
  F.V.alloc((size_t)(k + 1) * n);
  F.Z.alloc((size_t)k * n);
  F.w.alloc(n);
  F.t32a.alloc(n);
  F.t32b.alloc(n);
  F.h1.alloc((size_t)(k + 1) * k);
  F.h2.alloc((size_t)(k + 1) * k);
  F.nrm.alloc(k);
  F.beta.alloc(1);
  F.y.alloc(k);
  F.part.alloc((size_t)(k + 1) * kRedBlocks);
  F.npart.alloc(kRedBlocks);
  F.zero.alloc(1);
  FSI_CUDA(cudaMemsetAsync(F.zero.p, 0, sizeof(int), C.s));
  if (C.iter_graph) { cudaGraphExecDestroy(C.iter_graph); C.iter_graph = nullptr; }
}

// A_ff^-1 of the fluid solve: V-cycle(s), or the inner GMRES with FLUID_GMRES
template <class T>
void aff_inverse(Context& C, const T* r, T* x, cudaStream_t st) {
  if (!(C.prm.flags & FLUID_GMRES)) {
    amg_solve<T>(C, 2, C.prm.vc_fluid, r, x, st);
    return;
  }
  require(C.fg.k == C.prm.fluid_gmres_iters && C.fg.n == C.off[4] - C.off[3], "inner fluid GMRES not prepared");
  if (C.fg.n > 0) aff_gmres<T>(C, r, x, st);
}

// fluid sub-solve on (r_v, r_p) -> (x_v, x_p)
template <class T>
void fluid_solve(Context& C, const T* r, T* x, cudaStream_t st) {
  PrecWork<T>& W = pwork<T>(C);
  const int64_t nfv = C.off[4] - C.off[3];
  const T* r_v = r;
  const T* r_p = r + nfv;
  T* x_v = x;
  T* x_p = x + nfv;
  aff_inverse<T>(C, r_v, W.s3_y.p, st);                                       // y = A_ff^-1 r_v
  spmv2_resid<T>(C.B_pv, W.s3_y.p, nullptr, nullptr, r_p, W.s3_t.p, st);      // t = r_p - B_pv y
  amg_solve<T>(C, 3, C.prm.vc_pressure, W.s3_t.p, x_p, st);                   // x_p = S_p^-1 t
  spmv2_resid<T>(C.B_vp, x_p, nullptr, nullptr, r_v, W.s3_t.p, st);           // t = r_v - B_vp x_p
  aff_inverse<T>(C, W.s3_t.p, x_v, st);                                       // x_v = A_ff^-1 t
}

}  // namespace

Context::~Context() {
  if (iter_graph) cudaGraphExecDestroy(iter_graph);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (s2) cudaStreamDestroy(s2);
  if (pinned) cudaFreeHost(pinned);
  if (pinned_j) cudaFreeHost(pinned_j);
  if (own_stream && s) cudaStreamDestroy(s);
}

// Class blocks of the operator (Eq. mat:small): the four pieces of the outer
// operator and the preconditioner's blocks, all extracted on the device.
static void extract_blocks(Context& C, const CsrView& A) {
  const int d = C.dim;
  const int64_t* o = C.off;
  const int nV = (int)(o[4] / d);
  const int nP = (int)(o[5] - o[4]);
  const int nm = (int)((o[1] - o[0]) / d), nsv = (int)((o[2] - o[1]) / d), nsu = (int)((o[3] - o[2]) / d);
  const int ns = nsv + nsu, nfv = (int)((o[4] - o[3]) / d), nms = (int)(o[3] / d);
  cudaStream_t s = C.s;
  // outer operator
  extract_bsr(A, 0, nV, d, 0, nV, d, C.AVV, s);
  extract_bsr(A, 0, nV, d, o[4], nP, 1, C.AVP, s);
  extract_bsr(A, o[4], nP, 1, 0, nV, d, C.APV, s);
  extract_bsr(A, o[4], nP, 1, o[4], nP, 1, C.APP, s);
  bsr_make_pair_order(C.AVV, C.AVP, s);
  bsr_make_pair_order(C.APV, C.APP, s);
  // preconditioner blocks
  extract_bsr(A, o[0], nm, d, o[0], nm, d, C.Mblk, s);
  extract_bsr(A, o[0], nm, d, o[1], ns, d, C.C_ms, s);
  extract_bsr(A, o[1], nsv, d, o[1], nsv, d, C.Avv, s);
  extract_bsr(A, o[1], nsv, d, o[2], nsu, d, C.A_vu, s);
  extract_bsr(A, o[2], nsu, d, o[1], nsv, d, C.A_uv, s);
  extract_bsr(A, o[2], nsu, d, o[2], nsu, d, C.Auu, s);
  extract_bsr(A, o[1], ns, d, o[3], nfv, d, C.C_sv_f, s);
  extract_bsr(A, o[1], ns, d, o[4], nP, 1, C.C_sv_p, s);
  {
    // do the s_u rows of C_sf hold entries?  (The displacement equation couples
    // no fluid unknown, so normally not: then the S^-1 of step 4 of Alg. 2 sees
    // r_u = 0 and skips its mass solve, see solid_solve.)
    auto tail_empty = [&](const Bsr& B) {
      int rp[2] = {0, 0};
      const int b0 = nsv;   // first s_u block row
      if (B.nbr == 0) return true;
      FSI_CUDA(cudaMemcpyAsync(&rp[0], B.rowptr.p + b0, sizeof(int), cudaMemcpyDeviceToHost, s));
      FSI_CUDA(cudaMemcpyAsync(&rp[1], B.rowptr.p + B.nbr, sizeof(int), cudaMemcpyDeviceToHost, s));
      FSI_CUDA(cudaStreamSynchronize(s));
      return rp[0] == rp[1];
    };
    C.csf_u_zero = tail_empty(C.C_sv_f) && tail_empty(C.C_sv_p);
  }
  extract_bsr(A, o[3], nfv, d, o[0], nms, d, C.C_fv_ms, s);
  extract_bsr(A, o[4], nP, 1, o[0], nms, d, C.C_p_ms, s);
  extract_bsr(A, o[3], nfv, d, o[3], nfv, d, C.Aff, s);
  extract_bsr(A, o[3], nfv, d, o[4], nP, 1, C.B_vp, s);
  extract_bsr(A, o[4], nP, 1, o[3], nfv, d, C.B_pv, s);
  extract_bsr(A, o[4], nP, 1, o[4], nP, 1, C.Cpp, s);
}

void context_setup(Context& C, const int64_t* rowptr, const int32_t* colind, const double* vals,
                   const double* solid_coords) {
  SetupPhase setup_phase;
  auto t0 = clk::now();
  FSI_CUDA(cudaGetDevice(&C.device));
  FSI_CUDA(cudaStreamCreateWithFlags(&C.s2, cudaStreamNonBlocking));
  FSI_CUDA(cudaEventCreateWithFlags(&C.ev_fork, cudaEventDisableTiming));
  FSI_CUDA(cudaEventCreateWithFlags(&C.ev_join, cudaEventDisableTiming));
  const int d = C.dim;
  const int64_t* o = C.off;
  Csr A;
  A.n = C.n;
  A.nnz = rowptr[C.n];
  A.rowptr.alloc(C.n + 1);
  A.colind.alloc(A.nnz > 0 ? A.nnz : 1);
  A.vals.alloc(A.nnz > 0 ? A.nnz : 1);
  FSI_CUDA(cudaMemcpyAsync(A.rowptr.p, rowptr, sizeof(int64_t) * (C.n + 1), cudaMemcpyHostToDevice, C.s));
  if (A.nnz) {
    FSI_CUDA(cudaMemcpyAsync(A.colind.p, colind, sizeof(int) * A.nnz, cudaMemcpyHostToDevice, C.s));
    if (vals)
      FSI_CUDA(cudaMemcpyAsync(A.vals.p, vals, sizeof(double) * A.nnz, cudaMemcpyHostToDevice, C.s));
    else   // pattern only: the values come later from the device (fsi_update_values)
      FSI_CUDA(cudaMemsetAsync(A.vals.p, 0, sizeof(double) * A.nnz, C.s));
  }
  extract_blocks(C, A.view());
  // keep the pattern (not the values) for fsi_update_values
  FSI_CUDA(cudaStreamSynchronize(C.s));
  A.vals.release();
  C.pattern = std::move(A);
  const int nsv = (int)((o[2] - o[1]) / d);
  if (solid_coords && !(C.prm.flags & NO_RIGID_MODES)) upload(C.solid_B, rigid_modes(solid_coords, nsv, d), C.s);
  FSI_CUDA(cudaStreamSynchronize(C.s));
  C.setup_s = secs(t0, clk::now());
}

void context_update_values(Context& C, const double* vals_dev) {
  SetupPhase setup_phase;
  CsrView v = C.pattern.view();
  v.vals = vals_dev;
  extract_blocks(C, v);
  // every hierarchy, Schur operator, FP32 copy and captured graph refers to the old values
  C.built = false;
  C.fp32_ready = false;
  C.At_built = false;
  if (C.iter_graph) { cudaGraphExecDestroy(C.iter_graph); C.iter_graph = nullptr; }
  FSI_CUDA(cudaStreamSynchronize(C.s));
}

void precond_build(Context& C, int precision) {
  SetupPhase setup_phase;
  auto t0 = clk::now();
  auto& s = C.s;
  const int d = C.dim;
  if (!C.built) {
    // S_hat = A_vv + c A_vu  (Alg. 3)
    Bsr Shat;
    bsr_add(C.Avv, C.A_vu, C.prm.dt_theta, Shat, s);
    // S_p = C_pp - B_pv diag(A_ff)^-1 B_vp
    const int64_t nfv = C.Aff.rows();
    DBuf<double> diag(nfv > 0 ? nfv : 1), dinv(nfv > 0 ? nfv : 1);
    bsr_point_diagonal(C.Aff, diag.p, s);
    invert_nonzero(nfv, diag.p, dinv.p, s);
    Bsr Bs, BDB, Sp;
    bsr_clone(C.B_vp, Bs, s);
    bsr_scale_rows(Bs, dinv.p, s);
    bsr_spgemm(C.B_pv, Bs, BDB, s);
    bsr_add(C.Cpp, BDB, -1.0, Sp, s);
    // hierarchies
    DBuf<double> Bm, Bf, Bp;
    upload(Bm, translations(C.Mblk.nbr, d), s);
    upload(Bf, translations(C.Aff.nbr, d), s);
    upload(Bp, std::vector<double>((size_t)Sp.nbr, 1.0), s);
    const bool rigid = C.solid_B.p != nullptr;
    DBuf<double> Bst;
    if (!rigid) upload(Bst, translations(Shat.nbr, d), s);
    const int ks = rigid ? (d == 2 ? 3 : 6) : d;
    for (auto& H : C.H)
      H.coarse_mode = (C.prm.flags & CLUSTER_COARSE) ? COARSE_CLUSTER
                      : (C.prm.flags & GRID_COARSE)  ? COARSE_GRID
                                                     : COARSE_PER_LEVEL;
    amg_setup(C.H[0], std::move(C.Mblk), Bm.p, d, C.prm.amg, s);
    amg_setup(C.H[1], std::move(Shat), rigid ? C.solid_B.p : Bst.p, ks, C.prm.amg, s);
    amg_setup(C.H[2], std::move(C.Aff), Bf.p, d, C.prm.amg, s);
    amg_setup(C.H[3], std::move(Sp), Bp.p, 1, C.prm.amg, s);
    cheb_setup(C.mass, std::move(C.Auu), C.prm.mass_degree, C.prm.mass_ratio, C.prm.amg.cheb_upper,
               C.prm.amg.power_iters, s);
    {
      const int64_t nsu = C.off[3] - C.off[2];
      C.uv_w64.alloc(nsu > 0 ? nsu : 1);
      if (nsu > 0) {
        k_row_weight<<<div_up(nsu, 256), 256, 0, s>>>(C.A_uv.nbr, C.A_uv.br, C.A_uv.rowptr.p, C.prm.dt_theta,
                                                       C.uv_w64.p);
        FSI_CHECK_LAUNCH();
      }
    }
    C.Avv = Bsr();
    C.Cpp = Bsr();
    alloc_pw(C.pw64, C.n);
    C.built = true;
  }
  if (precision == 1 && !C.fp32_ready) {
    for (auto& H : C.H) amg_make_fp32(H, s);
    cheb_make_fp32(C.mass, s);
    {
      const int64_t nsu = C.off[3] - C.off[2];
      C.uv_w32.alloc(nsu > 0 ? nsu : 1);
      if (nsu > 0) cast<double, float>(nsu, C.uv_w64.p, C.uv_w32.p, s);
    }
    for (Bsr* B : {&C.C_ms, &C.A_vu, &C.A_uv, &C.C_sv_f, &C.C_sv_p, &C.C_fv_ms, &C.C_p_ms, &C.B_vp, &C.B_pv})
      bsr_make_fp32(*B, s);
    alloc_pw(C.pw32, C.n);
    C.fp32_ready = true;
  }
  C.precision = precision;
  if (C.iter_graph) { cudaGraphExecDestroy(C.iter_graph); C.iter_graph = nullptr; }
  FSI_CUDA(cudaStreamSynchronize(s));
  C.build_s = secs(t0, clk::now());
}

template <class T>
void precond_apply(Context& C, const T* r, T* z) {
  PrecWork<T>& W = pwork<T>(C);
  const int64_t* o = C.off;
  const T* r_m = r + o[0];
  const T* r_s = r + o[1];
  const T* r_f = r + o[3];
  T* z_m = z + o[0];
  T* z_s = z + o[1];
  T* z_f = z + o[3];
  const int64_t nfv = o[4] - o[3], ns = o[3] - o[1], nm = o[1] - o[0];
  const int variant = C.prm.precond_variant;
  if (variant == 2) {
    // (D + U)^-1: x_f = F^-1 r_f;  x_s = S^-1 (r_s - C_sf x_f);  x_m = M^-1 (r_m - C_ms x_s)
    fluid_solve<T>(C, r_f, z_f, C.s);
    spmv2_resid<T>(C.C_sv_f, z_f, &C.C_sv_p, z_f + nfv, r_s, W.a2_t.p, C.s);
    solid_solve<T>(C, W.a2_t.p, z_s, C.s);
    spmv2_resid<T>(C.C_ms, z_s, nullptr, nullptr, r_m, W.a2_t.p, C.s);
    mesh_solve<T>(C, W.a2_t.p, z_m, C.s);
    return;
  }
  // 1-2: independent, the mesh solve runs on the second stream (a parallel
  // branch when captured into a graph)
  FSI_CUDA(cudaEventRecord(C.ev_fork, C.s));
  FSI_CUDA(cudaStreamWaitEvent(C.s2, C.ev_fork, 0));
  mesh_solve<T>(C, r_m, z_m, C.s2);
  solid_solve<T>(C, r_s, z_s, C.s);
  if (variant == 3) fluid_solve<T>(C, r_f, z_f, C.s);        // D^-1: x_f = F^-1 r_f
  FSI_CUDA(cudaEventRecord(C.ev_join, C.s2));
  FSI_CUDA(cudaStreamWaitEvent(C.s, C.ev_join, 0));
  if (variant == 3) return;
  // 3: t_f = r_f - C_fm x_m - C_fs x_s  (x_m, x_s contiguous), x_f = F^-1 t_f
  spmv2_resid<T>(C.C_fv_ms, z, nullptr, nullptr, r_f, W.a2_t.p, C.s);
  spmv2_resid<T>(C.C_p_ms, z, nullptr, nullptr, r_f + nfv, W.a2_t.p + nfv, C.s);
  fluid_solve<T>(C, W.a2_t.p, z_f, C.s);
  if (variant == 1) return;                                    // (D + L)^-1: steps 1-3
  // 4: x_s -= S^-1 C_sf x_f
  spmv2_axpby<T>(C.C_sv_f, z_f, &C.C_sv_p, z_f + nfv, T(1), T(0), W.a2_t.p, C.s);
  solid_solve<T>(C, W.a2_t.p, W.a2_u.p, C.s, C.csf_u_zero);
  axpby<T>(ns, T(-1), W.a2_u.p, T(1), z_s, C.s);
  // 5: x_m -= M^-1 C_ms x_s
  spmv_axpby<T>(C.C_ms, z_s, T(1), T(0), W.a2_t.p, C.s);
  mesh_solve<T>(C, W.a2_t.p, W.a2_u.p, C.s);
  axpby<T>(nm, T(-1), W.a2_u.p, T(1), z_m, C.s);
}

template <class T>
void apply_block(Context& C, int which, const T* in, T* out) {
  ensure_fluid_gmres(C);
  switch (which) {
    case 0: amg_solve<T>(C, 0, C.prm.vc_mesh, in, out, C.s); break;
    case 1: amg_solve<T>(C, 1, C.prm.vc_solid, in, out, C.s); break;
    case 2: aff_inverse<T>(C, in, out, C.s); break;
    case 3: amg_solve<T>(C, 3, C.prm.vc_pressure, in, out, C.s); break;
    case 4: cheb_apply<T>(C.mass, in, out, C.s); break;
    case 5: solid_solve<T>(C, in, out, C.s); break;
    case 6: fluid_solve<T>(C, in, out, C.s); break;
    case 7: precond_apply<T>(C, in, out); break;
    default: throw Error(EINVAL_, "apply_block: unknown block");
  }
}

void apply_operator(Context& C, const double* x, double* y) {
  OuterOperatorScope outer;
  const int64_t nv = C.off[4];
  spmv2_axpby<double>(C.AVV, x, &C.AVP, x + nv, 1.0, 0.0, y, C.s);
  spmv2_axpby<double>(C.APV, x, &C.APP, x + nv, 1.0, 0.0, y + nv, C.s);
}

static void operator_resid(Context& C, const double* x, const double* b, double* r) {
  OuterOperatorScope outer;
  const int64_t nv = C.off[4];
  spmv2_resid<double>(C.AVV, x, &C.AVP, x + nv, b, r, C.s);
  spmv2_resid<double>(C.APV, x, &C.APP, x + nv, b + nv, r + nv, C.s);
}

double operator_bytes(const Context& C) {
  // values + indices + x (once) + y, both row classes
  return C.AVV.spmv_bytes(8) + C.AVP.spmv_bytes(8) + C.APV.spmv_bytes(8) + C.APP.spmv_bytes(8) -
         8.0 * (double)(C.AVV.rows() + C.APV.rows());   // y counted twice by the split
}

double precond_bytes(const Context& C, int vb) {
  const SolverParams& p = C.prm;
  // Alg. 2: two mesh solves, two solid solves (one mass solve each, none in the
  // second when its r_u is structurally zero, and the x_u update), one fluid solve
  // (two A_ff solves and one S_p solve), and the coupling products
  // (the other block factorisations: one mesh and one solid solve, and only their couplings)
  const bool ldu = p.precond_variant == 0;
  const double nmesh = ldu ? 2.0 : 1.0, nsolid = ldu ? 2.0 : 1.0;
  double b = 0;
  b += nmesh * p.vc_mesh * C.H[0].vcycle_bytes(vb) + nsolid * p.vc_solid * C.H[1].vcycle_bytes(vb) +
       1.0 * p.vc_pressure * C.H[3].vcycle_bytes(vb);
  if (p.flags & FLUID_GMRES) {
    // per A_ff^-1: k steps of (V-cycle, FP64 A_ff product, two Gram-Schmidt passes
    // over V_0..V_j: read V twice and w, write w), the start and x = Z y
    const double nf = (double)(C.off[4] - C.off[3]);
    const int k = p.fluid_gmres_iters;
    double g = 3.0 * 8.0 * nf + 8.0 * nf * (k + 2);
    for (int j = 0; j < k; ++j)
      g += p.vc_fluid * C.H[2].vcycle_bytes(vb) + C.H[2].levels[0].A.spmv_bytes(8) + 2.0 * 8.0 * nf * (2.0 * (j + 1) + 3.0) +
           (vb == 4 ? 2.0 * 12.0 * nf : 0.0) + 16.0 * nf;
    b += 2.0 * g;
  } else {
    b += 2.0 * p.vc_fluid * C.H[2].vcycle_bytes(vb);
  }
  const double mass_solves = ldu ? (C.csf_u_zero ? 1.0 : 2.0) : 1.0;   // step 4's S^-1 skips its mass solve when r_u = 0
  b += mass_solves * C.mass.degree * C.mass.A.spmv_bytes(vb);
  b += nsolid * 4.0 * vb * (double)(C.off[3] - C.off[2]);
  const int v = p.precond_variant;
  if (v == 0 || v == 2) for (const Bsr* B : {&C.C_ms, &C.C_sv_f, &C.C_sv_p}) b += B->spmv_bytes(vb);
  if (v == 0 || v == 1) for (const Bsr* B : {&C.C_fv_ms, &C.C_p_ms}) b += B->spmv_bytes(vb);
  b += mass_solves * C.A_vu.spmv_bytes(vb) + C.B_vp.spmv_bytes(vb) + C.B_pv.spmv_bytes(vb);
  return b;
}

// ------------------------------------------------------------------ FGMRES
namespace {

void ensure_krylov(Context& C) {
  const int m = C.prm.restart;
  if (C.m_alloc == m) return;
  const int64_t n = C.n;
  C.ldv = (n + 31) / 32 * 32;
  C.V.alloc((size_t)(m + 1) * C.ldv);
  C.Z.alloc((size_t)m * C.ldv);
  C.Hh.alloc((size_t)(m + 1) * m);
  C.cs.alloc(m + 1); C.sn.alloc(m + 1); C.g.alloc(m + 2); C.y.alloc(m + 1);
  C.h1.alloc(m + 2); C.h2.alloc(m + 2); C.scal.alloc(8);
  C.partials.alloc((size_t)(m + 2) * kRedBlocks);
  C.npart.alloc(kRedBlocks);
  C.zfix.alloc(n); C.wfix.alloc(n); C.rvec.alloc(n);
  C.jdev.alloc(1); C.kdev.alloc(1);
  C.dpart.alloc(kRedBlocks); C.reorth.alloc(2);
  if (!C.pinned) {
    FSI_CUDA(cudaHostAlloc(&C.pinned, 8 * sizeof(double), cudaHostAllocMapped));
    FSI_CUDA(cudaHostGetDevicePointer(&C.pinned_dev, C.pinned, 0));
    FSI_CUDA(cudaHostAlloc(&C.pinned_j, 4 * sizeof(int), cudaHostAllocDefault));
  }
  C.m_alloc = m;
  if (C.iter_graph) { cudaGraphExecDestroy(C.iter_graph); C.iter_graph = nullptr; }
}

// One FGMRES iteration for the index held in C.jdev: Z_j = P^-1 V_j,
// w = A Z_j, Gram-Schmidt against V_0..V_j, Givens update, V_{j+1} = w / ||w||.
// Second-pass threshold of the Arnoldi Gram-Schmidt: one pass leaves the new
// vector orthogonal to about u ||d|| / ||d'|| (u the unit roundoff), so a pass that
// keeps at least 1% of the norm leaves it within ~1e-14.
constexpr double kReorthEta = 1e-2;
template <class T>
void iteration_body(Context& C) {
  const int64_t n = C.n;
  const int m = C.prm.restart;
  PrecWork<T>& W = pwork<T>(C);
  launch_k(k_col_in<double, T>, grid_n(n), 256, 0, C.s, n, (const double*)C.V.p, C.ldv, (const int*)C.jdev.p, 0,
           W.in.p);
  precond_apply<T>(C, W.in.p, W.out.p);
  launch_k(k_col_out<T>, grid_n(n), 256, 0, C.s, n, (const T*)W.out.p, C.zfix.p, C.Z.p, C.ldv, (const int*)C.jdev.p);
  apply_operator(C, C.zfix.p, C.wfix.p);
  if (C.harvest) harvest_residual(n, C.V.p, C.ldv, C.jdev.p, C.wfix.p, C.harvest, C.harvest_n, C.s);
  if (C.prm.flags & LEARNED) {
    // learned stage: r' = v_j - A z_j, c = MLP(r'), t = A c; take z_j + c only
    // when ||r' - t|| < tau ||r'|| (otherwise the plain preconditioner's z_j stands)
    Learned& L = C.learned;
    learned_residual(n, C.V.p, C.ldv, C.jdev.p, C.wfix.p, L.rp.p, L.part.p, C.s);
    mlp_apply(learned_geom(L, C.off), L.w16.p, L.rp.p, L.c.p, C.s);
    apply_operator(C, L.c.p, L.t.p);
    learned_decide(n, L.rp.p, L.t.p, C.prm.learned_accept, L.part.p, L.counters.p, C.s);
    learned_commit(n, L.counters.p, L.c.p, L.t.p, C.Z.p, C.ldv, C.jdev.p, C.wfix.p, C.s);
  }
  // Arnoldi step on the defect d = v_j - w (classical Gram-Schmidt, a second pass
  // only when the first kept less than kReorthEta of ||d||): h = e_j - V^T d,
  // w - V h = -(d - V V^T d), so v_{j+1} = -d' / ||d'||.
  arnoldi_defect(n, C.V.p, C.ldv, C.jdev.p, C.wfix.p, C.dpart.p, C.s);
  mdot(n, C.V.p, C.ldv, C.jdev.p, 1, C.wfix.p, C.partials.p, C.h1.p, m + 1, C.s);
  maxpy(n, C.V.p, C.ldv, C.jdev.p, 1, C.h1.p, 1.0, C.wfix.p, C.npart.p, m + 1, C.s);
  reorth_flag(C.npart.p, C.dpart.p, kReorthEta, C.reorth.p, C.s);
  mdot(n, C.V.p, C.ldv, C.jdev.p, 1, C.wfix.p, C.partials.p, C.h2.p, m + 1, C.s, C.reorth.p);
  maxpy(n, C.V.p, C.ldv, C.jdev.p, 1, C.h2.p, 1.0, C.wfix.p, C.npart.p, m + 1, C.s, C.reorth.p);
  finish_norm(C.npart.p, C.scal.p, C.s);
  launch_k(k_givens, 1, 32, 0, C.s, m + 1, C.jdev.p, C.h1.p, C.h2.p, C.scal.p, C.Hh.p, C.cs.p, C.sn.p, C.g.p,
           C.scal.p + 5, C.pinned_dev, 1);
  launch_k(k_scale_col, grid_n(n), 256, 0, C.s, n, C.wfix.p, C.scal.p, C.V.p, C.ldv, C.jdev.p, -1.0);
}

void run_iteration(Context& C) {
  const bool graphs = (C.prm.flags & USE_GRAPHS) != 0;
  if (!graphs) {
    if (C.precision == 1) iteration_body<float>(C); else iteration_body<double>(C);
    return;
  }
  const bool learned = (C.prm.flags & LEARNED) != 0;
  const int fluid = (C.prm.flags & FLUID_GMRES) ? C.prm.fluid_gmres_iters : 0;
  if (!C.iter_graph || C.iter_graph_prec != C.precision || C.iter_graph_learned != learned ||
      C.iter_graph_harvest != C.harvest || C.iter_graph_harvest_n != C.harvest_n || C.iter_graph_fluid != fluid) {
    if (C.iter_graph) { cudaGraphExecDestroy(C.iter_graph); C.iter_graph = nullptr; }
    cudaGraph_t g;
    FSI_CUDA(cudaStreamBeginCapture(C.s, cudaStreamCaptureModeThreadLocal));
    const int64_t before = g_kernel_launches;
    try {
      if (C.precision == 1) iteration_body<float>(C); else iteration_body<double>(C);
    } catch (...) {
      cudaStreamEndCapture(C.s, &g);
      throw;
    }
    C.graph_kernels = g_kernel_launches - before;
    g_kernel_launches = before;       // captured, not executed
    FSI_CUDA(cudaStreamEndCapture(C.s, &g));
    FSI_CUDA(cudaGraphInstantiate(&C.iter_graph, g, 0));
    cudaGraphDestroy(g);
    C.iter_graph_prec = C.precision;
    C.iter_graph_learned = learned;
    C.iter_graph_harvest = C.harvest;
    C.iter_graph_harvest_n = C.harvest_n;
    C.iter_graph_fluid = fluid;
  }
  FSI_CUDA(cudaGraphLaunch(C.iter_graph, C.s));
  g_kernel_launches += C.graph_kernels;
}

}  // namespace

int fgmres_solve(Context& C, const double* b, double* x, double tol) {
  auto t0 = clk::now();
  const int64_t launches0 = g_kernel_launches;
  require(C.built, "fsi_solve before fsi_precond_build");
  if (C.prm.flags & LEARNED)
    require(C.learned.n_nodes > 0 && C.learned.has_weights,
            "FSI_LEARNED needs fsi_learned_setup and weights (fsi_learned_load or fsi_precond_build's path)");
  ensure_krylov(C);
  ensure_fluid_gmres(C);
  C.last_accepted = 0;
  C.last_reorth = 0;
  if (C.prm.flags & LEARNED) FSI_CUDA(cudaMemsetAsync(C.learned.counters.p, 0, 2 * sizeof(int), C.s));
  FSI_CUDA(cudaMemsetAsync(C.reorth.p, 0, 2 * sizeof(int), C.s));
  const int64_t n = C.n;
  const int m = C.prm.restart;
  C.hist.clear();
  const double bnorm = std::sqrt(dot_host<double>(n, b, b, C.partials.p, C.scal.p + 4, C.s));
  C.last_iters = 0; C.last_cycles = 0;
  if (!std::isfinite(bnorm)) {
    C.last_status = ENONFINITE_;
    C.solve_s = secs(t0, clk::now());
    throw Error(ENONFINITE_, "right-hand side is not finite");
  }
  if (!(C.prm.flags & X0_GIVEN)) FSI_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, C.s));
  if (bnorm == 0.0) {
    FSI_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, C.s));
    FSI_CUDA(cudaStreamSynchronize(C.s));
    C.last_true_relres = 0.0; C.last_status = OK;
    C.solve_s = secs(t0, clk::now());
    return OK;
  }
  C.pinned[4] = 1.0 / bnorm;
  FSI_CUDA(cudaMemcpyAsync(C.scal.p + 5, C.pinned + 4, sizeof(double), cudaMemcpyHostToDevice, C.s));
  int total = 0, status = ENOTCONV_;
  double relres = 0.0;
  bool breakdown = false, nonfinite = false;
  while (true) {
    operator_resid(C, x, b, C.rvec.p);
    const double beta = std::sqrt(dot_host<double>(n, C.rvec.p, C.rvec.p, C.partials.p, C.scal.p + 4, C.s));
    relres = beta / bnorm;
    if (!std::isfinite(relres)) { nonfinite = true; break; }
    if (relres <= tol) { status = OK; break; }
    if (total >= C.prm.maxit || breakdown) break;
    axpby<double>(n, 1.0 / beta, C.rvec.p, 0.0, C.V.p, C.s);
    launch_k(k_set_first, div_up(m + 2, 128), 128, 0, C.s, C.g.p, m + 2, beta);
    int k = 0;
    for (int j = 0; j < m; ++j) {
      C.pinned_j[0] = j;
      FSI_CUDA(cudaMemcpyAsync(C.jdev.p, C.pinned_j, sizeof(int), cudaMemcpyHostToDevice, C.s));
      run_iteration(C);
      FSI_CUDA(cudaStreamSynchronize(C.s));
      volatile double* pv = C.pinned;
      const double est = pv[0];
      const bool bd = pv[1] != 0.0;
      nonfinite = pv[3] != 0.0;
      C.hist.push_back(est);
      ++total;
      k = j + 1;
      if (nonfinite) break;
      if (bd) { breakdown = true; break; }
      if (est <= tol || total >= C.prm.maxit) break;
    }
    if (nonfinite) break;
    C.pinned_j[1] = k;
    FSI_CUDA(cudaMemcpyAsync(C.kdev.p, C.pinned_j + 1, sizeof(int), cudaMemcpyHostToDevice, C.s));
    launch_k(k_backsolve, 1, 32, 0, C.s, m + 1, C.kdev.p, C.Hh.p, C.g.p, C.y.p);
    maxpy(n, C.Z.p, C.ldv, C.kdev.p, 0, C.y.p, -1.0, x, nullptr, m, C.s);
    ++C.last_cycles;
  }
  FSI_CUDA(cudaStreamSynchronize(C.s));
  FSI_CUDA(cudaMemcpy(&C.last_reorth, C.reorth.p + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (C.learned.counters.p) {
    int cnt[3] = {0, 0, 0};
    FSI_CUDA(cudaMemcpy(cnt, C.learned.counters.p, sizeof(cnt), cudaMemcpyDeviceToHost));
    if (C.prm.flags & LEARNED) C.last_accepted = cnt[1];
    if (cnt[2] != 0) {
      FSI_CUDA(cudaMemset(C.learned.counters.p + 2, 0, sizeof(int)));
      C.last_status = ECUDA_;
      C.solve_s = secs(t0, clk::now());
      throw Error(ECUDA_, "a wait of the tensor-core MLP timed out; its corrections are not valid");
    }
  }
  if (spmv_stage_failed(C.s)) {
    C.last_status = ECUDA_;
    C.solve_s = secs(t0, clk::now());
    throw Error(ECUDA_, "a staged Chebyshev step timed out waiting for its copies; the result is not valid");
  }
  if (C.prm.flags & GRID_COARSE) {
    bool failed = false;
    for (auto& H : C.H) failed = coarse_failed(H, C.s) || failed;
    if (failed) {
      C.last_status = ECUDA_;
      C.solve_s = secs(t0, clk::now());
      throw Error(ECUDA_, "a grid barrier of the coarse-level kernel timed out; the result is not valid");
    }
  }
  C.last_iters = total;
  C.last_true_relres = relres;
  if (nonfinite) status = ENONFINITE_;
  else if (status != OK && breakdown) status = EBREAKDOWN_;
  C.last_status = status;
  C.solve_s = secs(t0, clk::now());
  C.last_launches = g_kernel_launches - launches0;
  return status;
}

template void precond_apply<double>(Context&, const double*, double*);
template void precond_apply<float>(Context&, const float*, float*);
template void apply_block<double>(Context&, int, const double*, double*);
template void apply_block<float>(Context&, int, const float*, float*);

}  // namespace fsi

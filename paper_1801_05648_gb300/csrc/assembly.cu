// Residual and Jacobian of the monolithic ALE fluid-structure system on the GPU
// (the Newton step of Alg. 1, Sec. 3.3; variational form Eq. (fsi:all) with the
// strong form of Sec. 2), on the structured Q2/Q2/Q1 box meshes the solver is
// benchmarked on.  Declarations and the data contract are in include/fsi.h
// (fsi_asm_*).
//
// Per cell and quadrature point, with F = I + grad u, J = det F, A = grad(v) F^-1,
// sigma_v = rho_f nu_f (A + A^T), dtt = dt theta, dto = dt (1 - theta):
//   fluid cells   f0 = rho_f J [(v - v_old) - A (u - u_old) + dtt A v]      tested with phi
//                 f1 = dtt J sigma_v F^-T - J p F^-T                         tested with grad phi
//                 g0 = J tr(A)                                               tested with psi (Q1)
//                 hm = grad(u) / J                                           tested with grad phi on mesh rows
//                 (theta < 1: rho_f (1 - theta)(J_old - J)(v - v_old) + rho_f dto J_old A_old v_old in f0,
//                  dto J_old sigma_v,old F_old^-T in f1: J^theta = theta J + (1 - theta) J_old)
//   solid cells   f0 = rho_s (v - v_old),  f1 = dtt F Sigma (+ dto F_old Sigma_old),
//                 Sigma = 2 mu_s E + lambda_s tr(E) I,  E = (F^T F - I) / 2
//                 k0 = (u - u_old) - dtt v (- dto v_old)                     tested with phi on u rows
//   outflow face  c = -dtt rho_f nu_f J F^-T grad(v)^T F^-T n (n = e_0; theta < 1 adds the
//   (fluid cells on x_0 = L_0)  previous level's term weighted dto)                  tested with phi on v rows
// The Jacobian is the exact derivative of this discrete residual: every point
// quantity is carried as a first-order dual number seeded along one local DOF,
// so a CTA computes one chunk of columns of the element matrix.
//
// Work decomposition: one CTA per (cell, column chunk).  Phase 1: one thread per
// (quadrature point, column) evaluates the point quantities above (value and one
// derivative) into shared memory.  Phase 2: one thread per (element row, column)
// sums its test-function weights over the points and adds the entry into the
// global CSR values (binary search of the column in the row).  Cells are launched
// colour by colour (the parities of their lattice coordinates): two cells of one
// colour share no node, so the in-place additions never race, and the order in
// which contributions reach an entry is fixed (deterministic, no atomics).
#include "../../include/fsi.h"
#include "common.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace fsi {
namespace {

// ------------------------------------------------------------------ first-order duals
struct D1 {
  double v, d;
};
__device__ __forceinline__ D1 dc(double a) { return {a, 0.0}; }
__device__ __forceinline__ D1 operator+(D1 a, D1 b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ D1 operator-(D1 a, D1 b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ D1 operator*(D1 a, D1 b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ D1 operator*(double s, D1 a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ D1 operator+(D1 a, double s) { return {a.v + s, a.d}; }
__device__ __forceinline__ D1 operator-(D1 a, double s) { return {a.v - s, a.d}; }
__device__ __forceinline__ D1 inv(D1 b) {
  const double r = 1.0 / b.v;
  return {r, -b.d * r * r};
}

// Element shape: PD = 0 continuous Q1 pressure (2^D vertex functions), PD = 1 the
// discontinuous P1 pressure of the paper's Q2-Q2-P1disc pair (D + 1 functions per cell).
template <int D, int PD> struct Sh;
template <int PD> struct Sh<2, PD> {
  static constexpr int NQ2 = 9, NQ1 = PD ? 3 : 4, NL = 36 + NQ1, NQP = 9, NFP = 3;
  static constexpr int CHUNK = 40;   // columns per CTA (all)
};
template <int PD> struct Sh<3, PD> {
  static constexpr int NQ2 = 27, NQ1 = PD ? 4 : 8, NL = 162 + NQ1, NQP = 27, NFP = 9;
  static constexpr int CHUNK = 17;   // 10 chunks of columns
};
// shared slots per (point, column): f0 (D), f1 (D x D), then hm (D x D) and g0 (fluid) or k0 (solid)
template <int D> constexpr int kSlots = D + D * D + D * D + 1;
constexpr int kAsmThreads = 256;

// Quadrature tables of one mesh (reference cell scaled by the cell size h).
struct Tables {
  const double* N;    // [NQP][NQ2]
  const double* dN;   // [NQP][NQ2][D]
  const double* Np;   // [NQP][NQ1]
  const double* w;    // [NQP]
  const double* Nf;   // [NFP][NQ2]   outflow face x_0 = 1 of the reference cell
  const double* dNf;  // [NFP][NQ2][D]
  const double* wf;   // [NFP]
};

struct Phys {
  double rho_f, nu_f, mu_s, lambda_s, rho_s, dt, theta;
};

struct CellGeom {
  int n[3];           // cells per direction
  int color;          // parity pattern of the launched cells
  int m[3];           // cells of this colour per direction
};

template <int D>
__device__ __forceinline__ int64_t colour_cell(const CellGeom& g, int64_t k, int* c) {
  int64_t r = k;
  for (int d = 0; d < D; ++d) {
    const int i = (int)(r % g.m[d]);
    r /= g.m[d];
    c[d] = 2 * i + ((g.color >> d) & 1);
  }
  int64_t idx = c[D - 1];
  for (int d = D - 2; d >= 0; --d) idx = idx * g.n[d] + c[d];
  return idx;
}

template <int D>
__device__ __forceinline__ D1 det(const D1 (&F)[D][D]) {
  if constexpr (D == 2) return F[0][0] * F[1][1] - F[0][1] * F[1][0];
  else
    return F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
           F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
}
// F^-1 = cof(F)^T / J
template <int D>
__device__ __forceinline__ void invert(const D1 (&F)[D][D], D1 iJ, D1 (&R)[D][D]) {
  if constexpr (D == 2) {
    R[0][0] = F[1][1] * iJ; R[0][1] = dc(0.0) - F[0][1] * iJ;
    R[1][0] = dc(0.0) - F[1][0] * iJ; R[1][1] = F[0][0] * iJ;
  } else {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const int j1 = (j + 1) % 3, j2 = (j + 2) % 3, i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        // (F^-1)_ij = cofactor_ji / J
        R[i][j] = (F[j1][i1] * F[j2][i2] - F[j1][i2] * F[j2][i1]) * iJ;
      }
  }
}

// Previous-level point data (constants: no derivative).
template <int D>
struct Old {
  double vo[D], uo[D], Gvo[D][D], Fo[D][D], Jo, Fio[D][D];
};

template <int D>
__device__ __forceinline__ void old_point(const double* N, const double* dN, const double* Vo, const double* Uo,
                                          bool need_grad, Old<D>& o) {
  constexpr int NQ2 = Sh<D, 0>::NQ2;
  for (int i = 0; i < D; ++i) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < NQ2; ++k) { a += N[k] * Vo[k * D + i]; b += N[k] * Uo[k * D + i]; }
    o.vo[i] = a; o.uo[i] = b;
  }
  o.Jo = 1.0;
  if (!need_grad) return;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      double gv = 0.0, gu = 0.0;
      for (int k = 0; k < NQ2; ++k) { gv += dN[k * D + j] * Vo[k * D + i]; gu += dN[k * D + j] * Uo[k * D + i]; }
      o.Gvo[i][j] = gv;
      o.Fo[i][j] = gu + (i == j ? 1.0 : 0.0);
    }
  D1 Fd[D][D], Rd[D][D];
  for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) Fd[i][j] = dc(o.Fo[i][j]);
  const D1 J = det<D>(Fd);
  o.Jo = J.v;
  invert<D>(Fd, inv(J), Rd);
  for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) o.Fio[i][j] = Rd[i][j].v;
}

// v, u, grad v, grad u at a point as duals seeded along local DOF `dir` (-1: none)
template <int D>
__device__ __forceinline__ void fields(const double* N, const double* dN, const double* U, int dir, D1 (&v)[D],
                                       D1 (&u)[D], D1 (&Gv)[D][D], D1 (&Gu)[D][D]) {
  constexpr int NQ2 = Sh<D, 0>::NQ2;
  for (int i = 0; i < D; ++i) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < NQ2; ++k) { a += N[k] * U[k * D + i]; b += N[k] * U[NQ2 * D + k * D + i]; }
    v[i] = dc(a); u[i] = dc(b);
    for (int j = 0; j < D; ++j) {
      double gv = 0.0, gu = 0.0;
      for (int k = 0; k < NQ2; ++k) { gv += dN[k * D + j] * U[k * D + i]; gu += dN[k * D + j] * U[NQ2 * D + k * D + i]; }
      Gv[i][j] = dc(gv); Gu[i][j] = dc(gu);
    }
  }
  if (dir >= 0 && dir < 2 * NQ2 * D) {
    const bool isv = dir < NQ2 * D;
    const int l = isv ? dir : dir - NQ2 * D;
    const int a = l / D, i = l % D;
    if (isv) {
      v[i].d = N[a];
      for (int j = 0; j < D; ++j) Gv[i][j].d = dN[a * D + j];
    } else {
      u[i].d = N[a];
      for (int j = 0; j < D; ++j) Gu[i][j].d = dN[a * D + j];
    }
  }
}

template <int D, int PD, bool JAC>
__global__ void __launch_bounds__(kAsmThreads) k_assemble(CellGeom geom, int chunk0_stride, Tables T, Phys P,
                                                          const int* __restrict__ cell_dof,
                                                          const unsigned* __restrict__ cell_flags,
                                                          const int64_t* __restrict__ rowptr,
                                                          const int* __restrict__ colind,
                                                          const unsigned char* __restrict__ row_fixed,
                                                          const double* __restrict__ Ug,
                                                          const double* __restrict__ Uold,
                                                          double* __restrict__ out, double* __restrict__ cell_minJ,
                                                          int* __restrict__ err) {
  using E = Sh<D, PD>;
  constexpr int NQ2 = E::NQ2, NQ1 = E::NQ1, NL = E::NL, NQP = E::NQP, NFP = E::NFP;
  constexpr int S = kSlots<D>;
  constexpr int NPT = NQP + NFP;
  constexpr int C = JAC ? E::CHUNK : 1;
  extern __shared__ double smem[];
  double* U = smem;                        // NL
  double* Vo = U + NL;                     // NQ2 * D
  double* Uo = Vo + NQ2 * D;               // NQ2 * D
  double* Q = Uo + NQ2 * D;                // [NPT][C][S]
  __shared__ int gdof[NL];
  __shared__ double jmin[kAsmThreads / 32];

  const int64_t k = blockIdx.x / chunk0_stride;
  const int chunk = blockIdx.x % chunk0_stride;
  int c[3] = {0, 0, 0};
  const int64_t cell = colour_cell<D>(geom, k, c);
  const unsigned flags = cell_flags[cell];
  const bool solid = flags & 1u;
  const bool outflow = (flags & 2u) && !solid;
  const bool prev = P.theta != 1.0;
  const double dtt = P.dt * P.theta, dto = P.dt * (1.0 - P.theta);
  const double mu = P.rho_f * P.nu_f;
  for (int t = threadIdx.x; t < NL; t += blockDim.x) {
    const int g = cell_dof[cell * NL + t];
    gdof[t] = g;
    U[t] = Ug[g];
  }
  for (int t = threadIdx.x; t < NQ2 * D; t += blockDim.x) {
    Vo[t] = Uold ? Uold[cell_dof[cell * NL + t]] : 0.0;
    Uo[t] = Uold ? Uold[cell_dof[cell * NL + NQ2 * D + t]] : 0.0;
  }
  __syncthreads();

  // ---- phase 1: point quantities
  double my_min = 1e300;
  for (int idx = threadIdx.x; idx < NPT * C; idx += blockDim.x) {
    const int pt = idx / C, cc = idx % C;
    const int dir = JAC ? chunk * C + cc : -1;
    double* q = Q + ((size_t)pt * C + cc) * S;
    if (JAC && dir >= NL) {
      for (int s = 0; s < S; ++s) q[s] = 0.0;
      continue;
    }
    const bool face = pt >= NQP;
    if (face && !outflow) continue;
    const double* N = face ? T.Nf + (pt - NQP) * NQ2 : T.N + pt * NQ2;
    const double* dN = face ? T.dNf + (size_t)(pt - NQP) * NQ2 * D : T.dN + (size_t)pt * NQ2 * D;
    D1 v[D], u[D], Gv[D][D], Gu[D][D];
    fields<D>(N, dN, U, dir, v, u, Gv, Gu);
    D1 F[D][D];
    for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) F[i][j] = Gu[i][j] + (i == j ? 1.0 : 0.0);
    const D1 J = det<D>(F);
    if (!face && J.v < my_min) my_min = J.v;
    Old<D> o;
    old_point<D>(N, dN, Vo, Uo, prev, o);
    auto put = [&](int s, D1 x) { q[s] = JAC ? x.d : x.v; };
    if (face) {
      // c_i = -dtt mu J sum_j Fi_ji t_j,  t_j = sum_k (grad v)_kj Fi_0k
      D1 Fi[D][D];
      invert<D>(F, inv(J), Fi);
      D1 t[D];
      for (int j = 0; j < D; ++j) {
        D1 s = dc(0.0);
        for (int kk = 0; kk < D; ++kk) s = s + Gv[kk][j] * Fi[0][kk];
        t[j] = s;
      }
      double to[D] = {};
      if (prev)
        for (int j = 0; j < D; ++j) {
          double s = 0.0;
          for (int kk = 0; kk < D; ++kk) s += o.Gvo[kk][j] * o.Fio[0][kk];
          to[j] = s;
        }
      for (int i = 0; i < D; ++i) {
        D1 b = dc(0.0);
        for (int j = 0; j < D; ++j) b = b + Fi[j][i] * t[j];
        D1 cval = (-dtt * mu) * (J * b);
        if (prev) {
          double s = 0.0;
          for (int j = 0; j < D; ++j) s += o.Fio[j][i] * to[j];
          cval = cval + (-dto * mu * o.Jo * s);
        }
        put(i, cval);
      }
      continue;
    }
    if (!solid) {
      D1 Fi[D][D];
      const D1 iJ = inv(J);
      invert<D>(F, iJ, Fi);
      const double* Np = T.Np + pt * NQ1;
      D1 p = dc(0.0);
      for (int a = 0; a < NQ1; ++a) p = p + Np[a] * dc(U[2 * NQ2 * D + a]);
      if (dir >= 2 * NQ2 * D) p.d = Np[dir - 2 * NQ2 * D];
      D1 A[D][D];
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          D1 s = dc(0.0);
          for (int kk = 0; kk < D; ++kk) s = s + Gv[i][kk] * Fi[kk][j];
          A[i][j] = s;
        }
      double Ao[D][D] = {};
      if (prev)
        for (int i = 0; i < D; ++i)
          for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int kk = 0; kk < D; ++kk) s += o.Gvo[i][kk] * o.Fio[kk][j];
            Ao[i][j] = s;
          }
      for (int i = 0; i < D; ++i) {
        const D1 dv = v[i] - o.vo[i];
        D1 s = dv;
        for (int j = 0; j < D; ++j) s = s - A[i][j] * (u[j] - o.uo[j]) + dtt * (A[i][j] * v[j]);
        D1 f0 = (P.rho_f * J) * s;
        if (prev) {
          double co = 0.0;
          for (int j = 0; j < D; ++j) co += Ao[i][j] * o.vo[j];
          f0 = f0 + (P.rho_f * (1.0 - P.theta)) * (o.Jo * dv - J * dv) + P.rho_f * dto * o.Jo * co;
        }
        put(i, f0);
      }
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          D1 s = dc(0.0);
          for (int kk = 0; kk < D; ++kk) s = s + (A[i][kk] + A[kk][i]) * Fi[j][kk];
          D1 f1 = (dtt * mu) * (J * s) - (J * p) * Fi[j][i];
          if (prev) {
            double so = 0.0;
            for (int kk = 0; kk < D; ++kk) so += (Ao[i][kk] + Ao[kk][i]) * o.Fio[j][kk];
            f1 = f1 + dto * mu * o.Jo * so;
          }
          put(D + i * D + j, f1);
          put(D + D * D + i * D + j, Gu[i][j] * iJ);     // mesh motion: grad(u) / J
        }
      D1 trA = dc(0.0);
      for (int i = 0; i < D; ++i) trA = trA + A[i][i];
      put(D + 2 * D * D, J * trA);
    } else {
      D1 E[D][D];
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          D1 s = dc(0.0);
          for (int kk = 0; kk < D; ++kk) s = s + F[kk][i] * F[kk][j];
          E[i][j] = 0.5 * (s - (i == j ? 1.0 : 0.0));
        }
      D1 trE = dc(0.0);
      for (int i = 0; i < D; ++i) trE = trE + E[i][i];
      D1 Sg[D][D];
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          Sg[i][j] = (2.0 * P.mu_s) * E[i][j];
          if (i == j) Sg[i][j] = Sg[i][j] + P.lambda_s * trE;
        }
      double So[D][D] = {};
      if (prev) {
        double Eo[D][D], trEo = 0.0;
        for (int i = 0; i < D; ++i)
          for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int kk = 0; kk < D; ++kk) s += o.Fo[kk][i] * o.Fo[kk][j];
            Eo[i][j] = 0.5 * (s - (i == j ? 1.0 : 0.0));
          }
        for (int i = 0; i < D; ++i) trEo += Eo[i][i];
        for (int i = 0; i < D; ++i)
          for (int j = 0; j < D; ++j) So[i][j] = 2.0 * P.mu_s * Eo[i][j] + (i == j ? P.lambda_s * trEo : 0.0);
      }
      for (int i = 0; i < D; ++i) {
        put(i, P.rho_s * (v[i] - o.vo[i]));
        D1 k0 = (u[i] - o.uo[i]) - dtt * v[i];
        if (prev) k0 = k0 - dto * o.vo[i];
        put(D + D * D + i, k0);
        for (int j = 0; j < D; ++j) {
          D1 s = dc(0.0);
          for (int kk = 0; kk < D; ++kk) s = s + F[i][kk] * Sg[kk][j];
          D1 f1 = dtt * s;
          if (prev) {
            double so = 0.0;
            for (int kk = 0; kk < D; ++kk) so += o.Fo[i][kk] * So[kk][j];
            f1 = f1 + dto * so;
          }
          put(D + i * D + j, f1);
        }
      }
    }
  }
  // smallest J of the cell's volume points (one value per cell, from the first chunk)
  for (int off = 16; off > 0; off >>= 1) my_min = fmin(my_min, __shfl_down_sync(0xffffffffu, my_min, off));
  if ((threadIdx.x & 31) == 0) jmin[threadIdx.x >> 5] = my_min;
  __syncthreads();
  if (threadIdx.x == 0 && chunk == 0) {
    double m = jmin[0];
    for (int wi = 1; wi < (int)(blockDim.x >> 5); ++wi) m = fmin(m, jmin[wi]);
    cell_minJ[cell] = m;
  }

  // ---- phase 2: element rows x columns, summed over the points
  const int nentries = NL * C;
  for (int e = threadIdx.x; e < nentries; e += blockDim.x) {
    const int r = e / C, cc = e % C;
    const int col = JAC ? chunk * C + cc : -1;
    if (JAC && col >= NL) continue;
    const int gr = gdof[r];
    if (row_fixed[gr]) continue;
    const bool prow = r >= 2 * NQ2 * D;
    const bool urow = !prow && r >= NQ2 * D;
    if (solid && prow) continue;                          // solid cells own no pressure rows
    int a = 0, i = 0;
    if (!prow) { const int l = urow ? r - NQ2 * D : r; a = l / D; i = l % D; }
    if (!solid && urow && !((flags >> (2 + a)) & 1u)) continue;   // fluid cell: mesh rows only
    if (JAC) {
      const int gc = gdof[col];
      if (row_fixed[gc] || (solid && col >= 2 * NQ2 * D)) continue;
    }
    double acc = 0.0;
    for (int pt = 0; pt < NQP; ++pt) {
      const double* q = Q + ((size_t)pt * C + cc) * S;
      const double w = T.w[pt];
      if (prow) {
        acc += w * T.Np[pt * NQ1 + (r - 2 * NQ2 * D)] * q[D + 2 * D * D];
      } else if (!urow) {
        double s = T.N[pt * NQ2 + a] * q[i];
        for (int j = 0; j < D; ++j) s += T.dN[((size_t)pt * NQ2 + a) * D + j] * q[D + i * D + j];
        acc += w * s;
      } else if (solid) {
        acc += w * T.N[pt * NQ2 + a] * q[D + D * D + i];
      } else {
        double s = 0.0;
        for (int j = 0; j < D; ++j) s += T.dN[((size_t)pt * NQ2 + a) * D + j] * q[D + D * D + i * D + j];
        acc += w * s;
      }
    }
    if (outflow && !urow && !prow)
      for (int f = 0; f < NFP; ++f) acc += T.wf[f] * T.Nf[f * NQ2 + a] * Q[((size_t)(NQP + f) * C + cc) * S + i];
    if (!JAC) {
      out[gr] += acc;
      continue;
    }
    const int gc = gdof[col];
    const int* ci = colind + rowptr[gr];
    const int len = (int)(rowptr[gr + 1] - rowptr[gr]);
    int lo = 0, hi = len;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ci[mid] < gc) lo = mid + 1; else hi = mid;
    }
    if (lo < len && ci[lo] == gc) out[rowptr[gr] + lo] += acc;
    else if (acc != 0.0) atomicExch(err, 1);                // an entry outside the pattern
  }
}

// fixed rows: identity entry (Jacobian) or zero (residual)
__global__ void k_fixed_rows(int64_t n, const int64_t* __restrict__ rowptr, const unsigned char* __restrict__ fixed,
                             double* __restrict__ out, int jac) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n || !fixed[r]) return;
  if (jac) out[rowptr[r]] = 1.0; else out[r] = 0.0;
}

__global__ void k_min_reduce(int64_t n, const double* __restrict__ x, double* __restrict__ out) {
  __shared__ double sh[32];
  double m = 1e300;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmin(m, x[i]);
  for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmin(m, sh[w]);
    out[0] = fmin(m, sh[0]);
  }
}

// max |R_i| over the rows (deterministic: fixed blocks, fixed order)
__global__ void k_absmax_partial(int64_t n, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sh[32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  double m = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) m = fmax(m, fabs(x[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    part[blockIdx.x] = m;
  }
}

__global__ void k_axpy_inplace(int64_t n, double alpha, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += alpha * x[i];
}

// ------------------------------------------------------------------ host tables
double q2b(int a, double x) { return a == 0 ? 2.0 * (x - 0.5) * (x - 1.0) : a == 1 ? -4.0 * x * (x - 1.0) : 2.0 * x * (x - 0.5); }
double q2d(int a, double x) { return a == 0 ? 4.0 * x - 3.0 : a == 1 ? 4.0 - 8.0 * x : 4.0 * x - 1.0; }
double q1b(int a, double x) { return a == 0 ? 1.0 - x : x; }

}  // namespace

struct Assembler {
  int dim = 2;
  int pdisc = 0;                  // pressure: 0 continuous Q1, 1 discontinuous P1
  int64_t n = 0, ncell = 0;
  int ncd[3] = {1, 1, 1};
  Phys phys{};
  cudaStream_t s = nullptr;
  bool own_stream = false;
  DBuf<double> tab;               // N, dN, Np, w, Nf, dNf, wf
  Tables T{};
  DBuf<int> cell_dof;
  DBuf<unsigned> cell_flags;
  DBuf<int64_t> rowptr;
  DBuf<int> colind;
  DBuf<unsigned char> fixed;
  DBuf<double> cell_minJ, scal, part;
  DBuf<int> err;
  int64_t nnz = 0;
  std::string msg;
  ~Assembler() {
    if (own_stream && s) cudaStreamDestroy(s);
  }
};

namespace {

void build_tables(Assembler& A, const double* h) {
  const int D = A.dim;
  const int NQ2 = D == 2 ? 9 : 27, NQ1 = A.pdisc ? D + 1 : (D == 2 ? 4 : 8), NQP = NQ2, NFP = D == 2 ? 3 : 9;
  // 3-point Gauss-Legendre rule on [0, 1]: nodes 1/2 -+ sqrt(3/5)/2, weights 5/18, 8/18, 5/18
  const double r = std::sqrt(0.6);
  const double gx[3] = {0.5 - 0.5 * r, 0.5, 0.5 + 0.5 * r};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  std::vector<double> N(NQP * NQ2), dN(NQP * NQ2 * D), Np(NQP * NQ1), w(NQP);
  std::vector<double> Nf(NFP * NQ2), dNf(NFP * NQ2 * D), wf(NFP);
  double vol = 1.0;
  for (int d = 0; d < D; ++d) vol *= h[d];
  auto basis = [&](const double* xi, double* Nrow, double* dNrow, double* Nprow) {
    for (int a = 0; a < NQ2; ++a) {
      const int ai[3] = {a % 3, (a / 3) % 3, a / 9};
      double val = 1.0;
      for (int d = 0; d < D; ++d) val *= q2b(ai[d], xi[d]);
      Nrow[a] = val;
      for (int j = 0; j < D; ++j) {
        double g = 1.0;
        for (int d = 0; d < D; ++d) g *= (d == j) ? q2d(ai[d], xi[d]) / h[d] : q2b(ai[d], xi[d]);
        dNrow[a * D + j] = g;
      }
    }
    if (Nprow)
      for (int a = 0; a < NQ1; ++a) {
        double val = 1.0;
        if (A.pdisc) {
          val = a == 0 ? 1.0 : 2.0 * xi[a - 1] - 1.0;   // P1disc: 1 and the centred linears of the cell
        } else {
          const int ai[3] = {a % 2, (a / 2) % 2, a / 4};
          for (int d = 0; d < D; ++d) val *= q1b(ai[d], xi[d]);
        }
        Nprow[a] = val;
      }
  };
  for (int q = 0; q < NQP; ++q) {
    const int qi[3] = {q % 3, (q / 3) % 3, q / 9};
    double xi[3] = {0, 0, 0}, ww = vol;
    for (int d = 0; d < D; ++d) { xi[d] = gx[qi[d]]; ww *= gw[qi[d]]; }
    w[q] = ww;
    basis(xi, &N[q * NQ2], &dN[(size_t)q * NQ2 * D], &Np[q * NQ1]);
  }
  double area = 1.0;
  for (int d = 1; d < D; ++d) area *= h[d];
  for (int f = 0; f < NFP; ++f) {
    const int fi[2] = {f % 3, f / 3};
    double xi[3] = {1.0, 0.0, 0.0}, ww = area;
    for (int d = 1; d < D; ++d) { xi[d] = gx[fi[d - 1]]; ww *= gw[fi[d - 1]]; }
    wf[f] = ww;
    basis(xi, &Nf[f * NQ2], &dNf[(size_t)f * NQ2 * D], nullptr);
  }
  std::vector<double> all;
  size_t off[7];
  const std::vector<double>* parts[7] = {&N, &dN, &Np, &w, &Nf, &dNf, &wf};
  for (int t = 0; t < 7; ++t) {
    off[t] = all.size();
    all.insert(all.end(), parts[t]->begin(), parts[t]->end());
  }
  A.tab.alloc(all.size());
  FSI_CUDA(cudaMemcpyAsync(A.tab.p, all.data(), sizeof(double) * all.size(), cudaMemcpyHostToDevice, A.s));
  FSI_CUDA(cudaStreamSynchronize(A.s));
  A.T = Tables{A.tab.p + off[0], A.tab.p + off[1], A.tab.p + off[2], A.tab.p + off[3],
               A.tab.p + off[4], A.tab.p + off[5], A.tab.p + off[6]};
}

template <int D, int PD, bool JAC>
size_t smem_bytes() {
  using E = Sh<D, PD>;
  constexpr int C = JAC ? E::CHUNK : 1;
  return sizeof(double) * (E::NL + 2 * E::NQ2 * D + (size_t)(E::NQP + E::NFP) * C * kSlots<D>);
}

template <int D, int PD, bool JAC>
void run_colours(Assembler& A, const double* U, const double* Uold, double* out) {
  using E = Sh<D, PD>;
  const size_t sm = smem_bytes<D, PD, JAC>();
  FSI_CUDA(cudaFuncSetAttribute(k_assemble<D, PD, JAC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const int chunks = JAC ? (E::NL + E::CHUNK - 1) / E::CHUNK : 1;
  for (int col = 0; col < (1 << D); ++col) {
    CellGeom g{};
    int64_t cnt = 1;
    for (int d = 0; d < 3; ++d) {
      g.n[d] = A.ncd[d];
      if (d < D) {
        const int b = (col >> d) & 1;
        g.m[d] = (A.ncd[d] - b + 1) / 2;
        cnt *= g.m[d];
      } else {
        g.m[d] = 1;
      }
    }
    g.color = col;
    if (cnt == 0) continue;
    const int64_t blocks = cnt * chunks;
    require(blocks < ((int64_t)1 << 31), "fsi_asm: too many cells for one launch");
    k_assemble<D, PD, JAC><<<(unsigned)blocks, kAsmThreads, sm, A.s>>>(g, chunks, A.T, A.phys, A.cell_dof.p,
                                                                    A.cell_flags.p, A.rowptr.p, A.colind.p, A.fixed.p,
                                                                    U, Uold, out, A.cell_minJ.p, A.err.p);
    FSI_CHECK_LAUNCH();
  }
}

double finish(Assembler& A, double* out, bool jac, double* minJ) {
  k_fixed_rows<<<div_up(A.n, 256), 256, 0, A.s>>>(A.n, A.rowptr.p, A.fixed.p, out, jac ? 1 : 0);
  FSI_CHECK_LAUNCH();
  k_min_reduce<<<1, 1024, 0, A.s>>>(A.ncell, A.cell_minJ.p, A.scal.p);
  FSI_CHECK_LAUNCH();
  double h[2] = {0, 0};
  int e = 0;
  FSI_CUDA(cudaMemcpyAsync(&h[0], A.scal.p, sizeof(double), cudaMemcpyDeviceToHost, A.s));
  FSI_CUDA(cudaMemcpyAsync(&e, A.err.p, sizeof(int), cudaMemcpyDeviceToHost, A.s));
  FSI_CUDA(cudaStreamSynchronize(A.s));
  if (minJ) *minJ = h[0];
  require(e == 0, "fsi_asm: a Jacobian entry falls outside the CSR pattern");
  return h[0];
}

}  // namespace

void asm_residual(Assembler& A, const double* U, const double* Uold, double* R, double* minJ, double* rmax) {
  FSI_CUDA(cudaMemsetAsync(R, 0, sizeof(double) * A.n, A.s));
  FSI_CUDA(cudaMemsetAsync(A.err.p, 0, sizeof(int), A.s));
  if (A.dim == 2) {
    if (A.pdisc) run_colours<2, 1, false>(A, U, Uold, R); else run_colours<2, 0, false>(A, U, Uold, R);
  } else {
    if (A.pdisc) run_colours<3, 1, false>(A, U, Uold, R); else run_colours<3, 0, false>(A, U, Uold, R);
  }
  finish(A, R, false, minJ);
  if (rmax) {
    const int nb = 256;
    k_absmax_partial<<<nb, 256, 0, A.s>>>(A.n, R, A.part.p);
    FSI_CHECK_LAUNCH();
    std::vector<double> hp(nb);
    FSI_CUDA(cudaMemcpyAsync(hp.data(), A.part.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, A.s));
    FSI_CUDA(cudaStreamSynchronize(A.s));
    double m = 0.0;
    for (double v : hp) m = v > m ? v : m;
    *rmax = m;
  }
}

void asm_jacobian(Assembler& A, const double* U, const double* Uold, double* vals, double* minJ) {
  FSI_CUDA(cudaMemsetAsync(vals, 0, sizeof(double) * A.nnz, A.s));
  FSI_CUDA(cudaMemsetAsync(A.err.p, 0, sizeof(int), A.s));
  if (A.dim == 2) {
    if (A.pdisc) run_colours<2, 1, true>(A, U, Uold, vals); else run_colours<2, 0, true>(A, U, Uold, vals);
  } else {
    if (A.pdisc) run_colours<3, 1, true>(A, U, Uold, vals); else run_colours<3, 0, true>(A, U, Uold, vals);
  }
  finish(A, vals, true, minJ);
}

void asm_axpy(Assembler& A, double alpha, const double* x, double* y) {
  const int cap = device_sms() * 16;
  k_axpy_inplace<<<div_up(A.n, 256) < cap ? div_up(A.n, 256) : cap, 256, 0, A.s>>>(A.n, alpha, x, y);
  FSI_CHECK_LAUNCH();
  FSI_CUDA(cudaStreamSynchronize(A.s));
}

void asm_create(Assembler& A, const fsi_asm_mesh& m, const fsi_asm_physics& p, void* stream) {
  require(m.dim == 2 || m.dim == 3, "fsi_asm: dim must be 2 or 3");
  require(m.n > 0 && m.n < ((int64_t)1 << 31), "fsi_asm: n out of range");
  require(m.cell_dof && m.cell_flags && m.rowptr && m.colind && m.row_fixed, "fsi_asm: null mesh array");
  require(m.pressure == 0 || m.pressure == 1, "fsi_asm: pressure must be 0 (continuous Q1) or 1 (P1disc)");
  A.dim = m.dim;
  A.pdisc = m.pressure;
  A.n = m.n;
  A.ncell = 1;
  for (int d = 0; d < m.dim; ++d) {
    require(m.cells[d] >= 1 && m.h[d] > 0.0, "fsi_asm: cells and h must be positive");
    A.ncd[d] = m.cells[d];
    A.ncell *= m.cells[d];
  }
  require(p.theta > 0.0 && p.theta <= 1.0 && p.dt > 0.0, "fsi_asm: need 0 < theta <= 1 and dt > 0");
  A.phys = Phys{p.rho_f, p.nu_f, p.mu_s, p.lambda_s, p.rho_s, p.dt, p.theta};
  if (stream) {
    A.s = static_cast<cudaStream_t>(stream);
  } else {
    FSI_CUDA(cudaStreamCreateWithFlags(&A.s, cudaStreamNonBlocking));
    A.own_stream = true;
  }
  const int NL = 2 * (m.dim == 2 ? 9 : 27) * m.dim + (m.pressure ? m.dim + 1 : (m.dim == 2 ? 4 : 8));
  A.nnz = m.rowptr[m.n];
  for (int64_t c = 0; c < A.ncell * NL; ++c)
    require(m.cell_dof[c] >= 0 && m.cell_dof[c] < m.n, "fsi_asm: cell DOF out of range");
  build_tables(A, m.h);
  A.cell_dof.alloc((size_t)A.ncell * NL);
  A.cell_flags.alloc(A.ncell);
  A.rowptr.alloc(A.n + 1);
  A.colind.alloc(A.nnz > 0 ? A.nnz : 1);
  A.fixed.alloc(A.n);
  A.cell_minJ.alloc(A.ncell);
  A.scal.alloc(2);
  A.part.alloc(256);
  A.err.alloc(1);
  FSI_CUDA(cudaMemcpyAsync(A.cell_dof.p, m.cell_dof, sizeof(int) * A.ncell * NL, cudaMemcpyHostToDevice, A.s));
  FSI_CUDA(cudaMemcpyAsync(A.cell_flags.p, m.cell_flags, sizeof(unsigned) * A.ncell, cudaMemcpyHostToDevice, A.s));
  FSI_CUDA(cudaMemcpyAsync(A.rowptr.p, m.rowptr, sizeof(int64_t) * (A.n + 1), cudaMemcpyHostToDevice, A.s));
  if (A.nnz) FSI_CUDA(cudaMemcpyAsync(A.colind.p, m.colind, sizeof(int) * A.nnz, cudaMemcpyHostToDevice, A.s));
  FSI_CUDA(cudaMemcpyAsync(A.fixed.p, m.row_fixed, A.n, cudaMemcpyHostToDevice, A.s));
  FSI_CUDA(cudaStreamSynchronize(A.s));
}

}  // namespace fsi

// ====================================================================== C ABI
struct fsi_asm {
  fsi::Assembler A;
};

namespace {
thread_local std::string g_asm_create_error;

template <class F>
int asm_guarded(fsi_asm* a, F&& f) {
  std::string& err = a ? a->A.msg : g_asm_create_error;
  try {
    f();
    err.clear();
    return FSI_OK;
  } catch (const fsi::Error& e) {
    err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    err = e.what();
    return FSI_ECUDA;
  }
}
}  // namespace

extern "C" {

int fsi_asm_create(fsi_asm** out, const fsi_asm_mesh* mesh, const fsi_asm_physics* phys, void* cuda_stream) {
  if (!out) return FSI_EINVAL;
  *out = nullptr;
  if (!mesh || !phys) return FSI_EINVAL;
  fsi_asm* a = nullptr;
  try {
    a = new fsi_asm();
  } catch (...) {
    return FSI_ENOMEM;
  }
  const int rc = asm_guarded(nullptr, [&] { fsi::asm_create(a->A, *mesh, *phys, cuda_stream); });
  if (rc != FSI_OK) {
    delete a;
    return rc;
  }
  *out = a;
  return FSI_OK;
}

int fsi_asm_residual(fsi_asm* a, const double* U_dev, const double* Uold_dev, double* R_dev, double* min_J,
                     double* r_absmax) {
  if (!a) return FSI_EINVAL;
  return asm_guarded(a, [&] {
    fsi::require(U_dev && R_dev, "fsi_asm_residual: null vector");
    fsi::asm_residual(a->A, U_dev, Uold_dev, R_dev, min_J, r_absmax);
  });
}

int fsi_asm_jacobian(fsi_asm* a, const double* U_dev, const double* Uold_dev, double* vals_dev, double* min_J) {
  if (!a) return FSI_EINVAL;
  return asm_guarded(a, [&] {
    fsi::require(U_dev && vals_dev, "fsi_asm_jacobian: null vector");
    fsi::asm_jacobian(a->A, U_dev, Uold_dev, vals_dev, min_J);
  });
}

int fsi_asm_axpy(fsi_asm* a, double alpha, const double* x_dev, double* y_dev) {
  if (!a) return FSI_EINVAL;
  return asm_guarded(a, [&] {
    fsi::require(x_dev && y_dev, "fsi_asm_axpy: null vector");
    fsi::asm_axpy(a->A, alpha, x_dev, y_dev);
  });
}

const char* fsi_asm_last_error(const fsi_asm* a) { return a ? a->A.msg.c_str() : g_asm_create_error.c_str(); }

void fsi_asm_free(fsi_asm* a) { delete a; }

}  // extern "C"

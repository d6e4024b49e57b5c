// Seeded FSI problem generator: residual and Jacobian of the monolithic ALE
// fluid-structure system on a structured box mesh.
//
// This file produces the INPUT of the linear solve (the matrix A_h of Eq.
// (mat:small), Sec. 3.4).  It contains no solver arithmetic.  Both the CPU
// oracle and the CUDA library consume the CSR it writes.
//
// Physics (Sec. 2, Form. 2.1 and the variational form Eq. (weak:FSI), with the
// time-discrete semilinear form Eq. (fsi:all), Sec. 3.2-3.3):
//   fluid momentum   (rho_f J (v - v_old), phi) - (rho_f J grad(v) F^-1 (u - u_old), phi)
//                    + dt*theta [ (rho_f J grad(v) F^-1 v, phi) + (J sigma_v F^-T, grad phi) ]
//                    - dt*theta < rho_f nu_f J F^-T grad(v)^T F^-T n, phi >_{Gamma_out}
//                    + (J (-p) F^-T, grad phi)
//   incompressibility (J tr(grad(v) F^-1), psi)               (weak form, Eq. weak:FSI)
//   solid momentum   (rho_s (v - v_old), phi) + dt*theta (F Sigma, grad phi)
//   solid kinematics (u - u_old - dt*theta v, phi)_s
//   mesh motion      (1/J grad u, grad phi)_f, test functions vanishing on the
//                    closed solid region (Sec. 3.1: the displacement test
//                    functions vanish on the interface).
// with F = I + grad u, J = det F, sigma_v = rho_f nu_f (grad v F^-1 + F^-T grad v^T),
// Sigma = 2 mu E + lambda tr(E) I, E = (F^T F - I)/2 (Sec. 2).
// Theta scheme, 0 < theta <= 1 (Sec. 3.2): the convection, viscous-stress,
// outflow and solid-stress terms and the kinematic velocity are weighted
// dt*theta at the new and dt*(1-theta) at the previous time level; the pressure,
// the incompressibility constraint and the mesh motion stay fully implicit; the
// fluid time derivative carries J^theta = theta J + (1-theta) J_old.  theta = 1
// is backward Euler (every previous-level term vanishes, J^theta = J),
// theta = 1/2 Crank-Nicolson, theta = 1/2 + dt the shifted variant.
//
// Discretisation: Q2 velocity and displacement; pressure either continuous Q1 on
// the whole box (nodes at cell vertices; the configurations' default) or the
// paper's discontinuous P1 (Sec. 3.4: Q2-Q2-P1disc), one linear polynomial per
// fluid cell, p = p_0 + p_1 (2 xi_1 - 1) + ... + p_d (2 xi_d - 1) in the cell's
// reference coordinates xi (linear in x on the affine box cells), no pressure in
// solid cells; 3^d Gauss points per cell.  The Jacobian
// is the exact derivative of the discrete residual, taken by forward-mode
// dual numbers per cell (Thm. 3.3 lists the derivatives this reproduces).
//
// DOF classes and order (block structure of Eq. mat:small, global variables of
// Sec. 5.2): m = u at nodes outside the closed solid region, s_v = v and
// s_u = u at nodes of the closed solid region (interface included), f_v = v at
// nodes outside it, f_p = p at every Q1 node.  Vector classes are node-major,
// component-minor.  Dirichlet DOFs and p nodes touching no fluid cell are
// identity rows with zeroed columns.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <vector>
#include <algorithm>
#include <string>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- dual numbers
template <int N>
struct Dual {
  double v;
  double d[N];
};

template <int N> inline Dual<N> dconst(double a) { Dual<N> r; r.v = a; for (int k = 0; k < N; ++k) r.d[k] = 0.0; return r; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v + b.v; for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v - b.v; for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a) { Dual<N> r; r.v = -a.v; for (int k = 0; k < N; ++k) r.d[k] = -a.d[k]; return r; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) { Dual<N> r; r.v = a.v * b.v; for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
template <int N> inline Dual<N> operator*(double s, const Dual<N>& a) { Dual<N> r; r.v = s * a.v; for (int k = 0; k < N; ++k) r.d[k] = s * a.d[k]; return r; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double s) { return s * a; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, double s) { Dual<N> r = a; r.v += s; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double s) { Dual<N> r = a; r.v -= s; return r; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; double ib = 1.0 / b.v; r.v = a.v * ib;
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <int N> inline Dual<N> operator/(double s, const Dual<N>& b) {
  Dual<N> r; double ib = 1.0 / b.v; r.v = s * ib;
  for (int k = 0; k < N; ++k) r.d[k] = -r.v * b.d[k] * ib;
  return r;
}
template <int N> inline Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a.v += b.v; for (int k = 0; k < N; ++k) a.d[k] += b.d[k]; return a; }
// a += s * b  (s plain)
template <int N> inline void axpy(Dual<N>& a, double s, const Dual<N>& b) { a.v += s * b.v; for (int k = 0; k < N; ++k) a.d[k] += s * b.d[k]; }
inline double dconstd(double a) { return a; }
inline void axpy(double& a, double s, double b) { a += s * b; }
inline double value_of(double a) { return a; }
template <int N> inline double value_of(const Dual<N>& a) { return a.v; }

template <class T> struct Zero { static T get() { return T(0.0); } };
template <int N> struct Zero<Dual<N>> { static Dual<N> get() { return dconst<N>(0.0); } };

// ----------------------------------------------------------------- parameters
struct Params {
  int dim;
  int n[3];          // cells per direction
  double L[3];       // box lengths
  double solid_h;    // solid = cells whose centroid has last coordinate < solid_h
  double rho_f, nu_f, mu_s, lambda_s, rho_s, dt, theta;
  int pressure;      // 0: continuous Q1, 1: discontinuous P1 (Q2-Q2-P1disc)
};

// 1D Q2 Lagrange basis on [0,1] with nodes 0, 1/2, 1, and derivatives.
inline double q2(int a, double x) {
  switch (a) { case 0: return 2.0 * (x - 0.5) * (x - 1.0); case 1: return -4.0 * x * (x - 1.0); default: return 2.0 * x * (x - 0.5); }
}
inline double dq2(int a, double x) {
  switch (a) { case 0: return 4.0 * x - 3.0; case 1: return -8.0 * x + 4.0; default: return 4.0 * x - 1.0; }
}
inline double q1(int a, double x) { return a == 0 ? 1.0 - x : x; }

// 3-point Gauss rule on [0,1].
const double GX[3] = {0.5 - 0.5 * 0.7745966692414834, 0.5, 0.5 + 0.5 * 0.7745966692414834};
const double GW[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};

struct Problem {
  Params P;
  int dim;
  int nq2[3];   // Q2 nodes per direction (2n+1)
  int nq1[3];   // Q1 nodes per direction (n+1)
  int64_t n_q2, n_q1, n_cells;
  std::vector<uint8_t> cell_solid;     // per cell
  std::vector<uint8_t> node_solid;     // Q2 node in the closed solid region
  std::vector<uint8_t> node_vdir;      // Q2 node: v Dirichlet
  std::vector<uint8_t> node_udir;      // Q2 node: u Dirichlet
  std::vector<uint8_t> p_active;       // Q1 node touches a fluid cell
  std::vector<int64_t> dof_v, dof_u;   // Q2 node -> first global DOF of its v / u block
  std::vector<int64_t> dof_p;          // Q1 node -> global DOF (continuous Q1 pressure)
  std::vector<int64_t> cell_pdof;      // cell -> first of its d+1 pressure DOFs, -1 in solid cells (P1disc)
  bool pdisc = false;                  // discontinuous P1 pressure
  int64_t off[6];                      // m | s_v | s_u | f_v | f_p | n
  int64_t ndof;
  // CSR pattern
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colind;
  std::vector<uint8_t> row_fixed;      // identity row (Dirichlet or inactive p)
  std::string err;
  // element tables
  int nloc, nq2loc, nq1loc, nqp, nfqp;
  std::vector<double> Nq, dNq, Npq, wq;   // volume quadrature tables
  std::vector<double> Nf, dNf, Npf, wf;   // outflow-face quadrature tables (face x0 = 1)
};

inline int64_t q2_index(const Problem& p, const int* ijk) {
  int64_t idx = ijk[p.dim - 1];
  for (int d = p.dim - 2; d >= 0; --d) idx = idx * p.nq2[d] + ijk[d];
  return idx;
}
inline int64_t q1_index(const Problem& p, const int* ijk) {
  int64_t idx = ijk[p.dim - 1];
  for (int d = p.dim - 2; d >= 0; --d) idx = idx * p.nq1[d] + ijk[d];
  return idx;
}
inline int64_t cell_index(const Problem& p, const int* c) {
  int64_t idx = c[p.dim - 1];
  for (int d = p.dim - 2; d >= 0; --d) idx = idx * p.P.n[d] + c[d];
  return idx;
}
inline void unflatten(int64_t idx, const int* ext, int dim, int* out) {
  for (int d = 0; d < dim; ++d) { out[d] = (int)(idx % ext[d]); idx /= ext[d]; }
}

// Range of cells along one direction that contain Q2 node coordinate i.
inline void cells_of_q2(int i, int ncell, int& lo, int& hi) {
  if (i % 2 == 1) { lo = hi = (i - 1) / 2; return; }
  lo = std::max(0, i / 2 - 1); hi = std::min(ncell - 1, i / 2);
}
inline void cells_of_q1(int i, int ncell, int& lo, int& hi) {
  lo = std::max(0, i - 1); hi = std::min(ncell - 1, i);
}

void build_tables(Problem& p) {
  const int D = p.dim;
  p.nq2loc = (D == 2) ? 9 : 27;
  p.nq1loc = p.pdisc ? D + 1 : ((D == 2) ? 4 : 8);   // pressure basis functions per cell
  p.nloc = 2 * p.nq2loc * D + p.nq1loc;
  p.nqp = (D == 2) ? 9 : 27;
  p.nfqp = (D == 2) ? 3 : 9;
  double h[3];
  for (int d = 0; d < D; ++d) h[d] = p.P.L[d] / p.P.n[d];
  double vol = 1.0; for (int d = 0; d < D; ++d) vol *= h[d];
  p.Nq.assign(p.nqp * p.nq2loc, 0); p.dNq.assign(p.nqp * p.nq2loc * D, 0); p.Npq.assign(p.nqp * p.nq1loc, 0); p.wq.assign(p.nqp, 0);
  for (int q = 0; q < p.nqp; ++q) {
    int qi[3] = {q % 3, (q / 3) % 3, q / 9};
    double xi[3], w = vol;
    for (int d = 0; d < D; ++d) { xi[d] = GX[qi[d]]; w *= GW[qi[d]]; }
    p.wq[q] = w;
    for (int a = 0; a < p.nq2loc; ++a) {
      int ai[3] = {a % 3, (a / 3) % 3, a / 9};
      double val = 1.0;
      for (int d = 0; d < D; ++d) val *= q2(ai[d], xi[d]);
      p.Nq[q * p.nq2loc + a] = val;
      for (int j = 0; j < D; ++j) {
        double g = 1.0;
        for (int d = 0; d < D; ++d) g *= (d == j) ? dq2(ai[d], xi[d]) / h[d] : q2(ai[d], xi[d]);
        p.dNq[(q * p.nq2loc + a) * D + j] = g;
      }
    }
    for (int a = 0; a < p.nq1loc; ++a) {
      double val = 1.0;
      if (p.pdisc) {
        val = (a == 0) ? 1.0 : 2.0 * xi[a - 1] - 1.0;
      } else {
        int ai[3] = {a % 2, (a / 2) % 2, a / 4};
        for (int d = 0; d < D; ++d) val *= q1(ai[d], xi[d]);
      }
      p.Npq[q * p.nq1loc + a] = val;
    }
  }
  // outflow face x0 = 1 (the cell's right face); Gauss points in the other directions
  double area = 1.0; for (int d = 1; d < D; ++d) area *= h[d];
  p.Nf.assign(p.nfqp * p.nq2loc, 0); p.dNf.assign(p.nfqp * p.nq2loc * D, 0); p.Npf.assign(p.nfqp * p.nq1loc, 0); p.wf.assign(p.nfqp, 0);
  for (int q = 0; q < p.nfqp; ++q) {
    int qi[2] = {q % 3, q / 3};
    double xi[3], w = area;
    xi[0] = 1.0;
    for (int d = 1; d < D; ++d) { xi[d] = GX[qi[d - 1]]; w *= GW[qi[d - 1]]; }
    p.wf[q] = w;
    for (int a = 0; a < p.nq2loc; ++a) {
      int ai[3] = {a % 3, (a / 3) % 3, a / 9};
      double val = 1.0;
      for (int d = 0; d < D; ++d) val *= q2(ai[d], xi[d]);
      p.Nf[q * p.nq2loc + a] = val;
      for (int j = 0; j < D; ++j) {
        double g = 1.0;
        for (int d = 0; d < D; ++d) g *= (d == j) ? dq2(ai[d], xi[d]) / h[d] : q2(ai[d], xi[d]);
        p.dNf[(q * p.nq2loc + a) * D + j] = g;
      }
    }
  }
}

// -------------------------------------------------------------- small tensors
template <class T, int D> struct Mat { T a[D][D]; };

template <class T, int D>
inline T det(const Mat<T, D>& F) {
  if constexpr (D == 2) return F.a[0][0] * F.a[1][1] - F.a[0][1] * F.a[1][0];
  else return F.a[0][0] * (F.a[1][1] * F.a[2][2] - F.a[1][2] * F.a[2][1])
            - F.a[0][1] * (F.a[1][0] * F.a[2][2] - F.a[1][2] * F.a[2][0])
            + F.a[0][2] * (F.a[1][0] * F.a[2][1] - F.a[1][1] * F.a[2][0]);
}
template <class T, int D>
inline Mat<T, D> inverse(const Mat<T, D>& F, const T& J) {
  Mat<T, D> R;
  T iJ = 1.0 / J;
  if constexpr (D == 2) {
    R.a[0][0] = F.a[1][1] * iJ; R.a[0][1] = -F.a[0][1] * iJ;
    R.a[1][0] = -F.a[1][0] * iJ; R.a[1][1] = F.a[0][0] * iJ;
  } else {
    R.a[0][0] = (F.a[1][1] * F.a[2][2] - F.a[1][2] * F.a[2][1]) * iJ;
    R.a[0][1] = (F.a[0][2] * F.a[2][1] - F.a[0][1] * F.a[2][2]) * iJ;
    R.a[0][2] = (F.a[0][1] * F.a[1][2] - F.a[0][2] * F.a[1][1]) * iJ;
    R.a[1][0] = (F.a[1][2] * F.a[2][0] - F.a[1][0] * F.a[2][2]) * iJ;
    R.a[1][1] = (F.a[0][0] * F.a[2][2] - F.a[0][2] * F.a[2][0]) * iJ;
    R.a[1][2] = (F.a[0][2] * F.a[1][0] - F.a[0][0] * F.a[1][2]) * iJ;
    R.a[2][0] = (F.a[1][0] * F.a[2][1] - F.a[1][1] * F.a[2][0]) * iJ;
    R.a[2][1] = (F.a[0][1] * F.a[2][0] - F.a[0][0] * F.a[2][1]) * iJ;
    R.a[2][2] = (F.a[0][0] * F.a[1][1] - F.a[0][1] * F.a[1][0]) * iJ;
  }
  return R;
}

// ------------------------------------------------------------ cell residual
// Local DOF layout: v of node a comp i at a*D+i; u at NQ2*D + a*D+i; p of
// vertex P at 2*NQ2*D + P.  `mesh_row[a]` is 1 when node a carries a mesh-motion
// row (outside the closed solid region), `outflow` when the cell's x0=1 face
// lies on the do-nothing boundary.
template <int D, class T>
void cell_residual(const Problem& pb, bool solid, bool outflow, const uint8_t* mesh_row,
                   const T* U, const double* Vold, const double* Uold, T* R, double* minJ) {
  constexpr int NQ2 = (D == 2) ? 9 : 27;
  const int NQ1 = pb.nq1loc;   // pressure basis functions of the cell
  const Params& P = pb.P;
  const int NL = 2 * NQ2 * D + NQ1;
  const T zero = Zero<T>::get();
  for (int k = 0; k < NL; ++k) R[k] = zero;
  const T* Uv = U;
  const T* Uu = U + NQ2 * D;
  const T* Up = U + 2 * NQ2 * D;
  T* Rv = R;
  T* Ru = R + NQ2 * D;
  T* Rp = R + 2 * NQ2 * D;
  const double dtt = P.dt * P.theta;
  const bool prev = P.theta != 1.0;           // previous-level terms present
  const double dto = P.dt * (1.0 - P.theta);

  for (int q = 0; q < pb.nqp; ++q) {
    const double* N = &pb.Nq[q * NQ2];
    const double* dN = &pb.dNq[q * NQ2 * D];
    const double* Np = &pb.Npq[q * NQ1];
    const double w = pb.wq[q];
    T v[D], u[D];
    double vo[D], uo[D];
    Mat<T, D> Gv, Gu;
    for (int i = 0; i < D; ++i) {
      v[i] = zero; u[i] = zero; vo[i] = 0.0; uo[i] = 0.0;
      for (int j = 0; j < D; ++j) { Gv.a[i][j] = zero; Gu.a[i][j] = zero; }
    }
    for (int a = 0; a < NQ2; ++a) {
      for (int i = 0; i < D; ++i) {
        axpy(v[i], N[a], Uv[a * D + i]);
        axpy(u[i], N[a], Uu[a * D + i]);
        vo[i] += N[a] * Vold[a * D + i];
        uo[i] += N[a] * Uold[a * D + i];
        for (int j = 0; j < D; ++j) {
          axpy(Gv.a[i][j], dN[a * D + j], Uv[a * D + i]);
          axpy(Gu.a[i][j], dN[a * D + j], Uu[a * D + i]);
        }
      }
    }
    Mat<T, D> F;
    for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) F.a[i][j] = Gu.a[i][j] + (i == j ? 1.0 : 0.0);
    T J = det<T, D>(F);
    if (value_of(J) < *minJ) *minJ = value_of(J);
    // previous time level (theta < 1): gradients, F_old, J_old
    Mat<double, D> Gvo, Fo;
    double Jo = 1.0;
    if (prev) {
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          double gv = 0.0, gu = 0.0;
          for (int a = 0; a < NQ2; ++a) {
            gv += dN[a * D + j] * Vold[a * D + i];
            gu += dN[a * D + j] * Uold[a * D + i];
          }
          Gvo.a[i][j] = gv;
          Fo.a[i][j] = gu + (i == j ? 1.0 : 0.0);
        }
      Jo = det<double, D>(Fo);
    }
    if (!solid) {
      Mat<T, D> Fi = inverse<T, D>(F, J);
      T p = zero;
      for (int a = 0; a < NQ1; ++a) axpy(p, Np[a], Up[a]);
      // A = grad(v) F^-1
      Mat<T, D> A;
      for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) {
        T s = zero;
        for (int k = 0; k < D; ++k) s += Gv.a[i][k] * Fi.a[k][j];
        A.a[i][j] = s;
      }
      // f0 = rho_f J [ (v - v_old) - A (u - u_old) + dt*theta A v ]
      T f0[D];
      for (int i = 0; i < D; ++i) {
        T s = v[i] - vo[i];
        for (int j = 0; j < D; ++j) s = s - A.a[i][j] * (u[j] - uo[j]) + dtt * (A.a[i][j] * v[j]);
        f0[i] = (P.rho_f * J) * s;
      }
      // f1 = dt*theta J sigma_v F^-T - J p F^-T,  sigma_v = rho_f nu_f (A + A^T)
      T f1[D][D];
      const double mu = P.rho_f * P.nu_f;
      for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) {
        T s = zero;
        for (int k = 0; k < D; ++k) s += (A.a[i][k] + A.a[k][i]) * Fi.a[j][k];   // (sigma F^-T)_ij = sum_k sigma_ik F^-1_jk
        f1[i][j] = (dtt * mu) * (J * s) - (J * p) * Fi.a[j][i];
      }
      if (prev) {
        // J^theta (v - v_old) instead of J (v - v_old), and the previous level's
        // convection rho_f J_old A_old v_old and viscous stress J_old sigma_v,old F_old^-T
        Mat<double, D> Fio = inverse<double, D>(Fo, Jo), Ao;
        for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) {
          double s = 0.0;
          for (int k = 0; k < D; ++k) s += Gvo.a[i][k] * Fio.a[k][j];
          Ao.a[i][j] = s;
        }
        for (int i = 0; i < D; ++i) {
          double co = 0.0;
          for (int j = 0; j < D; ++j) co += Ao.a[i][j] * vo[j];
          const T dv = v[i] - vo[i];
          f0[i] = f0[i] + (P.rho_f * (1.0 - P.theta)) * (dv * Jo - dv * J) + P.rho_f * dto * Jo * co;
        }
        for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) {
          double s = 0.0;
          for (int k = 0; k < D; ++k) s += (Ao.a[i][k] + Ao.a[k][i]) * Fio.a[j][k];
          f1[i][j] = f1[i][j] + dto * mu * Jo * s;
        }
      }
      // incompressibility g0 = J tr(A)
      T trA = zero;
      for (int i = 0; i < D; ++i) trA += A.a[i][i];
      T g0 = J * trA;
      // mesh motion h1 = (1/J) grad u
      T iJ = 1.0 / J;
      for (int a = 0; a < NQ2; ++a) {
        for (int i = 0; i < D; ++i) {
          T& r = Rv[a * D + i];
          axpy(r, w * N[a], f0[i]);
          for (int j = 0; j < D; ++j) axpy(r, w * dN[a * D + j], f1[i][j]);
        }
        if (mesh_row[a]) {
          for (int i = 0; i < D; ++i) {
            T s = zero;
            for (int j = 0; j < D; ++j) axpy(s, dN[a * D + j], Gu.a[i][j]);
            axpy(Ru[a * D + i], w, iJ * s);
          }
        }
      }
      for (int a = 0; a < NQ1; ++a) axpy(Rp[a], w * Np[a], g0);
    } else {
      // E = (F^T F - I)/2, Sigma = 2 mu E + lambda tr(E) I, f1 = dt*theta F Sigma
      Mat<T, D> E;
      for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) {
        T s = zero;
        for (int k = 0; k < D; ++k) s += F.a[k][i] * F.a[k][j];
        E.a[i][j] = 0.5 * (s - (i == j ? 1.0 : 0.0));
      }
      T trE = zero;
      for (int i = 0; i < D; ++i) trE += E.a[i][i];
      Mat<T, D> S;
      for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) {
        S.a[i][j] = (2.0 * P.mu_s) * E.a[i][j];
        if (i == j) S.a[i][j] += P.lambda_s * trE;
      }
      T f1[D][D];
      for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) {
        T s = zero;
        for (int k = 0; k < D; ++k) s += F.a[i][k] * S.a[k][j];
        f1[i][j] = dtt * s;
      }
      T f0[D], k0[D];
      for (int i = 0; i < D; ++i) {
        f0[i] = P.rho_s * (v[i] - vo[i]);
        k0[i] = (u[i] - uo[i]) - dtt * v[i];
      }
      if (prev) {
        // previous level: dt (1-theta) F_old Sigma_old and dt (1-theta) v_old
        Mat<double, D> Eo, So;
        for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) {
          double s = 0.0;
          for (int k = 0; k < D; ++k) s += Fo.a[k][i] * Fo.a[k][j];
          Eo.a[i][j] = 0.5 * (s - (i == j ? 1.0 : 0.0));
        }
        double trEo = 0.0;
        for (int i = 0; i < D; ++i) trEo += Eo.a[i][i];
        for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j)
          So.a[i][j] = 2.0 * P.mu_s * Eo.a[i][j] + (i == j ? P.lambda_s * trEo : 0.0);
        for (int i = 0; i < D; ++i) {
          for (int j = 0; j < D; ++j) {
            double s = 0.0;
            for (int k = 0; k < D; ++k) s += Fo.a[i][k] * So.a[k][j];
            f1[i][j] = f1[i][j] + dto * s;
          }
          k0[i] = k0[i] - dto * vo[i];
        }
      }
      for (int a = 0; a < NQ2; ++a) {
        for (int i = 0; i < D; ++i) {
          T& r = Rv[a * D + i];
          axpy(r, w * N[a], f0[i]);
          for (int j = 0; j < D; ++j) axpy(r, w * dN[a * D + j], f1[i][j]);
          axpy(Ru[a * D + i], w * N[a], k0[i]);
        }
      }
    }
  }
  // do-nothing correction on the outflow face: -dt*theta <rho_f nu_f J F^-T grad(v)^T F^-T n, phi>, n = e_0
  if (!solid && outflow) {
    const double mu = P.rho_f * P.nu_f;
    for (int q = 0; q < pb.nfqp; ++q) {
      const double* N = &pb.Nf[q * NQ2];
      const double* dN = &pb.dNf[q * NQ2 * D];
      const double w = pb.wf[q];
      Mat<T, D> Gv, Gu;
      for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) { Gv.a[i][j] = zero; Gu.a[i][j] = zero; }
      for (int a = 0; a < NQ2; ++a)
        for (int i = 0; i < D; ++i)
          for (int j = 0; j < D; ++j) {
            axpy(Gv.a[i][j], dN[a * D + j], Uv[a * D + i]);
            axpy(Gu.a[i][j], dN[a * D + j], Uu[a * D + i]);
          }
      Mat<T, D> F;
      for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) F.a[i][j] = Gu.a[i][j] + (i == j ? 1.0 : 0.0);
      T J = det<T, D>(F);
      Mat<T, D> Fi = inverse<T, D>(F, J);
      // c_k = (F^-T n)_k = Fi[0][k];  t_j = sum_k (grad v)_kj c_k = (grad v^T F^-T n)_j;  b_i = sum_j Fi[j][i] t_j
      T t[D];
      for (int j = 0; j < D; ++j) {
        T s = zero;
        for (int k = 0; k < D; ++k) s += Gv.a[k][j] * Fi.a[0][k];
        t[j] = s;
      }
      // previous level: -dt (1-theta) <rho_f nu_f J_old F_old^-T grad(v_old)^T F_old^-T n, phi>
      double bo[D];
      for (int i = 0; i < D; ++i) bo[i] = 0.0;
      if (prev) {
        Mat<double, D> Gvo, Fo;
        for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) {
          double gv = 0.0, gu = 0.0;
          for (int a = 0; a < NQ2; ++a) {
            gv += dN[a * D + j] * Vold[a * D + i];
            gu += dN[a * D + j] * Uold[a * D + i];
          }
          Gvo.a[i][j] = gv;
          Fo.a[i][j] = gu + (i == j ? 1.0 : 0.0);
        }
        const double Jo = det<double, D>(Fo);
        Mat<double, D> Fio = inverse<double, D>(Fo, Jo);
        double to[D];
        for (int j = 0; j < D; ++j) {
          double s = 0.0;
          for (int k = 0; k < D; ++k) s += Gvo.a[k][j] * Fio.a[0][k];
          to[j] = s;
        }
        for (int i = 0; i < D; ++i) {
          double s = 0.0;
          for (int j = 0; j < D; ++j) s += Fio.a[j][i] * to[j];
          bo[i] = -dto * mu * Jo * s;
        }
      }
      for (int i = 0; i < D; ++i) {
        T b = zero;
        for (int j = 0; j < D; ++j) b += Fi.a[j][i] * t[j];
        T c = (-dtt * mu) * (J * b);
        if (prev) c = c + bo[i];
        for (int a = 0; a < NQ2; ++a)
          if (N[a] != 0.0) axpy(Rv[a * D + i], w * N[a], c);
      }
    }
  }
}

// ------------------------------------------------------------ problem set-up
void classify(Problem& p) {
  const int D = p.dim;
  const Params& P = p.P;
  p.n_q2 = 1; p.n_q1 = 1; p.n_cells = 1;
  for (int d = 0; d < D; ++d) {
    p.nq2[d] = 2 * P.n[d] + 1; p.nq1[d] = P.n[d] + 1;
    p.n_q2 *= p.nq2[d]; p.n_q1 *= p.nq1[d]; p.n_cells *= P.n[d];
  }
  p.cell_solid.assign(p.n_cells, 0);
  const int zd = D - 1;
  const double hz = P.L[zd] / P.n[zd];
  for (int64_t c = 0; c < p.n_cells; ++c) {
    int ci[3]; unflatten(c, P.n, D, ci);
    double cz = (ci[zd] + 0.5) * hz;
    p.cell_solid[c] = cz < P.solid_h ? 1 : 0;
  }
  p.node_solid.assign(p.n_q2, 0); p.node_vdir.assign(p.n_q2, 0); p.node_udir.assign(p.n_q2, 0);
  std::vector<uint8_t> node_fluid(p.n_q2, 0);
  for (int64_t a = 0; a < p.n_q2; ++a) {
    int ii[3]; unflatten(a, p.nq2, D, ii);
    int lo[3], hi[3];
    for (int d = 0; d < D; ++d) cells_of_q2(ii[d], P.n[d], lo[d], hi[d]);
    int c[3] = {0, 0, 0};
    for (c[2] = (D == 3 ? lo[2] : 0); c[2] <= (D == 3 ? hi[2] : 0); ++c[2])
      for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
        for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0]) {
          if (p.cell_solid[cell_index(p, c)]) p.node_solid[a] = 1; else node_fluid[a] = 1;
        }
    bool on_bnd = false, inflow = ii[0] == 0, outflow = ii[0] == p.nq2[0] - 1;
    for (int d = 0; d < D; ++d) if (ii[d] == 0 || ii[d] == p.nq2[d] - 1) on_bnd = true;
    p.node_udir[a] = on_bnd ? 1 : 0;
    // v: Dirichlet everywhere on the outer boundary except the fluid part of the outflow face
    bool vdir = on_bnd;
    if (on_bnd && outflow && !p.node_solid[a]) {
      // outflow-face node outside the closed solid region: free unless it also lies on another face
      bool other = false;
      for (int d = 1; d < D; ++d) if (ii[d] == 0 || ii[d] == p.nq2[d] - 1) other = true;
      if (!inflow && !other) vdir = false;
    }
    p.node_vdir[a] = vdir ? 1 : 0;
  }
  p.p_active.assign(p.n_q1, 0);
  for (int64_t a = 0; a < p.n_q1; ++a) {
    int ii[3]; unflatten(a, p.nq1, D, ii);
    int lo[3], hi[3];
    for (int d = 0; d < D; ++d) cells_of_q1(ii[d], P.n[d], lo[d], hi[d]);
    int c[3] = {0, 0, 0};
    for (c[2] = (D == 3 ? lo[2] : 0); c[2] <= (D == 3 ? hi[2] : 0); ++c[2])
      for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
        for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0])
          if (!p.cell_solid[cell_index(p, c)]) p.p_active[a] = 1;
  }
  // DOF numbering: m | s_v | s_u | f_v | f_p
  int64_t n_s = 0, n_f = 0;
  for (int64_t a = 0; a < p.n_q2; ++a) (p.node_solid[a] ? n_s : n_f)++;
  p.off[0] = 0;
  p.off[1] = n_f * D;
  p.off[2] = p.off[1] + n_s * D;
  p.off[3] = p.off[2] + n_s * D;
  p.off[4] = p.off[3] + n_f * D;
  int64_t n_fluid_cells = 0;
  for (int64_t c = 0; c < p.n_cells; ++c) n_fluid_cells += p.cell_solid[c] ? 0 : 1;
  p.off[5] = p.off[4] + (p.pdisc ? (int64_t)(D + 1) * n_fluid_cells : p.n_q1);
  p.ndof = p.off[5];
  p.dof_v.assign(p.n_q2, -1); p.dof_u.assign(p.n_q2, -1); p.dof_p.assign(p.n_q1, -1);
  int64_t is = 0, jf = 0;
  for (int64_t a = 0; a < p.n_q2; ++a) {
    if (p.node_solid[a]) { p.dof_v[a] = p.off[1] + is * D; p.dof_u[a] = p.off[2] + is * D; ++is; }
    else { p.dof_u[a] = p.off[0] + jf * D; p.dof_v[a] = p.off[3] + jf * D; ++jf; }
  }
  if (!p.pdisc) {
    for (int64_t a = 0; a < p.n_q1; ++a) p.dof_p[a] = p.off[4] + a;
  } else {
    p.cell_pdof.assign(p.n_cells, -1);
    int64_t k = p.off[4];
    for (int64_t c = 0; c < p.n_cells; ++c)
      if (!p.cell_solid[c]) { p.cell_pdof[c] = k; k += D + 1; }
    for (int64_t a = 0; a < p.n_q1; ++a) p.p_active[a] = 0;   // no nodal pressure
  }
}

// Shared-cell flags between two Q2 nodes (or a Q1 node and a Q2 node): bit0 = a
// fluid cell contains both, bit1 = a solid cell contains both.
inline int shared_cells(const Problem& p, const int* lo_a, const int* hi_a, const int* lo_b, const int* hi_b) {
  const int D = p.dim;
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) {
    lo[d] = std::max(lo_a[d], lo_b[d]); hi[d] = std::min(hi_a[d], hi_b[d]);
    if (lo[d] > hi[d]) return 0;
  }
  int flags = 0;
  int c[3] = {0, 0, 0};
  for (c[2] = lo[2]; c[2] <= hi[2]; ++c[2])
    for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
      for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0])
        flags |= p.cell_solid[cell_index(p, c)] ? 2 : 1;
  return flags;
}

struct NodeNbr { int64_t node; int flags; };

// Q2 neighbours of a Q2 node (lattice order) with shared-cell flags.
void q2_neighbours_of_q2(const Problem& p, int64_t a, std::vector<NodeNbr>& out) {
  const int D = p.dim;
  out.clear();
  int ii[3] = {0, 0, 0}; unflatten(a, p.nq2, D, ii);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) cells_of_q2(ii[d], p.P.n[d], lo[d], hi[d]);
  int jlo[3] = {0, 0, 0}, jhi[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) { jlo[d] = 2 * lo[d]; jhi[d] = 2 * hi[d] + 2; }
  int jj[3] = {0, 0, 0};
  for (jj[2] = jlo[2]; jj[2] <= jhi[2]; ++jj[2])
    for (jj[1] = jlo[1]; jj[1] <= jhi[1]; ++jj[1])
      for (jj[0] = jlo[0]; jj[0] <= jhi[0]; ++jj[0]) {
        int blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) cells_of_q2(jj[d], p.P.n[d], blo[d], bhi[d]);
        int f = shared_cells(p, lo, hi, blo, bhi);
        if (f) out.push_back({q2_index(p, jj), f});
      }
}
// Q1 neighbours of a Q2 node.
void q1_neighbours_of_q2(const Problem& p, int64_t a, std::vector<NodeNbr>& out) {
  const int D = p.dim;
  out.clear();
  int ii[3] = {0, 0, 0}; unflatten(a, p.nq2, D, ii);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) cells_of_q2(ii[d], p.P.n[d], lo[d], hi[d]);
  int jj[3] = {0, 0, 0};
  for (jj[2] = lo[2]; jj[2] <= hi[2] + (D == 3 ? 1 : 0); ++jj[2])
    for (jj[1] = lo[1]; jj[1] <= hi[1] + 1; ++jj[1])
      for (jj[0] = lo[0]; jj[0] <= hi[0] + 1; ++jj[0]) {
        int blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) cells_of_q1(jj[d], p.P.n[d], blo[d], bhi[d]);
        int f = shared_cells(p, lo, hi, blo, bhi);
        if (f) out.push_back({q1_index(p, jj), f});
      }
}
// Q2 neighbours of a Q1 node.
void q2_neighbours_of_q1(const Problem& p, int64_t a, std::vector<NodeNbr>& out) {
  const int D = p.dim;
  out.clear();
  int ii[3] = {0, 0, 0}; unflatten(a, p.nq1, D, ii);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) cells_of_q1(ii[d], p.P.n[d], lo[d], hi[d]);
  int jlo[3] = {0, 0, 0}, jhi[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) { jlo[d] = 2 * lo[d]; jhi[d] = 2 * hi[d] + 2; }
  int jj[3] = {0, 0, 0};
  for (jj[2] = jlo[2]; jj[2] <= jhi[2]; ++jj[2])
    for (jj[1] = jlo[1]; jj[1] <= jhi[1]; ++jj[1])
      for (jj[0] = jlo[0]; jj[0] <= jhi[0]; ++jj[0]) {
        int blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) cells_of_q2(jj[d], p.P.n[d], blo[d], bhi[d]);
        int f = shared_cells(p, lo, hi, blo, bhi);
        if (f) out.push_back({q2_index(p, jj), f});
      }
}

// Column list of one row, in increasing global order.  kind: 0 = v row, 1 = u
// row (of Q2 node a), 2 = p row (Q1 node a).  Fixed rows return the diagonal.
void row_columns(const Problem& p, int kind, int64_t a, int64_t row, std::vector<NodeNbr>& nb2,
                 std::vector<NodeNbr>& nb1, std::vector<int64_t>& cols) {
  const int D = p.dim;
  cols.clear();
  bool fixed = (kind == 0 && p.node_vdir[a]) || (kind == 1 && p.node_udir[a]) ||
               (kind == 2 && !p.pdisc && !p.p_active[a]);
  if (fixed) { cols.push_back(row); return; }
  if (kind == 2 && p.pdisc) {
    // discontinuous pressure row of fluid cell a: the v and u DOFs of the cell's Q2
    // nodes, class by class (m, s_v, s_u, f_v), nodes in increasing index order
    int c[3] = {0, 0, 0}; unflatten(a, p.P.n, D, c);
    std::vector<int64_t> nodes;
    const int NQ2 = p.nq2loc;
    for (int l = 0; l < NQ2; ++l) {
      int ai[3] = {l % 3, (l / 3) % 3, l / 9}, ii[3] = {0, 0, 0};
      for (int d = 0; d < D; ++d) ii[d] = 2 * c[d] + ai[d];
      nodes.push_back(q2_index(p, ii));
    }
    std::sort(nodes.begin(), nodes.end());
    for (int64_t b : nodes) if (!p.node_solid[b] && !p.node_udir[b]) for (int i = 0; i < D; ++i) cols.push_back(p.dof_u[b] + i);
    for (int64_t b : nodes) if (p.node_solid[b] && !p.node_vdir[b]) for (int i = 0; i < D; ++i) cols.push_back(p.dof_v[b] + i);
    for (int64_t b : nodes) if (p.node_solid[b] && !p.node_udir[b]) for (int i = 0; i < D; ++i) cols.push_back(p.dof_u[b] + i);
    for (int64_t b : nodes) if (!p.node_solid[b] && !p.node_vdir[b]) for (int i = 0; i < D; ++i) cols.push_back(p.dof_v[b] + i);
    return;
  }
  nb2.clear(); nb1.clear();
  int need = 0;   // bit0: fluid-cell couplings, bit1: solid-cell couplings
  bool want_v = true, want_p = false;
  if (kind == 0) { q2_neighbours_of_q2(p, a, nb2); q1_neighbours_of_q2(p, a, nb1); need = 3; want_p = true; }
  else if (kind == 1) {
    q2_neighbours_of_q2(p, a, nb2);
    if (p.node_solid[a]) { need = 2; }                 // kinematic rows: solid cells, u and v
    else { need = 1; want_v = false; }                 // mesh-motion rows: fluid cells, u only
  } else { q2_neighbours_of_q1(p, a, nb2); need = 1; }  // p rows: fluid cells, u and v
  // m (u of non-solid nodes)
  for (auto& b : nb2) if ((b.flags & need) && !p.node_solid[b.node] && !p.node_udir[b.node])
    for (int i = 0; i < D; ++i) cols.push_back(p.dof_u[b.node] + i);
  // s_v
  if (want_v) for (auto& b : nb2) if ((b.flags & need) && p.node_solid[b.node] && !p.node_vdir[b.node])
    for (int i = 0; i < D; ++i) cols.push_back(p.dof_v[b.node] + i);
  // s_u
  for (auto& b : nb2) if ((b.flags & need) && p.node_solid[b.node] && !p.node_udir[b.node])
    for (int i = 0; i < D; ++i) cols.push_back(p.dof_u[b.node] + i);
  // f_v
  if (want_v) for (auto& b : nb2) if ((b.flags & need) && !p.node_solid[b.node] && !p.node_vdir[b.node])
    for (int i = 0; i < D; ++i) cols.push_back(p.dof_v[b.node] + i);
  // f_p (only through fluid cells)
  if (want_p && !p.pdisc)
    for (auto& b : nb1) if ((b.flags & 1) && p.p_active[b.node]) cols.push_back(p.dof_p[b.node]);
  if (want_p && p.pdisc) {
    // the pressure DOFs of the fluid cells containing node a (cells in lexicographic order)
    int ii[3] = {0, 0, 0}; unflatten(a, p.nq2, D, ii);
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) cells_of_q2(ii[d], p.P.n[d], lo[d], hi[d]);
    int c[3] = {0, 0, 0};
    for (c[2] = lo[2]; c[2] <= hi[2]; ++c[2])
      for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
        for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0]) {
          const int64_t pd = p.cell_pdof[cell_index(p, c)];
          if (pd >= 0) for (int k = 0; k <= D; ++k) cols.push_back(pd + k);
        }
  }
}

struct RowInfo { std::vector<int8_t> kind; std::vector<int64_t> node; };

void build_row_info(const Problem& p, RowInfo& ri) {
  ri.kind.assign(p.ndof, -1); ri.node.assign(p.ndof, -1);
  for (int64_t a = 0; a < p.n_q2; ++a)
    for (int i = 0; i < p.dim; ++i) {
      ri.kind[p.dof_v[a] + i] = 0; ri.node[p.dof_v[a] + i] = a;
      ri.kind[p.dof_u[a] + i] = 1; ri.node[p.dof_u[a] + i] = a;
    }
  if (!p.pdisc) {
    for (int64_t a = 0; a < p.n_q1; ++a) { ri.kind[p.dof_p[a]] = 2; ri.node[p.dof_p[a]] = a; }
  } else {
    for (int64_t c = 0; c < p.n_cells; ++c)
      if (p.cell_pdof[c] >= 0)
        for (int k = 0; k <= p.dim; ++k) { ri.kind[p.cell_pdof[c] + k] = 2; ri.node[p.cell_pdof[c] + k] = c; }
  }
}

void build_pattern(Problem& p) {
  RowInfo ri; build_row_info(p, ri);
  const int64_t n = p.ndof;
  p.rowptr.assign(n + 1, 0);
  p.row_fixed.assign(n, 0);
  std::vector<int64_t> counts(n, 0);
#pragma omp parallel
  {
    std::vector<NodeNbr> nb2, nb1; std::vector<int64_t> cols;
#pragma omp for schedule(dynamic, 1024)
    for (int64_t r = 0; r < n; ++r) {
      row_columns(p, ri.kind[r], ri.node[r], r, nb2, nb1, cols);
      counts[r] = (int64_t)cols.size();
      int k = ri.kind[r]; int64_t a = ri.node[r];
      p.row_fixed[r] = ((k == 0 && p.node_vdir[a]) || (k == 1 && p.node_udir[a]) ||
                        (k == 2 && !p.pdisc && !p.p_active[a])) ? 1 : 0;
    }
  }
  for (int64_t r = 0; r < n; ++r) p.rowptr[r + 1] = p.rowptr[r] + counts[r];
  p.colind.assign(p.rowptr[n], 0);
#pragma omp parallel
  {
    std::vector<NodeNbr> nb2, nb1; std::vector<int64_t> cols;
#pragma omp for schedule(dynamic, 1024)
    for (int64_t r = 0; r < n; ++r) {
      row_columns(p, ri.kind[r], ri.node[r], r, nb2, nb1, cols);
      for (size_t k = 0; k < cols.size(); ++k) p.colind[p.rowptr[r] + k] = (int32_t)cols[k];
    }
  }
}

// Global DOF indices of a cell's local DOFs, with the cell's node metadata.
void cell_dofs(const Problem& p, const int* c, int64_t* gdof, int64_t* q2nodes, int64_t* q1nodes) {
  const int D = p.dim;
  const int NQ2 = p.nq2loc, NQ1 = p.nq1loc;
  for (int a = 0; a < NQ2; ++a) {
    int ai[3] = {a % 3, (a / 3) % 3, a / 9};
    int ii[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) ii[d] = 2 * c[d] + ai[d];
    int64_t node = q2_index(p, ii);
    q2nodes[a] = node;
    for (int i = 0; i < D; ++i) {
      gdof[a * D + i] = p.dof_v[node] + i;
      gdof[NQ2 * D + a * D + i] = p.dof_u[node] + i;
    }
  }
  if (p.pdisc) {
    // solid cells carry no pressure: their pressure slots point at the first p DOF and are masked
    const int64_t pd = p.cell_pdof[cell_index(p, c)];
    for (int a = 0; a < NQ1; ++a) { q1nodes[a] = -1; gdof[2 * NQ2 * D + a] = pd >= 0 ? pd + a : p.off[4]; }
    return;
  }
  for (int a = 0; a < NQ1; ++a) {
    int ai[3] = {a % 2, (a / 2) % 2, a / 4};
    int ii[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) ii[d] = c[d] + ai[d];
    int64_t node = q1_index(p, ii);
    q1nodes[a] = node;
    gdof[2 * NQ2 * D + a] = p.dof_p[node];
  }
}

// Residual (J == nullptr) or Jacobian assembly over all cells, 2^d colouring.
template <int D, int NL>
int assemble(Problem& p, const double* Uglob, const double* Uold, double* Rglob, double* vals, double* minJ_out) {
  const int64_t ncell = p.n_cells;
  const int NQ2 = p.nq2loc, NQ1 = p.nq1loc;
  int fail = 0;
  double minJ = 1e300;
  const int ncolors = 1 << D;
  for (int color = 0; color < ncolors; ++color) {
#pragma omp parallel reduction(min : minJ) reduction(| : fail)
    {
      std::vector<Dual<NL>> Ud(NL), Rd(NL);
      std::vector<double> Ux(NL), Rx(NL), Vo(NQ2 * D), Uo(NQ2 * D);
      std::vector<int64_t> gdof(NL), q2n(NQ2), q1n(NQ1);
      std::vector<uint8_t> mesh_row(NQ2), rowok(NL), colok(NL);
#pragma omp for schedule(dynamic, 64)
      for (int64_t cidx = 0; cidx < ncell; ++cidx) {
        int c[3] = {0, 0, 0}; unflatten(cidx, p.P.n, D, c);
        int col = 0; for (int d = 0; d < D; ++d) col |= (c[d] & 1) << d;
        if (col != color) continue;
        const bool solid = p.cell_solid[cidx];
        const bool outflow = (c[0] == p.P.n[0] - 1) && !solid;
        cell_dofs(p, c, gdof.data(), q2n.data(), q1n.data());
        for (int a = 0; a < NQ2; ++a) mesh_row[a] = p.node_solid[q2n[a]] ? 0 : 1;
        for (int a = 0; a < NQ2; ++a)
          for (int i = 0; i < D; ++i) {
            Vo[a * D + i] = Uold ? Uold[gdof[a * D + i]] : 0.0;
            Uo[a * D + i] = Uold ? Uold[gdof[NQ2 * D + a * D + i]] : 0.0;
          }
        double mj = 1e300;
        if (vals) {
          for (int k = 0; k < NL; ++k) {
            Ud[k] = dconst<NL>(Uglob[gdof[k]]);
            Ud[k].d[k] = 1.0;
          }
          cell_residual<D, Dual<NL>>(p, solid, outflow, mesh_row.data(), Ud.data(), Vo.data(), Uo.data(), Rd.data(), &mj);
        } else {
          for (int k = 0; k < NL; ++k) Ux[k] = Uglob[gdof[k]];
          cell_residual<D, double>(p, solid, outflow, mesh_row.data(), Ux.data(), Vo.data(), Uo.data(), Rx.data(), &mj);
        }
        if (mj < minJ) minJ = mj;
        for (int k = 0; k < NL; ++k) {
          int64_t g = gdof[k];
          bool ok = !p.row_fixed[g];
          // solid cells own no p rows/cols; fluid cells own no kinematic u rows
          if (solid && k >= 2 * NQ2 * D) ok = false;
          if (!solid && k >= NQ2 * D && k < 2 * NQ2 * D && !mesh_row[(k - NQ2 * D) / D]) ok = false;
          rowok[k] = ok;
          colok[k] = !p.row_fixed[g] && !(solid && k >= 2 * NQ2 * D);
        }
        for (int r = 0; r < NL; ++r) {
          if (!rowok[r]) continue;
          const int64_t gr = gdof[r];
          if (!vals) { Rglob[gr] += Rx[r]; continue; }
          const int32_t* cb = &p.colind[p.rowptr[gr]];
          const int32_t* ce = &p.colind[p.rowptr[gr + 1]];
          for (int cc = 0; cc < NL; ++cc) {
            if (!colok[cc]) continue;
            double v = Rd[r].d[cc];
            const int32_t gc = (int32_t)gdof[cc];
            const int32_t* it = std::lower_bound(cb, ce, gc);
            if (it == ce || *it != gc) { if (v != 0.0) fail = 1; continue; }
            vals[it - p.colind.data()] += v;
          }
        }
      }
    }
  }
  *minJ_out = minJ;
  return fail;
}

// Element assembly for the problem's element (NL = 2 * NQ2 * dim + pressure basis size).
int assemble_any(Problem& p, const double* U, const double* Uold, double* R, double* vals, double* minJ) {
  if (p.dim == 2) return p.pdisc ? assemble<2, 39>(p, U, Uold, R, vals, minJ) : assemble<2, 40>(p, U, Uold, R, vals, minJ);
  return p.pdisc ? assemble<3, 166>(p, U, Uold, R, vals, minJ) : assemble<3, 170>(p, U, Uold, R, vals, minJ);
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

struct fsigen_params {
  int dim;
  int n[3];
  double L[3];
  double solid_h;
  double rho_f, nu_f, mu_s, lambda_s, rho_s, dt, theta;
  int pressure;   // 0: continuous Q1 pressure, 1: discontinuous P1 (Q2-Q2-P1disc)
};

void* fsigen_create(const fsigen_params* in) {
  if (!in || (in->dim != 2 && in->dim != 3)) return nullptr;
  if (!(in->theta > 0.0 && in->theta <= 1.0)) return nullptr;
  Problem* p = new Problem();
  p->dim = in->dim;
  p->P.dim = in->dim;
  for (int d = 0; d < 3; ++d) { p->P.n[d] = in->n[d]; p->P.L[d] = in->L[d]; }
  for (int d = 0; d < in->dim; ++d) if (in->n[d] < 1) { delete p; return nullptr; }
  p->P.solid_h = in->solid_h;
  p->P.rho_f = in->rho_f; p->P.nu_f = in->nu_f; p->P.mu_s = in->mu_s; p->P.lambda_s = in->lambda_s;
  p->P.rho_s = in->rho_s; p->P.dt = in->dt; p->P.theta = in->theta;
  if (in->pressure != 0 && in->pressure != 1) { delete p; return nullptr; }
  p->P.pressure = in->pressure;
  p->pdisc = in->pressure == 1;
  classify(*p);
  build_tables(*p);
  build_pattern(*p);
  return p;
}

void fsigen_free(void* h) { delete static_cast<Problem*>(h); }

// out[0..5] = class offsets m|s_v|s_u|f_v|f_p|n ; out[6] = nnz ; out[7] = #Q2 nodes ; out[8] = #Q1 nodes
void fsigen_sizes(void* h, int64_t* out) {
  Problem* p = static_cast<Problem*>(h);
  for (int k = 0; k < 6; ++k) out[k] = p->off[k];
  out[6] = p->rowptr.back();
  out[7] = p->n_q2;
  out[8] = p->n_q1;
}

void fsigen_pattern(void* h, int64_t* rowptr, int32_t* colind) {
  Problem* p = static_cast<Problem*>(h);
  std::memcpy(rowptr, p->rowptr.data(), sizeof(int64_t) * p->rowptr.size());
  std::memcpy(colind, p->colind.data(), sizeof(int32_t) * p->colind.size());
}

// Per DOF: coordinates (dim doubles), field (0 v, 1 u, 2 p), component, fixed-row flag.
void fsigen_dof_info(void* h, double* coords, int32_t* field, int32_t* comp, uint8_t* fixed) {
  Problem* p = static_cast<Problem*>(h);
  const int D = p->dim;
  double hq[3];
  for (int d = 0; d < D; ++d) hq[d] = p->P.L[d] / (2.0 * p->P.n[d]);
  for (int64_t a = 0; a < p->n_q2; ++a) {
    int ii[3] = {0, 0, 0}; unflatten(a, p->nq2, D, ii);
    for (int i = 0; i < D; ++i) {
      for (int f = 0; f < 2; ++f) {
        int64_t g = (f == 0 ? p->dof_v[a] : p->dof_u[a]) + i;
        for (int d = 0; d < D; ++d) coords[g * D + d] = ii[d] * hq[d];
        field[g] = f; comp[g] = i; fixed[g] = p->row_fixed[g];
      }
    }
  }
  if (p->pdisc) {
    // discontinuous pressure: the cell centre, component = basis function index
    for (int64_t c = 0; c < p->n_cells; ++c) {
      if (p->cell_pdof[c] < 0) continue;
      int ci[3] = {0, 0, 0}; unflatten(c, p->P.n, D, ci);
      for (int k = 0; k <= D; ++k) {
        const int64_t g = p->cell_pdof[c] + k;
        for (int d = 0; d < D; ++d) coords[g * D + d] = (2.0 * ci[d] + 1.0) * hq[d];
        field[g] = 2; comp[g] = k; fixed[g] = p->row_fixed[g];
      }
    }
    return;
  }
  for (int64_t a = 0; a < p->n_q1; ++a) {
    int ii[3] = {0, 0, 0}; unflatten(a, p->nq1, D, ii);
    int64_t g = p->dof_p[a];
    for (int d = 0; d < D; ++d) coords[g * D + d] = ii[d] * 2.0 * hq[d];
    field[g] = 2; comp[g] = 0; fixed[g] = p->row_fixed[g];
  }
}


// Jacobian values on the pattern at state U (previous step Uold, nullable = 0).
// Returns 0, or 1 if a nonzero fell outside the pattern, 2 if J <= 0 somewhere.
int fsigen_jacobian(void* h, const double* U, const double* Uold, double* vals, double* minJ) {
  Problem* p = static_cast<Problem*>(h);
  const int64_t nnz = p->rowptr.back();
  std::memset(vals, 0, sizeof(double) * nnz);
  const int fail = assemble_any(*p, U, Uold, nullptr, vals, minJ);
  for (int64_t r = 0; r < p->ndof; ++r)
    if (p->row_fixed[r]) vals[p->rowptr[r]] = 1.0;
  if (fail) return 1;
  return (*minJ <= 0.0) ? 2 : 0;
}

// Residual R(U) (fixed rows zero).
int fsigen_residual(void* h, const double* U, const double* Uold, double* R, double* minJ) {
  Problem* p = static_cast<Problem*>(h);
  std::memset(R, 0, sizeof(double) * p->ndof);
  assemble_any(*p, U, Uold, R, nullptr, minJ);
  for (int64_t r = 0; r < p->ndof; ++r) if (p->row_fixed[r]) R[r] = 0.0;
  return (*minJ <= 0.0) ? 2 : 0;
}

// Node map of a 2D mesh for the learned correction stage: per Q2 node (lattice
// order) node_dof[4] = {first v DOF, first u DOF, p DOF or -1 (not a vertex),
// flags: bit0 closed solid region, bit1 v fixed, bit2 u fixed, bit3 interface
// (in the solid closure and in a fluid cell), bit4 i odd, bit5 j odd, bit6 p row
// fixed}, and patch[9] = the 3x3 lattice
// neighbourhood (row-major, dx fastest, -1 outside the mesh).  Returns 0, or -1
// for 3D problems.
int fsigen_node_map(void* h, int32_t* node_dof, int32_t* patch) {
  Problem* p = static_cast<Problem*>(h);
  if (p->pdisc) return -1;   // the stage's patch layout assumes nodal Q1 pressure
  const int D = p->dim;
  const int nx = p->nq2[0], ny = p->nq2[1], nz = D == 3 ? p->nq2[2] : 1;
  const int slots = D == 3 ? 27 : 9;
  for (int64_t a = 0; a < p->n_q2; ++a) {
    const int i = (int)(a % nx), j = (int)((a / nx) % ny), k = D == 3 ? (int)(a / ((int64_t)nx * ny)) : 0;
    node_dof[a * 4 + 0] = (int32_t)p->dof_v[a];
    node_dof[a * 4 + 1] = (int32_t)p->dof_u[a];
    int32_t pd = -1;
    if (i % 2 == 0 && j % 2 == 0 && k % 2 == 0)
      pd = (int32_t)p->dof_p[((int64_t)(k / 2) * p->nq1[1] + j / 2) * p->nq1[0] + i / 2];
    node_dof[a * 4 + 2] = pd;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    cells_of_q2(i, p->P.n[0], lo[0], hi[0]);
    cells_of_q2(j, p->P.n[1], lo[1], hi[1]);
    if (D == 3) cells_of_q2(k, p->P.n[2], lo[2], hi[2]);
    bool fluid_cell = false;
    for (int ck = lo[2]; ck <= hi[2]; ++ck)
      for (int cj = lo[1]; cj <= hi[1]; ++cj)
        for (int ci = lo[0]; ci <= hi[0]; ++ci) {
          const int c[3] = {ci, cj, ck};
          if (!p->cell_solid[cell_index(*p, c)]) fluid_cell = true;
        }
    int32_t flags = 0;
    if (p->node_solid[a]) flags |= 1;
    if (p->node_vdir[a]) flags |= 2;
    if (p->node_udir[a]) flags |= 4;
    if (p->node_solid[a] && fluid_cell) flags |= 8;
    flags |= (i % 2) << 4;
    flags |= (j % 2) << 5;
    if (pd >= 0 && p->row_fixed[pd]) flags |= 64;
    flags |= (k % 2) << 7;
    node_dof[a * 4 + 3] = flags;
    for (int dk = (D == 3 ? -1 : 0); dk <= (D == 3 ? 1 : 0); ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          const int ii = i + di, jj = j + dj, kk = k + dk;
          const int slot = (D == 3 ? (dk + 1) * 9 : 0) + (dj + 1) * 3 + (di + 1);
          const bool in = ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz;
          patch[a * slots + slot] = in ? (int32_t)(((int64_t)kk * ny + jj) * nx + ii) : -1;
        }
  }
  return 0;
}

// Per cell (lexicographic, direction 0 fastest): the global DOF of each local DOF
// in the element layout of cell_residual (v of Q2 node a comp i at a*dim + i, u at
// NQ2*dim + a*dim + i, p of Q1 vertex P at 2*NQ2*dim + P), and flags: bit 0 solid
// cell, bit 1 fluid cell on the outflow face x_0 = L_0, bit 2 + a local Q2 node a
// outside the closed solid region (carries a mesh-motion row).  This is the mesh
// description a device assembler needs; it holds no residual arithmetic.
void fsigen_cell_map(void* h, int32_t* cell_dof, uint32_t* cell_flags) {
  Problem* p = static_cast<Problem*>(h);
  const int D = p->dim;
  const int NL = p->nloc, NQ2 = p->nq2loc, NQ1 = p->nq1loc;
  std::vector<int64_t> gdof(NL), q2n(NQ2), q1n(NQ1);
  for (int64_t cidx = 0; cidx < p->n_cells; ++cidx) {
    int c[3] = {0, 0, 0}; unflatten(cidx, p->P.n, D, c);
    cell_dofs(*p, c, gdof.data(), q2n.data(), q1n.data());
    for (int k = 0; k < NL; ++k) cell_dof[cidx * NL + k] = (int32_t)gdof[k];
    const bool solid = p->cell_solid[cidx];
    uint32_t f = solid ? 1u : 0u;
    if (!solid && c[0] == p->P.n[0] - 1) f |= 2u;
    for (int a = 0; a < NQ2; ++a) if (!p->node_solid[q2n[a]]) f |= 1u << (2 + a);
    cell_flags[cidx] = f;
  }
}

int fsigen_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"

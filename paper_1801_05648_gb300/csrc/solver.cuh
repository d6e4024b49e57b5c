// Solver context: the monolithic operator split into class blocks, the block-LDU
// preconditioner of Alg. 2 (with the Alg. 3 solid and pressure-Schur fluid
// sub-solves) and the right-preconditioned FGMRES outer iteration.
#pragma once
#include "amg.cuh"
#include "learned.cuh"
#include "sparse_util.cuh"

#include <string>
#include <vector>

namespace fsi {

struct SolverParams {
  int restart = 100;
  int maxit = 1000;
  int flags = 0;
  double dt_theta = 0.01;
  AmgParams amg;
  int vc_mesh = 1, vc_solid = 2, vc_fluid = 1, vc_pressure = 1;
  int mass_degree = 12;
  double mass_ratio = 8.0;
  int spmv_unroll = 4;
  double learned_accept = 0.1;   // accept the learned correction when ||r' - A c|| < this * ||r'||
  int spmv_prefetch = 1;
  double cluster_max_bytes = 6.0e6;
  int fluid_gmres_iters = 4;     // FLUID_GMRES: inner GMRES steps per A_ff^-1
  int precond_variant = 0;       // 0 Alg. 2 (LDU), 1 (D + L)^-1, 2 (D + U)^-1, 3 D^-1
  int spmv_lane_shift = 0;       // FP32 SpMV lanes per block row divided by 2^shift
  int spmv_stage = 0;            // staged 2 x 2 FP32 Chebyshev steps (opt-in)
  int spmv_order = 1;            // outer-operator rows in the length order of Bsr::ord2
  int inject = 0;                // fault injection for the bounded-wait tests (fsi_debug_inject)
};

enum Flags { X0_GIVEN = 1, USE_GRAPHS = 2, NO_RIGID_MODES = 4, CLUSTER_COARSE = 8, LEARNED = 16, NO_PDL = 32,
             GRID_COARSE = 64, FLUID_GMRES = 128, MLP_CUDA_CORES = 256 };

constexpr int kFluidGmresMax = 32;

// Workspace of the inner fluid GMRES (Sec. 4.4): k steps on the n_fv fluid-velocity
// DOFs; basis V ((k+1) x n) and preconditioned directions Z (k x n) in FP64.
struct FluidGmres {
  int k = 0;
  int64_t n = 0;
  DBuf<double> V, Z, w, h1, h2, nrm, beta, y, part, npart;
  DBuf<float> t32a, t32b;     // FP32 V-cycle input/output (FP32-AMG form)
  DBuf<int> zero;             // device 0: the vector counts of mdot/maxpy are offsets from it
};

template <class T>
struct PrecWork {
  DBuf<T> in, out;            // fixed input/output of P^-1 (length n)
  DBuf<T> a2_t, a2_u;         // Alg. 2 temporaries
  DBuf<T> s3_y, s3_t;         // Alg. 3 / fluid Schur temporaries
  bool ready = false;
};

struct Context {
  cudaStream_t s = nullptr;
  bool own_stream = false;
  int device = -1;                        // CUDA device current at fsi_setup; every entry point runs on it
  void* noalloc_scratch = nullptr;        // device address of the no-allocation entry point's scratch array
  cudaStream_t s2 = nullptr;              // second branch of Alg. 2 (mesh solve next to the solid solve)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int dim = 2;
  int64_t n = 0;
  int64_t off[6] = {0, 0, 0, 0, 0, 0};
  SolverParams prm;
  std::string err;
  // outer operator: vector rows (first off[4] DOFs, d x d blocks) and p rows
  Bsr AVV, AVP, APV, APP;
  // preconditioner blocks
  Bsr C_ms;                   // m rows x (s_v, s_u) cols
  Bsr A_vu, A_uv;             // solid couplings
  DBuf<double> uv_w64;        // dt*theta on the free s_u rows (A_uv = -dt*theta A_uu there), 0 on fixed rows
  DBuf<float> uv_w32;
  Bsr C_sv_f, C_sv_p;         // s rows x f_v cols, s rows x p cols
  bool csf_u_zero = false;    // the s_u rows of C_sv_f and C_sv_p hold no entries
  Bsr C_fv_ms, C_p_ms;        // f_v rows x (m, s) cols, p rows x (m, s) cols
  Bsr B_vp, B_pv;             // fluid velocity-pressure couplings
  Bsr Mblk, Avv, Auu, Aff, Cpp;   // diagonal blocks, consumed by precond_build
  Hierarchy H[4];             // M, S_hat, A_ff, S_p
  ChebSolver mass;            // A_uu (solid mass)
  bool built = false;
  bool fp32_ready = false;    // FP32 copies of the current hierarchies and couplings exist
  Csr pattern;                // device CSR pattern of the operator (values not kept), for fsi_update_values
  int precision = 0;          // 0 FP64, 1 FP32 AMG
  PrecWork<double> pw64;
  PrecWork<float> pw32;
  FluidGmres fg;
  DBuf<double> solid_B;       // near-nullspace of S_hat (rigid-body modes)
  // learned correction stage, its training operator A^T, and the residual harvest
  Learned learned;
  Bsr AVVt, AVPt, APVt, APPt;
  bool At_built = false;
  double* harvest = nullptr;  // device, harvest_n x n: V_j - A z_j of the first iterations
  int harvest_n = 0;
  int last_accepted = 0;      // learned corrections taken in the last solve
  int last_reorth = 0;        // Arnoldi steps of the last solve with a second Gram-Schmidt pass
  // FGMRES storage; basis columns V_i, Z_i at stride ldv (n rounded up to 32: 16-byte aligned columns)
  int m_alloc = 0;
  int64_t ldv = 0;
  DBuf<double> V, Z, Hh, cs, sn, g, y, h1, h2, scal, partials, npart, zfix, wfix, rvec;
  DBuf<int> jdev, kdev;
  DBuf<double> dpart;         // per-block sums of squares of the Arnoldi defect
  DBuf<int> reorth;           // [0] second-pass flag of the current step, [1] second passes in this solve
  double* pinned = nullptr;   // host-mapped: [0] |g_{j+1}|/|b|, [1] breakdown flag, [2] h_{j+1,j}
  double* pinned_dev = nullptr;
  int* pinned_j = nullptr;    // pinned host staging for the iteration index
  cudaGraphExec_t iter_graph = nullptr;
  int iter_graph_prec = -1;
  bool iter_graph_learned = false;
  const double* iter_graph_harvest = nullptr;
  int iter_graph_harvest_n = 0;
  int iter_graph_fluid = 0;   // inner fluid GMRES steps the graph was captured with (0: off)
  int64_t graph_kernels = 0;  // kernel launches inside one replay of iter_graph
  int64_t last_launches = 0;  // kernels launched by the last solve
  // stats
  std::vector<double> hist;
  double setup_s = 0, build_s = 0, solve_s = 0;
  int last_iters = 0, last_cycles = 0, last_status = 0;
  double last_true_relres = 0;
  ~Context();
};

void context_setup(Context& C, const int64_t* rowptr, const int32_t* colind, const double* vals,
                   const double* solid_coords);
// New operator values (device, CSR order of the pattern given to context_setup):
// re-extract every class block; the preconditioner must be built again.
void context_update_values(Context& C, const double* vals_dev);
void precond_build(Context& C, int precision);
template <class T> void precond_apply(Context& C, const T* r, T* z);
void apply_operator(Context& C, const double* x, double* y);
int fgmres_solve(Context& C, const double* b, double* x, double tol);
// sub-solve hooks (which: 0..3 hierarchies, 4 mass, 5 solid Alg. 3, 6 fluid, 7 Alg. 2)
template <class T> void apply_block(Context& C, int which, const T* in, T* out);
double precond_bytes(const Context& C, int vb);
double operator_bytes(const Context& C);
// y = A^T x (transposed blocks built on first use)
void apply_operator_t(Context& C, const double* x, double* y);

// Training of the learned stage (learned.cu)
void trainer_init(Trainer& T, const TrainParams& p);
void trainer_set_master(Trainer& T, const float* w);
// one residual vector r' of context C: loss ||r' - A c||^2 / ||r'||^2, gradient
// accumulated when grad is true
double trainer_step(Trainer& T, Context& C, const double* rp, bool grad = true);
// AdamW with the mean of the accumulated gradients at learning rate lr (<= 0: the parameters' rate)
void trainer_update(Trainer& T, cudaStream_t s, double lr = 0.0);

}  // namespace fsi

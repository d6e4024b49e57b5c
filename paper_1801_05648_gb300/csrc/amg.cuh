// Smoothed-aggregation AMG (Vanek, Mandel & Brezina 1996) on the GPU: set-up
// (strength, distance-2 MIS aggregation, tentative prolongator by per-aggregate
// modified Gram-Schmidt, Jacobi-smoothed prolongator, Galerkin triple product)
// and the V-cycle apply with Chebyshev smoothing, in FP64 or FP32.
//
// Set-up per level:
//   strength   j != i strong iff max(f_ij, f_ji) > 0 and >= theta*sqrt(f_ii f_jj),
//              f = Frobenius norm of the node block (squares summed in row-major
//              order without fused multiply-add)
//   aggregate  distance-2 maximal independent set with keys
//              (state << 59 | priority << 27 | index), priorities
//              splitmix64(i + level*2^32) >> 32 (Bell, Dalton & Olson 2012);
//              roots seed aggregates, neighbours of roots join them, every other
//              non-isolated node joins its aggregated neighbour of largest
//              (priority, index); isolated nodes stay out
//   P_tent     per aggregate MGS QR of the near-nullspace rows (members in
//              increasing node order), dropped columns below drop_tol
//   P          (I - omega D^-1 A) P_tent, omega = 4/(3 lambda),
//              lambda = |lambda_max(D^-1 A)| by power iteration from
//              x_i = 1 + u_i (splitmix64 stream 256 + level)
//   A_c        R (A P),  R = P^T
//   RAn        -(R A), so that a V-cycle forms the restricted residual R (b - A x)
//              as R b + RAn x in one pass (the residual b - A x is never stored)
// Coarsest level: dense inverse (all-zero rows replaced by identity rows).
#pragma once
#include "common.cuh"

namespace fsi {

struct AmgParams {
  double theta = 0.08;
  int coarse_max = 500;
  int max_levels = 10;
  int cheb_degree = 4;
  double cheb_ratio = 30.0;
  double cheb_upper = 1.3;
  int power_iters = 15;
  double drop_tol = 1e-10;
  int presmooth = 1;
  int postsmooth = 1;
  int cheb_degree_coarse = 2;   // Chebyshev degree on levels >= 1 (0: cheb_degree)
  int degree(int level) const { return level > 0 && cheb_degree_coarse > 0 ? cheb_degree_coarse : cheb_degree; }
};

template <class T>
struct LevelWork {
  DBuf<T> b, x, xb, r, d;   // rhs, iterate, ping-pong iterate, residual, Chebyshev direction
  bool zeroed = false;      // cleared once for the timing hook
};

struct AmgLevel {
  Bsr A;
  DBuf<double> dinv64;
  DBuf<float> dinv32;
  double lam = 0.0;
  Bsr P, R;
  Bsr RAn;                    // -(R A): the coarse right-hand side R (b - A x) = R b + RAn x in one product
  int nagg = 0;
  DBuf<int> agg;              // aggregate of each node (-1 = none), for inspection
  LevelWork<double> w64;
  LevelWork<float> w32;
  int64_t n() const { return A.rows(); }
};

// ---- coarse end of a V-cycle in one launch (coarse.cu): a thread-block cluster, or a
// cooperative grid over half the GPU with a software grid barrier
constexpr int kCoarseThreads = 512;       // threads per CTA of the coarse kernel
constexpr int kCoarseMaxLevels = 8;
constexpr int kCoarseMaxDeg = 16;
// levels whose matrix has at most this many value bytes run in the cluster (fsi_params.cluster_max_bytes)
inline double& coarse_max_bytes() {
  thread_local double b = 6.0e6;   // per thread, like the other launch knobs (common.cuh)
  return b;
}

struct CoarseMat {
  int nbr = 0, br = 1, bc = 1, tpr = 1;
  int64_t nnzb = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const void* v = nullptr;
};
struct CoarseLevel {
  CoarseMat A, P, R;
  const void* dinv = nullptr;
  void* b = nullptr; void* x = nullptr; void* xb = nullptr; void* r = nullptr; void* d = nullptr;
  double inv_theta = 0.0;
  int deg = 0;   // Chebyshev degree of this level
  double c1[kCoarseMaxDeg] = {}, c2[kCoarseMaxDeg] = {};
};
struct CoarsePlan {
  int nlev = 0, presmooth = 1, postsmooth = 1;
  CoarseLevel lev[kCoarseMaxLevels];
  const void* cinv = nullptr;
  int ncoarse = 0;
};
enum CoarseMode { COARSE_PER_LEVEL = 0, COARSE_CLUSTER = 1, COARSE_GRID = 2 };

template <class T>
struct CoarseRun {
  DBuf<CoarsePlan> plan;
  int mode = COARSE_PER_LEVEL;
  int ctas = 0;      // CTAs of the launch (cluster size, or cooperative grid size); 0: not available
  int first = -1;    // first level handled by the coarse kernel (-1: none)
  DBuf<unsigned> bar;   // grid barrier: arrivals, generation
  DBuf<int> err;        // set when a grid barrier wait gave up
};

struct Hierarchy {
  std::vector<AmgLevel> levels;
  CoarseRun<double> crun64;
  CoarseRun<float> crun32;
  int coarse_mode = COARSE_PER_LEVEL;   // how the small coarse levels run (opt-in: one launch)
  int ncoarse = 0;
  DBuf<double> cinv64;
  DBuf<float> cinv32;
  AmgParams prm;
  bool has_fp32 = false;
  double operator_complexity() const;
  // algorithmic bytes of one V-cycle (value size vb)
  double vcycle_bytes(int vb) const;
};

// Build the hierarchy of A (FP64 values, square, br == bc) with near-nullspace B
// (device, (A.rows()) x k, node-major rows, row-major k columns).
void amg_setup(Hierarchy& H, Bsr&& A, const double* B, int k, const AmgParams& prm, cudaStream_t s);
// Enqueue `reps` fused Chebyshev SpMV steps on level `level` (timing hook; the
// level's own work vectors, zeroed on first use).  Returns algorithmic bytes per step.
template <class T> double amg_smoother_steps(Hierarchy& H, int level, int reps, cudaStream_t s);
// Algorithmic bytes of one fused Chebyshev step on A (value size vb): the SpMV
// (values, indices, row pointers, x once, x' written) plus b, D^-1 and d read, d written.
inline double cheb_step_bytes(const Bsr& A, int vb) { return A.spmv_bytes(vb) + 4.0 * vb * A.rows(); }

// FP32 copies of every level's matrices, diagonal and coarse inverse.
void amg_make_fp32(Hierarchy& H, cudaStream_t s);
// x = V(b): one V-cycle from x = 0 (x, b: level-0 sized, distinct)
template <class T> void amg_vcycle(Hierarchy& H, const T* b, T* x, cudaStream_t s);

// Plan the cluster launch for levels [first, end) of H (value type T); run.first
// stays -1 when no cluster launch is possible.
template <class T> void coarse_plan_build(Hierarchy& H, int first, CoarseRun<T>& run, cudaStream_t s);
// V-cycle of levels [run.first, end) from x = 0 in one launch (b, x: level run.first sized).
template <class T> void coarse_vcycle(const CoarseRun<T>& run, const T* b, T* x, cudaStream_t s);
// True when a grid-barrier wait of the hierarchy's coarse kernel gave up since the
// last check (the barrier state is then reset).  Waits for the stream.
bool coarse_failed(Hierarchy& H, cudaStream_t s);
// First level from which every level is small enough for the cluster kernel, or
// -1 when that leaves only the dense coarsest level.
int coarse_first_level(const Hierarchy& H, int value_bytes);

// Chebyshev polynomial smoother/solver on D^-1 A from x = 0 (used for the solid
// mass matrix): x = p(D^-1 A) D^-1 b with `degree` steps over [lam/ratio, upper*lam].
struct ChebSolver {
  Bsr A;
  DBuf<double> dinv64;
  DBuf<float> dinv32;
  double lam = 0.0;
  int degree = 12;
  double ratio = 8.0, upper = 1.3;
  LevelWork<double> w64;
  LevelWork<float> w32;
};
void cheb_setup(ChebSolver& C, Bsr&& A, int degree, double ratio, double upper, int power_iters, cudaStream_t s);
void cheb_make_fp32(ChebSolver& C, cudaStream_t s);
template <class T> void cheb_apply(ChebSolver& C, const T* b, T* x, cudaStream_t s);
// Same polynomial, FP64, with caller-provided scratch vectors xb and d (each of
// C.A.rows() entries) instead of the solver's own work vectors.
void cheb_apply_scratch(const ChebSolver& C, const double* b, double* x, double* xb, double* d, cudaStream_t s);

// |lambda_max(D^-1 A)| estimate by power iteration (see above), FP64.
double power_lambda(const Bsr& A, const double* dinv, int iters, int stream_id, cudaStream_t s);

}  // namespace fsi

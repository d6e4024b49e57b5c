/*
 * fsi.h - C ABI of the GB300 (sm_103a) solver for one linearised monolithic
 * ALE fluid-structure Jacobian.
 *
 * The operation is the linear solve A_h dU = F_h of one Newton step (Alg. 1,
 * Sec. 3.3) for the block system of Eq. (mat:small), Sec. 3.4:
 *
 *       [ M     C_ms  0    ]   m : mesh displacement u outside the solid
 *   A = [ C_sm  S     C_sf ]   s : solid velocity v and displacement u (closed solid region)
 *       [ C_fm  C_fs  F    ]   f : fluid velocity v and pressure p
 *
 * solved by right-preconditioned FGMRES whose preconditioner is the approximate
 * block-LDU factorisation of Sec. 4.1 (Alg. 2) with the solid Schur solve of
 * Sec. 4.3 (Alg. 3), a pressure Schur-complement fluid solve (Sec. 4.4) and
 * smoothed-aggregation AMG V-cycles for the sub-block inverses (Sec. 4.2-4.4).
 *
 * Conventions shared by all calls
 *   - Unknowns are ordered by class: m | s_v | s_u | f_v | f_p.  The vector
 *     classes (m, s_v, s_u, f_v) are node-major, component-minor (dim values per
 *     node); s_v and s_u list the same nodes in the same order.
 *   - Matrix input is CSR with 64-bit row pointers, 32-bit column indices sorted
 *     within each row, FP64 values.  Fixed (Dirichlet) DOFs are identity rows
 *     with their columns removed.
 *   - Device pointers (`*_dev`) are CUDA device memory the caller owns (e.g.
 *     PyTorch tensors) and must stay valid during the call; the library works on
 *     the stream given to fsi_setup and returns after that stream has finished
 *     the call's work.
 *   - A context belongs to the CUDA device that is current when fsi_setup is
 *     called; the other calls taking a context switch to that device for their
 *     duration and restore the caller's current device before they return.
 *   - Every call returns FSI_OK (0) or a negative FSI_E* code; fsi_last_error()
 *     gives the message of the last failure on that context.  No call aborts the
 *     process.  Device memory the library allocates is released by fsi_free().
 */
#ifndef FSI_H_
#define FSI_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FSI_OK = 0,
  FSI_EINVAL = -1,       /* bad argument, malformed CSR or offsets, call out of order */
  FSI_ENOMEM = -2,       /* device allocation failed */
  FSI_ECUDA = -3,        /* CUDA runtime error */
  FSI_ENOTCONV = -4,     /* maxit reached: x holds the last iterate, stats are filled */
  FSI_EBREAKDOWN = -5,   /* Arnoldi breakdown before the tolerance was met */
  FSI_ENONFINITE = -6    /* non-finite right-hand side or iterate */
};

enum { FSI_FP64 = 0, FSI_FP32_AMG = 1 };

enum {
  FSI_X0_GIVEN = 1,        /* fsi_solve starts from the x passed in (else from 0) */
  FSI_USE_GRAPHS = 2,      /* replay each FGMRES iteration as one captured CUDA graph */
  FSI_NO_RIGID_MODES = 4,  /* solid AMG with translations only, even when coordinates are given */
  FSI_CLUSTER_COARSE = 8,  /* run the coarse AMG levels (matrices <= cluster_max_bytes) of each
                              V-cycle in one 16-CTA thread-block-cluster launch instead of one launch
                              per step (fewer launches, but measured slower than the per-level path) */
  FSI_LEARNED = 16,        /* apply the learned correction stage after P^-1 in every FGMRES
                              iteration (needs fsi_learned_setup and weights; see below) */
  FSI_NO_PDL = 32,         /* launch the context's kernels without programmatic dependent launch
                              (each kernel then waits for the previous one to finish before it
                              is scheduled) */
  FSI_GRID_COARSE = 64,    /* like FSI_CLUSTER_COARSE, but the coarse levels run as one cooperative
                              launch over half the GPU with a software grid barrier (bounded
                              waits: a barrier that times out makes fsi_solve return FSI_ECUDA).
                              Not together with FSI_CLUSTER_COARSE */
  FSI_FLUID_GMRES = 128,   /* Sec. 4.4: every A_ff^-1 of the fluid Schur solve (and fsi_apply_block 2)
                              is fluid_gmres_iters steps of GMRES on A_ff from a zero start,
                              right-preconditioned by the A_ff V-cycle(s), Arnoldi in FP64 (classical
                              Gram-Schmidt twice), least squares by Givens rotations on the device; a
                              fixed step count, no stopping test.  The preconditioner then depends
                              nonlinearly on its input, which FGMRES allows */
  FSI_MLP_CUDA_CORES = 256 /* evaluate the learned stage's MLP with FP32 FMAs on the CUDA cores instead
                              of tcgen05 MMAs on the tensor cores (TF32 operands, the activations split
                              into two TF32 terms, FP32 accumulation).  Both agree with FP32 arithmetic
                              to about 1e-6 relative.  A tensor-core wait that gives up (about one
                              second; not seen in correct operation) sets a flag that the next
                              fsi_solve of the context reports as FSI_ECUDA */
};

typedef struct fsi_params {
  int restart;              /* FGMRES restart length m (default 100) */
  int maxit;                /* maximum FGMRES iterations (default 1000) */
  int flags;                /* FSI_X0_GIVEN | FSI_USE_GRAPHS | FSI_NO_RIGID_MODES | FSI_CLUSTER_COARSE |
                               FSI_LEARNED | FSI_NO_PDL | FSI_GRID_COARSE | FSI_FLUID_GMRES |
                               FSI_MLP_CUDA_CORES */
  double dt_theta;          /* c = dt*theta of the solid Schur complement S_hat = A_vv + c A_vu (0.01) */
  /* smoothed-aggregation AMG */
  double strength_theta;    /* strength threshold on node-block Frobenius norms (0.08) */
  int coarse_max;           /* coarsen until <= this many scalar rows (1500) */
  int max_levels;           /* (10) */
  int cheb_degree;          /* Chebyshev smoother degree (4) */
  double cheb_ratio;        /* smoothing interval [lambda/ratio, upper*lambda] (30) */
  double cheb_upper;        /* (1.3) */
  int power_iters;          /* power iterations for lambda_max(D^-1 A) (15) */
  double drop_tol;          /* near-nullspace column drop in the tentative prolongator (1e-10) */
  int presmooth, postsmooth;/* Chebyshev sweeps before/after the coarse correction (1, 1) */
  /* V-cycles per application of each block inverse */
  int vcycles_mesh, vcycles_solid, vcycles_fluid, vcycles_pressure;   /* (1, 2, 1, 1) */
  /* solid mass solve: Chebyshev polynomial on D^-1 A_uu */
  int mass_degree;          /* (12) */
  double mass_ratio;        /* interval [lambda/ratio, upper*lambda] (8 in 2D, 20 in 3D) */
  /* SpMV launch shape: lanes per block row follow the mean row length (each lane
     takes at least 2 blocks in FP32, 8 in FP64); each lane loads spmv_unroll blocks
     (4 or 8; 8 applies to blocks of at most 24 bytes) before multiplying (4).
     Like every launch knob, it applies to the calls on this context only. */
  int spmv_unroll;
  /* learned stage: take the correction only when ||r' - A c|| < learned_accept * ||r'||
     (0.1; at 0.3 and above the trained stage's accepted corrections stall FGMRES) */
  double learned_accept;
  /* SpMV L2 prefetch: 0 none, 1 each CTA bulk-prefetches the head of its slice of the
     matrix arrays (at most 32 KB per matrix) into L2 before waiting for the previous
     kernel, 2 the same with at most 5 persistent CTAs per SM walking longer slices (1) */
  int spmv_prefetch;
  /* FSI_CLUSTER_COARSE / FSI_GRID_COARSE: levels whose matrix values take at most this
     many bytes run in the single coarse launch (6e6) */
  double cluster_max_bytes;
  /* Chebyshev degree on the coarser AMG levels (>= 1); 0 = cheb_degree on every level (2) */
  int cheb_degree_coarse;
  /* FSI_FLUID_GMRES: inner GMRES steps k per A_ff^-1, 1..32 (4) */
  int fluid_gmres_iters;
  /* block factorisation of the preconditioner (the LDU form depends on the block
     ordering, Sec. 4.1): FSI_PRECOND_LDU Alg. 2 (default); FSI_PRECOND_LOWER (D + L)^-1,
     Alg. 2 steps 1-3; FSI_PRECOND_UPPER (D + U)^-1: x_f = F^-1 r_f,
     x_s = S^-1 (r_s - C_sf x_f), x_m = M^-1 (r_m - C_ms x_s); FSI_PRECOND_DIAG D^-1.
     D = diag(M, S, F), L (C_sm dropped) / U the strict block triangles; the same
     approximate inverses in every variant */
  int precond_variant;
  /* FP32 SpMV launches: lanes per block row = the automatic count (see spmv_unroll)
     divided by 2^spmv_lane_shift, at least 1 (0..4; 0).  Fewer lanes per row put
     more rows, and more blocks per lane, into each pass of a warp */
  int spmv_lane_shift;
  /* 2 x 2 FP32 Chebyshev steps on large matrices by persistent CTAs that have the TMA
     engine (cp.async.bulk) copy each chunk's 16-bit column offsets into shared memory
     one chunk ahead: 1 on, 0 off (0).  Bit-identical to the default kernel, and measured
     slower on the GB300 (116 vs 104 us per 1024x512 level-0 step) */
  int spmv_stage;
  /* the outer operator's two-matrix SpMVs (A_VV next to A_VP, A_PV next to A_PP) take
     each CTA's block rows sorted by length within 32-row windows, so that the rows of a
     warp have equal length and no FP64 lane idles while a longer row of its warp
     finishes: 1 on, 0 off (1).  Changes which thread sums a row, not how: bit-identical */
  int spmv_order;
} fsi_params;

enum { FSI_PRECOND_LDU = 0, FSI_PRECOND_LOWER = 1, FSI_PRECOND_UPPER = 2, FSI_PRECOND_DIAG = 3 };

typedef struct fsi_stats {
  int iters;                /* FGMRES iterations of the last solve */
  int cycles;               /* restart cycles */
  int status;               /* FSI_OK / FSI_ENOTCONV / ... */
  double true_relres;       /* ||b - A x|| / ||b|| of the returned x (FP64 on the device) */
  double setup_s;           /* fsi_setup wall seconds */
  double precond_build_s;   /* fsi_precond_build wall seconds */
  double solve_s;           /* fsi_solve wall seconds (stream synchronised) */
  double operator_bytes;    /* algorithmic bytes of one outer SpMV */
  double precond_bytes;     /* algorithmic bytes of one application of Alg. 2 */
  const double* relres_hist;/* |g_{j+1}|/||b|| per iteration; owned by the context, valid until the next solve */
  int hist_len;
  int64_t kernel_launches;  /* CUDA kernels the solve executed (graph replays counted per kernel node) */
  int learned_accepted;     /* FSI_LEARNED: iterations whose learned correction was taken */
  int reorth_passes;        /* Arnoldi steps that took a second Gram-Schmidt pass (see fsi_solve) */
} fsi_stats;

typedef struct fsi_ctx fsi_ctx;

/* Defaults for dim = 2 or 3 (mass_ratio depends on dim). */
void fsi_default_params(fsi_params* p, int dim);

/*
 * fsi_setup - copy one monolithic Jacobian to the device and split it into the
 * class blocks of Eq. (mat:small).
 *   out            receives the new context (NULL on failure; then only the
 *                  return code reports the error)
 *   dim            2 or 3
 *   n              number of unknowns (= block_offsets[5])
 *   rowptr/colind/vals   host CSR, n+1 / nnz / nnz entries (deep-copied; the
 *                  caller may free them after return).  vals may be NULL: the
 *                  pattern only, with the values supplied later from device
 *                  memory by fsi_update_values (e.g. a Jacobian assembled on the
 *                  device by fsi_asm_jacobian)
 *   block_offsets  host, 6 entries: start of m, s_v, s_u, f_v, f_p, and n;
 *                  non-decreasing, vector classes multiples of dim, |s_v| = |s_u|
 *   node_coords    host, nullable: dim coordinates per s_v node (rigid-body
 *                  near-nullspace of the solid AMG); copied
 *   p              nullable (defaults)
 *   cuda_stream    cudaStream_t to run on (NULL = a stream the context creates)
 * Errors: FSI_EINVAL on inconsistent sizes, unsorted or out-of-range columns,
 * non-finite values; FSI_ENOMEM / FSI_ECUDA from the device.
 */
int fsi_setup(fsi_ctx** out, int dim, int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
              const int64_t* block_offsets, const double* node_coords, const fsi_params* p, void* cuda_stream);

/*
 * fsi_precond_build - build the preconditioner of Alg. 2 on the device: the
 * Schur approximations S_hat = A_vv + c A_vu (Alg. 3) and
 * S_p = C_pp - B_pv diag(A_ff)^-1 B_vp (Sec. 4.4), and smoothed-aggregation
 * hierarchies for M, S_hat, A_ff and S_p (set-up timed apart from the solve).
 *   precision   FSI_FP64, or FSI_FP32_AMG: hierarchies, smoothers and the
 *               couplings inside P^-1 stored and run in FP32 (FP32 accumulation)
 *               while the outer SpMV, Gram-Schmidt and Givens stay FP64.
 *               May be called again to switch precision (the FP64 hierarchy is
 *               built once).
 *   learned_weights  nullable: path of a weights file for the learned stage
 *               (as fsi_learned_load; needs fsi_learned_setup first).
 */
int fsi_precond_build(fsi_ctx* ctx, int precision, const char* learned_weights);

/*
 * fsi_solve - FGMRES (right preconditioned, restart m) until
 * ||b - A x||_2 / ||b||_2 <= rtol, confirmed on the true residual.
 *   rhs_dev  device, n doubles (not modified)
 *   x_dev    device, n doubles: initial guess when FSI_X0_GIVEN is set, else
 *            overwritten from 0; receives the solution (best iterate on
 *            FSI_ENOTCONV)
 *   out      nullable; filled on FSI_OK, FSI_ENOTCONV and FSI_EBREAKDOWN
 */
int fsi_solve(fsi_ctx* ctx, const double* rhs_dev, double* x_dev, double rtol, fsi_stats* out);

/* Release every device and host resource of the context (NULL is ignored). */
void fsi_free(fsi_ctx* ctx);

/* Message of the last failed call on ctx ("" if none).  For ctx = NULL: the
 * last failure on this thread of a call made without a context (fsi_setup,
 * fsi_trainer_create / _set_master / _get / _save). */
const char* fsi_last_error(const fsi_ctx* ctx);

/* ------------------------------------------------------------------------
 * Component entry points (same context, after fsi_precond_build).  They expose
 * the pieces of the solve for parity checks and per-kernel timing.
 */

/* y = A x, the monolithic operator (Eq. mat:small), FP64; x_dev, y_dev: n doubles.
 * Like fsi_apply_block, this call only enqueues its kernels on the context's
 * stream and returns; synchronise that stream before reading y. */
int fsi_apply_operator(fsi_ctx* ctx, const double* x_dev, double* y_dev);

/*
 * out = B^-1 in for one block inverse of Alg. 2, in the built precision (FP64
 * inputs/outputs; converted internally in the FP32 form):
 *   which 0  M^-1      (mesh,   m DOFs):   vcycles_mesh V-cycles
 *         1  S_hat^-1  (solid velocity Schur, s_v DOFs)
 *         2  A_ff^-1   (fluid velocity, f_v DOFs)
 *         3  S_p^-1    (pressure Schur, f_p DOFs)
 *         4  A_uu^-1   (solid mass Chebyshev, s_u DOFs)
 *         5  S^-1      (Alg. 3 on s_v,s_u DOFs)
 *         6  F^-1      (fluid Schur solve on f_v,f_p DOFs)
 *         7  P^-1      (Alg. 2, all n DOFs)
 * Enqueued on the context's stream without waiting (see fsi_apply_operator).
 */
int fsi_apply_block(fsi_ctx* ctx, int which, const double* in_dev, double* out_dev);

/*
 * Enqueue `reps` fused Chebyshev smoothing steps (one SpMV each:
 * r = D^-1 (b - A x); d = c1 d + c2 r; x' = x + d) on `level` (which must have a
 * coarser level) of hierarchy `which` (0..3), in the built precision, on that
 * level's own work vectors; returns without waiting.  This is the V-cycle's
 * dominant kernel, exposed for timing.  *bytes_per_step (nullable) receives its
 * algorithmic bytes: matrix values and indices, x read once, x' written, and b,
 * D^-1, d read and d written.
 */
int fsi_smoother_step(fsi_ctx* ctx, int which, int level, int reps, double* bytes_per_step);

/*
 * AMG hierarchy inspection (which 0..3 as above, level >= 0).
 *   info[0] levels, [1] block rows of this level, [2] block size, [3] nnz blocks,
 *   [4] aggregates formed from this level (0 on the coarsest), [5] scalar rows of
 *   the coarsest level;  *lambda = lambda_max(D^-1 A) estimate of the level.
 */
int fsi_amg_info(fsi_ctx* ctx, int which, int level, int64_t info[6], double* lambda);
/*
 * Copy one array of a level to host memory `dst` (caller sizes it from
 * fsi_amg_info): what 0 aggregate id per node (int32, -1 = unaggregated),
 * 1 A row pointers (int32, rows+1), 2 A block columns (int32), 3 A values
 * (double, nnzb*b*b, row-major blocks), 4 P row pointers, 5 P block columns,
 * 6 P values (b x k blocks), 7 P block columns count as int64 in dst[0].
 */
int fsi_amg_export(fsi_ctx* ctx, int which, int level, int what, void* dst);

/*
 * fsi_mass_solve_noalloc - out = A_uu^-1 in, the solid-mass Chebyshev solve of
 * fsi_apply_block(ctx, 4, ...) in FP64 (whatever precision was built), for
 * callers that cannot allocate device memory when they call: code running
 * while its stream is captured into a CUDA graph (cudaMalloc is not permitted
 * there) or code whose device memory is owned by another allocator.  The paper
 * has no counterpart; it is an interface convenience.
 *   in_dev, out_dev  device, one double per s_u DOF (block_offsets[3] - [2])
 * Allocates nothing: its two scratch vectors live in a static device array of
 * 2 x 2^20 doubles (16 MiB) that every GPU loading the library keeps until the
 * process exits, so the solid block may have at most 2^20 displacement DOFs
 * (larger blocks return FSI_EINVAL).  The first call on a context looks up the
 * array's device address on the context's device (cudaGetSymbolAddress) and
 * keeps it with the context; make that first call before any stream capture.
 * All calls share the array: calls whose work overlaps on the GPU (other streams,
 * or other contexts on the same device) race on it.  Its contents are fully
 * overwritten by each call before they are read.  Enqueued on the context's
 * stream without waiting.
 */
int fsi_mass_solve_noalloc(fsi_ctx* ctx, const double* in_dev, double* out_dev);

/*
 * fsi_update_values - replace the operator's values by a new Jacobian on the
 * same pattern, without a host round trip (Alg. 1, Sec. 3.3: a Newton step
 * re-assembles the Jacobian, the pattern stays).
 *   vals_dev  device, one double per stored entry of the CSR given to fsi_setup
 *             (same order); read during the call only
 * Re-extracts every class block on the device and drops the preconditioner:
 * fsi_precond_build must be called again before the next solve (FSI_EINVAL
 * otherwise).  The learned stage's node map and weights are kept.
 */
int fsi_update_values(fsi_ctx* ctx, const double* vals_dev);

/* ------------------------------------------------------------------------
 * Residual and Jacobian assembly on the device (Alg. 1, Sec. 3.3; variational
 * form Eq. (fsi:all), Sec. 3.2-3.3, strong form Sec. 2) for structured box meshes
 * of Q2 velocity, Q2 displacement and continuous Q1 pressure: the Newton loop of
 * the time step then runs without host assembly.  The residual is
 *   fluid cells  (rho_f J (v - v_old), phi) - (rho_f J grad(v) F^-1 (u - u_old), phi)
 *                + dt theta [(rho_f J grad(v) F^-1 v, phi) + (J sigma_v F^-T, grad phi)]
 *                + (J (-p) F^-T, grad phi) + (J tr(grad(v) F^-1), psi)
 *                + (grad(u) / J, grad phi) on the mesh-motion rows
 *                - dt theta <rho_f nu_f J F^-T grad(v)^T F^-T e_0, phi> on the outflow face
 *   solid cells  (rho_s (v - v_old), phi) + dt theta (F Sigma, grad phi)
 *                + (u - u_old - dt theta v, phi) on the displacement rows
 * with F = I + grad u, J = det F, sigma_v = rho_f nu_f (grad v F^-1 + F^-T grad v^T),
 * Sigma = 2 mu_s E + lambda_s tr(E) I, E = (F^T F - I)/2; for theta < 1 the
 * previous level adds its dt (1 - theta) share of the convection, viscous,
 * outflow and solid stress terms and of the kinematic velocity, and the fluid
 * time derivative carries theta J + (1 - theta) J_old.  3^dim Gauss points per
 * cell, 3^(dim-1) on the outflow face.  The Jacobian is the exact derivative of
 * this discrete residual (dual numbers).  Fixed rows: residual 0, Jacobian row =
 * the identity entry.
 */
typedef struct fsi_asm fsi_asm;

typedef struct fsi_asm_mesh {
  int dim;                  /* 2 or 3 */
  int pressure;             /* 0: continuous Q1 pressure (vertex functions); 1: the discontinuous P1
                               pressure of the Q2-Q2-P1disc pair (Sec. 3.4), per fluid cell
                               p = p_0 + sum_k p_k (2 xi_k - 1) in the cell's reference coordinates */
  int cells[3];             /* cells per direction of the box; cells are numbered
                               lexicographically, direction 0 fastest */
  double h[3];              /* cell size per direction */
  int64_t n;                /* unknowns */
  const int32_t* cell_dof;  /* host, cells x NL (Q1: NL = 40 in 2D, 170 in 3D; P1disc: 39, 166):
                               global DOF of each local DOF.  Local order: v of Q2 node a component i
                               at a*dim + i, u at NQ2*dim + a*dim + i, pressure function P at
                               2*NQ2*dim + P; Q2 nodes a = a0 + 3 a1 (+ 9 a2) and Q1 vertices
                               P = P0 + 2 P1 (+ 4 P2), each index running along its direction from
                               the cell's lower corner; P1disc: P = 0 the constant, P = k the k-th
                               centred linear.  Entries of the pressure slots of solid cells are any
                               valid DOF (solid cells carry no pressure) */
  const uint32_t* cell_flags; /* host, one per cell: bit 0 solid cell, bit 1 the cell's upper face
                               in direction 0 is the do-nothing outflow boundary, bit 2 + a local Q2
                               node a carries a mesh-motion row (lies outside the closed solid) */
  const int64_t* rowptr;    /* host, n + 1: the Jacobian's CSR pattern (as given to fsi_setup) */
  const int32_t* colind;    /* host, rowptr[n] sorted column indices */
  const uint8_t* row_fixed; /* host, n: identity (Dirichlet / inactive pressure) rows */
} fsi_asm_mesh;

typedef struct fsi_asm_physics {
  double rho_f, nu_f;       /* fluid density, kinematic viscosity */
  double mu_s, lambda_s;    /* St. Venant-Kirchhoff Lame parameters */
  double rho_s;             /* solid density */
  double dt, theta;         /* time step, theta of the one-step-theta scheme (0 < theta <= 1) */
} fsi_asm_physics;

/* Copy the mesh tables to the device (host arrays may be freed after return);
 * cuda_stream as in fsi_setup.  FSI_EINVAL on inconsistent tables. */
int fsi_asm_create(fsi_asm** out, const fsi_asm_mesh* mesh, const fsi_asm_physics* phys, void* cuda_stream);
/* R(U) at state U_dev with previous time level Uold_dev (device, n doubles each;
 * Uold_dev NULL = 0).  R_dev (device, n) is overwritten.  *min_J (nullable): the
 * smallest det F over the volume quadrature points; *r_absmax (nullable):
 * max_i |R_i|.  Waits for the stream. */
int fsi_asm_residual(fsi_asm* a, const double* U_dev, const double* Uold_dev, double* R_dev, double* min_J,
                     double* r_absmax);
/* dR/dU at U_dev into vals_dev (device, rowptr[n] doubles, CSR order), which is
 * overwritten.  FSI_EINVAL if a nonzero falls outside the pattern.  Waits. */
int fsi_asm_jacobian(fsi_asm* a, const double* U_dev, const double* Uold_dev, double* vals_dev, double* min_J);
/* y += alpha x (device, n doubles each): the Newton update U += dU.  Waits. */
int fsi_asm_axpy(fsi_asm* a, double alpha, const double* x_dev, double* y_dev);
const char* fsi_asm_last_error(const fsi_asm* a);
void fsi_asm_free(fsi_asm* a);

/* ------------------------------------------------------------------------
 * Learned correction stage (2D and 3D meshes).  The paper has no such stage: it is an
 * extra smoothing step after Alg. 2 inside each FGMRES iteration.  With
 * z_j = P^-1 v_j and q = A z_j:
 *     r' = v_j - q,  c = MLP(r'),  t = A c;
 *     if ||r' - t||_2 < tau ||r'||_2:  z_j <- z_j + c,  w = q + t   (accepted;
 *                                  tau = fsi_params.learned_accept, default 0.1)
 *     else:                        w = q                        (plain preconditioner)
 * so the stage changes the search space of FGMRES but never its answer.  One
 * more FP64 outer SpMV and one MLP pass per iteration.
 *
 * MLP (per Q2 node a of a D-dimensional mesh, 3^D lattice patch N(a), slots
 * s = 3 (dj+1) + (di+1) in 2D, 9 (dk+1) + 3 (dj+1) + (di+1) in 3D; C = 2D+1
 * components k = v_x v_y [v_z] u_x u_y [u_z] p per node):
 *   x_{s,k} = r'[dof_k(N_s(a))] / sigma_in[class]
 *             (0 outside the mesh and for p at a node that carries no p)
 *   rho_a   = sqrt(sum of the 3^D C squares / (3^D C))       (45 in 2D, 189 in 3D)
 *   f_a     = [x / rho_a, one-hot of (i odd) + 2 (j odd) [+ 4 (k odd)] (2^D),
 *              flags solid, v fixed, u fixed, interface (4)]   53 inputs in 2D, 201 in 3D
 *   y_a     = W3^T gelu(W2^T gelu(W1^T f_a + b1) + b2) + b3     64, 64, C
 *   c[dof_k(a)] = y_{a,k} rho_a sigma_out[class]  (0 on fixed rows, at rho_a = 0)
 * Classes are m, s_v, s_u, f_v, f_p (0..4).  Weights bfloat16 (round to nearest
 * even), arithmetic FP32, c written in FP64.  The parameter vector (7,941 values
 * in 2D, 17,543 in 3D) is W1 [in][64], b1 [64], W2 [64][64], b2 [64], W3 [64][C],
 * b3 [C], row-major, W_l mapping its layer's input (rows) to output (columns).
 * Weights file: 8 bytes "FSIMLP01", int32 {in, 64, C, 0}, float32 sigma_in[5],
 * sigma_out[5], then the bfloat16 parameters, little endian.  A context takes
 * only the file of its mesh's dimension.  The tensor-core evaluation
 * (default) is 2D; 3D meshes use the CUDA-core kernel.
 */
#define FSI_MLP_PARAMS 7941
#define FSI_MLP_INPUTS 53
#define FSI_MLP_PARAMS_3D 17543
#define FSI_MLP_INPUTS_3D 201

/*
 * fsi_learned_setup - the node map of the context's mesh (host arrays, copied):
 *   n_nodes    Q2 nodes
 *   node_dof   n_nodes x 4 int32: first v DOF (the other D-1 components
 *              follow), first u DOF (likewise), p DOF or -1, flags (1 solid
 *              closure, 2 v fixed, 4 u fixed, 8 interface, 16 lattice i odd,
 *              32 lattice j odd, 64 p row fixed, 128 lattice k odd)
 *   patch      n_nodes x 3^D int32: the lattice neighbourhood (slots as above,
 *              i fastest), -1 outside the mesh
 * Every DOF must belong to exactly one node (FSI_EINVAL otherwise).
 */
int fsi_learned_setup(fsi_ctx* ctx, int64_t n_nodes, const int32_t* node_dof, const int32_t* patch);
/* Load the stage's weights from a file (format above). */
int fsi_learned_load(fsi_ctx* ctx, const char* path);
/* Set the stage's weights from host memory: sigma_in[5], sigma_out[5] (> 0), params bfloat16
 * (FSI_MLP_PARAMS of them on a 2D mesh, FSI_MLP_PARAMS_3D on a 3D one). */
int fsi_learned_set_weights(fsi_ctx* ctx, const float* sigma_in, const float* sigma_out, const uint16_t* params);
/* c = MLP(r') (device, n doubles each; every entry of c written).  Enqueued without waiting. */
int fsi_learned_apply(fsi_ctx* ctx, const double* r_dev, double* c_dev);
/* Features f_a (device, n_nodes x FSI_MLP_INPUTS[_3D] floats, node-major) and rho_a (n_nodes
 * floats) of r'.  Enqueued. */
int fsi_learned_features(fsi_ctx* ctx, const double* r_dev, float* feat_dev, float* rho_dev);
/* Change fsi_params.learned_accept (in (0, 1]) of a context. */
int fsi_set_learned_accept(fsi_ctx* ctx, double tau);
/* Change the run-time flags of a context (FSI_X0_GIVEN, FSI_USE_GRAPHS, FSI_LEARNED, FSI_FLUID_GMRES,
 * FSI_MLP_CUDA_CORES);
 * FSI_NO_RIGID_MODES, FSI_CLUSTER_COARSE, FSI_GRID_COARSE and FSI_NO_PDL are fixed at fsi_setup
 * (FSI_EINVAL if they differ). */
int fsi_set_flags(fsi_ctx* ctx, int flags);
/*
 * fsi_set_harvest - during later fsi_solve calls, store the preconditioned
 * residual r'_j = v_j - A P^-1 v_j of iterations j < nvec of each restart cycle
 * (a later cycle overwrites) into buf_dev + j*n (device, nvec x n doubles, owned
 * by the caller and kept valid while set).  nvec = 0 (or buf_dev NULL) stops it.
 */
int fsi_set_harvest(fsi_ctx* ctx, double* buf_dev, int nvec);

/*
 * fsi_check_device_errors - wait for the context's stream, then report whether a
 * bounded wait inside a kernel gave up since the last check (or the last fsi_solve,
 * which checks by itself): the grid barrier of the FSI_GRID_COARSE kernel, the
 * staged Chebyshev step (spmv_stage), the tensor-core MLP.  Such a wait gives up
 * after about a second, sets a flag and lets the kernel end, so the context stays
 * usable; the results of the calls since the last check are then not valid.
 * Returns FSI_OK, or FSI_ECUDA with the message naming the waits (flags cleared).
 * The asynchronous entry points (fsi_apply_block, fsi_apply_operator,
 * fsi_learned_apply, fsi_smoother_step) leave this check to the caller.
 */
int fsi_check_device_errors(fsi_ctx* ctx);

/*
 * fsi_debug_inject - fault injection for tests of the bounded waits (0: none, the
 * default).  Bit 1: the grid barrier of the FSI_GRID_COARSE kernel waits for one CTA
 * more than its launch has; bit 2: the tensor-core MLP does not commit its first
 * layer's MMAs to the barrier it then waits on.  The waits then run out (about a
 * second each) and fsi_check_device_errors / fsi_solve report FSI_ECUDA.  Applies to
 * the context's later launches; FSI_EINVAL for other bits.
 */
int fsi_debug_inject(fsi_ctx* ctx, int mask);

/*
 * Training of the stage on residuals r' of one or more contexts.  Loss per
 * residual: L = ||r' - A c(r')||^2 / ||r'||^2 (A of the context given), i.e. the
 * error e - c of the pair (r', e = A^-1 r') in the residual norm that the accept
 * test compares.  Gradients by backpropagation (dL/dc = -2 A^T (r' - A c) /
 * ||r'||^2, FP64; through the MLP in FP32 with the bfloat16 weights), AdamW
 * (decoupled weight decay) on FP32 master weights; the forward pass uses their
 * bfloat16 rounding.  Initial weights: Glorot uniform from SplitMix64
 * (draw i: splitmix64((seed << 32) + i), top 53 bits as a uniform in [0, 1)),
 * the last layer scaled by init_out_scale, biases zero.
 */
typedef struct fsi_train_params {
  double lr, beta1, beta2, eps, weight_decay;   /* AdamW (1e-3, 0.9, 0.999, 1e-8, 0) */
  uint64_t seed;
  double init_out_scale;                        /* (0.01) */
  float sigma_in[5], sigma_out[5];              /* class scales, > 0 */
  int dim;                                      /* mesh dimension trained on, 2 or 3 (2); fixes
                                                   the parameter count; fsi_trainer_step refuses
                                                   a context of the other dimension */
} fsi_train_params;
typedef struct fsi_trainer fsi_trainer;

void fsi_default_train_params(fsi_train_params* p);
int fsi_trainer_create(fsi_trainer** out, const fsi_train_params* p);
/* Add the gradient of L for r' (device, n doubles of ctx, which needs fsi_learned_setup); *loss
 * (nullable) receives L.  Runs on ctx's stream and waits for it. */
int fsi_trainer_step(fsi_trainer* tr, fsi_ctx* ctx, const double* rprime_dev, double* loss);
/* L for r' with the current weights, no gradient (validation).  Waits. */
int fsi_trainer_loss(fsi_trainer* tr, fsi_ctx* ctx, const double* rprime_dev, double* loss);
/* One AdamW step with the mean of the gradients added since the last update, at
 * learning rate lr (lr <= 0: the fsi_train_params rate), on ctx's stream; waits. */
int fsi_trainer_update(fsi_trainer* tr, fsi_ctx* ctx, double lr);
/* Replace the master weights (host, FSI_MLP_PARAMS[_3D] floats by the trainer's dim); resets the
 * AdamW moments and gradients. */
int fsi_trainer_set_master(fsi_trainer* tr, const float* params);
/* Copy out (host, nullable each): master weights (floats), bfloat16 weights, accumulated gradient (floats). */
int fsi_trainer_get(fsi_trainer* tr, float* master, uint16_t* params_bf16, float* grad);
/* Write the current weights with the trainer's class scales as a weights file. */
int fsi_trainer_save(fsi_trainer* tr, const char* path);
void fsi_trainer_free(fsi_trainer* tr);

#ifdef __cplusplus
}
#endif

#endif /* FSI_H_ */

// C ABI of the solver (declarations and contract in include/fsi.h).
#include "../../include/fsi.h"
#include "solver.cuh"
#include "spmv.cuh"
#include "vec.cuh"

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

struct fsi_ctx {
  fsi::Context C;
};

struct fsi_trainer {
  fsi::Trainer T;
};

namespace {

thread_local std::string g_setup_error;

// The context's launch knobs (SpMV unroll depth and L2 prefetch, programmatic
// dependent launch, the coarse V-cycle threshold, the MLP's unit) applied to this thread for one
// call, the thread's previous values restored afterwards.
struct KnobScope {
  fsi::SpmvTuning tuning;
  bool pdl, mlp_tc;
  int inject;
  double coarse_bytes;
  explicit KnobScope(const fsi::SolverParams& p)
      : tuning(fsi::spmv_tuning()), pdl(fsi::pdl_enabled()), mlp_tc(fsi::mlp_tensor_cores()),
        inject(fsi::fault_inject()), coarse_bytes(fsi::coarse_max_bytes()) {
    fsi::fault_inject() = p.inject;
    fsi::spmv_tuning().unroll = p.spmv_unroll;
    fsi::spmv_tuning().prefetch = p.spmv_prefetch;
    fsi::spmv_tuning().lane_shift = p.spmv_lane_shift;
    fsi::spmv_tuning().stage = p.spmv_stage;
    fsi::spmv_tuning().order = p.spmv_order;
    fsi::pdl_enabled() = (p.flags & FSI_NO_PDL) == 0;
    fsi::mlp_tensor_cores() = (p.flags & FSI_MLP_CUDA_CORES) == 0;
    fsi::coarse_max_bytes() = p.cluster_max_bytes;
  }
  ~KnobScope() {
    const int depth = fsi::spmv_tuning().setup_depth;
    fsi::spmv_tuning() = tuning;
    fsi::spmv_tuning().setup_depth = depth;
    fsi::pdl_enabled() = pdl;
    fsi::mlp_tensor_cores() = mlp_tc;
    fsi::fault_inject() = inject;
    fsi::coarse_max_bytes() = coarse_bytes;
  }
  KnobScope(const KnobScope&) = delete;
  KnobScope& operator=(const KnobScope&) = delete;
};

// Run f, turning exceptions into status codes; the message goes to the context
// (or, for calls without one, to the thread's fsi_last_error(NULL) text).  Calls
// with a context run on its device and with its launch knobs.
template <class F>
int guarded(fsi_ctx* ctx, F&& f) {
  std::string& err = ctx ? ctx->C.err : g_setup_error;
  try {
    fsi::DeviceGuard on_device(ctx ? ctx->C.device : -1);
    KnobScope knobs(ctx ? ctx->C.prm : fsi::SolverParams());
    f();
    err.clear();
    return FSI_OK;
  } catch (const fsi::Error& e) {
    err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    err = "host allocation failed";
    return FSI_ENOMEM;
  } catch (const std::exception& e) {
    err = e.what();
    return FSI_ECUDA;
  }
}

void to_solver_params(const fsi_params& p, fsi::SolverParams& s) {
  s.restart = p.restart;
  s.maxit = p.maxit;
  s.flags = p.flags;
  s.dt_theta = p.dt_theta;
  s.amg.theta = p.strength_theta;
  s.amg.coarse_max = p.coarse_max;
  s.amg.max_levels = p.max_levels;
  s.amg.cheb_degree = p.cheb_degree;
  s.amg.cheb_degree_coarse = p.cheb_degree_coarse;
  s.amg.cheb_ratio = p.cheb_ratio;
  s.amg.cheb_upper = p.cheb_upper;
  s.amg.power_iters = p.power_iters;
  s.amg.drop_tol = p.drop_tol;
  s.amg.presmooth = p.presmooth;
  s.amg.postsmooth = p.postsmooth;
  s.vc_mesh = p.vcycles_mesh;
  s.vc_solid = p.vcycles_solid;
  s.vc_fluid = p.vcycles_fluid;
  s.vc_pressure = p.vcycles_pressure;
  s.mass_degree = p.mass_degree;
  s.mass_ratio = p.mass_ratio;
  s.spmv_unroll = p.spmv_unroll;
  s.learned_accept = p.learned_accept;
  s.spmv_prefetch = p.spmv_prefetch;
  s.cluster_max_bytes = p.cluster_max_bytes;
  s.fluid_gmres_iters = p.fluid_gmres_iters;
  s.precond_variant = p.precond_variant;
  s.spmv_lane_shift = p.spmv_lane_shift;
  s.spmv_stage = p.spmv_stage;
  s.spmv_order = p.spmv_order;
}

void validate_params(const fsi::SolverParams& s) {
  using fsi::require;
  require(s.restart >= 1 && s.restart <= 1000, "restart must be in [1, 1000]");
  require(s.maxit >= 1, "maxit must be >= 1");
  require(s.amg.cheb_degree >= 1 && s.amg.presmooth >= 1 && s.amg.postsmooth >= 0, "smoother settings");
  require(s.amg.cheb_degree_coarse >= 0 && s.amg.cheb_degree_coarse <= 16, "cheb_degree_coarse must be in [0, 16]");
  require(s.amg.cheb_ratio > 1.0 && s.amg.cheb_upper >= 1.0, "Chebyshev interval settings");
  require(s.amg.coarse_max >= 1 && s.amg.max_levels >= 1 && s.amg.power_iters >= 1, "AMG level settings");
  require(s.vc_mesh >= 1 && s.vc_solid >= 1 && s.vc_fluid >= 1 && s.vc_pressure >= 1, "V-cycle counts");
  require(s.mass_degree >= 1 && s.mass_ratio > 1.0, "mass solve settings");
  require(std::isfinite(s.dt_theta), "dt_theta");
  require(s.spmv_unroll == 4 || s.spmv_unroll == 8, "spmv_unroll must be 4 or 8");
  require(s.learned_accept > 0.0 && s.learned_accept <= 1.0, "learned_accept must be in (0, 1]");
  require(s.spmv_prefetch >= 0 && s.spmv_prefetch <= 2, "spmv_prefetch must be 0, 1 or 2");
  require(s.cluster_max_bytes >= 0.0 && std::isfinite(s.cluster_max_bytes), "cluster_max_bytes must be >= 0");
  require(!((s.flags & FSI_CLUSTER_COARSE) && (s.flags & FSI_GRID_COARSE)),
          "FSI_CLUSTER_COARSE and FSI_GRID_COARSE exclude each other");
  require((s.flags & ~(FSI_X0_GIVEN | FSI_USE_GRAPHS | FSI_NO_RIGID_MODES | FSI_CLUSTER_COARSE | FSI_LEARNED |
                       FSI_NO_PDL | FSI_GRID_COARSE | FSI_FLUID_GMRES | FSI_MLP_CUDA_CORES)) == 0,
                 "unknown flag bits");
  require(s.fluid_gmres_iters >= 1 && s.fluid_gmres_iters <= fsi::kFluidGmresMax, "fluid_gmres_iters must be in [1, 32]");
  require(s.precond_variant >= FSI_PRECOND_LDU && s.precond_variant <= FSI_PRECOND_DIAG,
          "precond_variant must be FSI_PRECOND_LDU, _LOWER, _UPPER or _DIAG");
  require(s.spmv_lane_shift >= 0 && s.spmv_lane_shift <= 4, "spmv_lane_shift must be in [0, 4]");
  require(s.spmv_stage == 0 || s.spmv_stage == 1, "spmv_stage must be 0 or 1");
  require(s.spmv_order == 0 || s.spmv_order == 1, "spmv_order must be 0 or 1");
}

void validate_csr(int dim, int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
                  const int64_t* off) {
  using fsi::require;
  require(dim == 2 || dim == 3, "dim must be 2 or 3");
  require(n > 0 && n < (int64_t)1 << 31, "n out of range");
  require(rowptr && colind && off, "null CSR or offsets");
  require(off[0] == 0 && off[5] == n, "block_offsets must start at 0 and end at n");
  for (int k = 0; k < 5; ++k) require(off[k] <= off[k + 1], "block_offsets must be non-decreasing");
  for (int k = 0; k < 4; ++k) require((off[k + 1] - off[k]) % dim == 0, "vector classes must be multiples of dim");
  require(off[2] - off[1] == off[3] - off[2], "s_v and s_u must have the same size");
  require(rowptr[0] == 0, "rowptr[0] must be 0");
  for (int64_t r = 0; r < n; ++r) {
    require(rowptr[r + 1] >= rowptr[r], "rowptr must be non-decreasing");
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      require(colind[k] >= 0 && colind[k] < n, "column index out of range");
      require(k == rowptr[r] || colind[k] > colind[k - 1], "columns must be strictly increasing within a row");
      require(!vals || std::isfinite(vals[k]), "non-finite matrix value");
    }
  }
}

// The captured FGMRES iteration holds the learned stage's buffers and class
// scales by value: any change to them drops the graph (re-captured on the next solve).
void drop_graph(fsi::Context& C) {
  if (C.iter_graph) {
    cudaGraphExecDestroy(C.iter_graph);
    C.iter_graph = nullptr;
  }
}

}  // namespace

extern "C" {

void fsi_default_params(fsi_params* p, int dim) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->restart = 100;
  p->maxit = 1000;
  p->flags = 0;
  p->dt_theta = 0.01;
  p->strength_theta = 0.08;
  p->coarse_max = 1500;
  p->max_levels = 10;
  p->cheb_degree = 4;
  p->cheb_ratio = 30.0;
  p->cheb_upper = 1.3;
  p->power_iters = 15;
  p->drop_tol = 1e-10;
  p->presmooth = 1;
  p->postsmooth = 1;
  p->vcycles_mesh = 1;
  p->vcycles_solid = 2;
  p->vcycles_fluid = 1;
  p->vcycles_pressure = 1;
  p->mass_degree = 12;
  p->mass_ratio = dim == 3 ? 20.0 : 8.0;
  p->spmv_unroll = 4;
  p->learned_accept = 0.1;
  p->spmv_prefetch = 1;
  p->cluster_max_bytes = 6.0e6;
  p->cheb_degree_coarse = 2;
  p->fluid_gmres_iters = 4;
  p->precond_variant = FSI_PRECOND_LDU;
  p->spmv_lane_shift = 0;
  p->spmv_stage = 0;
  p->spmv_order = 1;
}

int fsi_setup(fsi_ctx** out, int dim, int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
              const int64_t* block_offsets, const double* node_coords, const fsi_params* p, void* cuda_stream) {
  if (!out) return FSI_EINVAL;
  *out = nullptr;
  fsi_ctx* ctx = nullptr;
  try {
    ctx = new fsi_ctx();
  } catch (...) {
    return FSI_ENOMEM;
  }
  int rc = guarded(ctx, [&] {
    validate_csr(dim, n, rowptr, colind, vals, block_offsets);
    fsi_params def;
    fsi_default_params(&def, dim);
    to_solver_params(p ? *p : def, ctx->C.prm);
    validate_params(ctx->C.prm);
    ctx->C.dim = dim;
    ctx->C.learned.dim = dim;
    ctx->C.n = n;
    for (int k = 0; k < 6; ++k) ctx->C.off[k] = block_offsets[k];
    if (cuda_stream) {
      ctx->C.s = static_cast<cudaStream_t>(cuda_stream);
    } else {
      FSI_CUDA(cudaStreamCreateWithFlags(&ctx->C.s, cudaStreamNonBlocking));
      ctx->C.own_stream = true;
    }
    KnobScope knobs(ctx->C.prm);
    fsi::context_setup(ctx->C, rowptr, colind, vals, node_coords);
  });
  if (rc != FSI_OK) {
    g_setup_error = ctx->C.err;
    delete ctx;
    return rc;
  }
  *out = ctx;
  return FSI_OK;
}

int fsi_update_values(fsi_ctx* ctx, const double* vals_dev) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::require(vals_dev != nullptr, "null values");
    fsi::context_update_values(ctx->C, vals_dev);
  });
}

int fsi_precond_build(fsi_ctx* ctx, int precision, const char* learned_weights) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::require(precision == FSI_FP64 || precision == FSI_FP32_AMG, "precision must be FSI_FP64 or FSI_FP32_AMG");
    fsi::precond_build(ctx->C, precision);
    if (learned_weights) {
      fsi::require(ctx->C.learned.n_nodes > 0, "learned_weights given before fsi_learned_setup");
      drop_graph(ctx->C);
      fsi::learned_load_file(ctx->C.learned, learned_weights, ctx->C.s);
    }
  });
}

int fsi_solve(fsi_ctx* ctx, const double* rhs_dev, double* x_dev, double rtol, fsi_stats* out) {
  if (!ctx) return FSI_EINVAL;
  int status = FSI_OK;
  int rc = guarded(ctx, [&] {
    fsi::require(rhs_dev && x_dev, "null rhs or x");
    fsi::require(rtol > 0.0 && std::isfinite(rtol), "rtol must be positive");
    status = fsi::fgmres_solve(ctx->C, rhs_dev, x_dev, rtol);
  });
  fsi::Context& C = ctx->C;
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->iters = C.last_iters;
    out->cycles = C.last_cycles;
    out->status = rc != FSI_OK ? rc : status;
    out->true_relres = C.last_true_relres;
    out->setup_s = C.setup_s;
    out->precond_build_s = C.build_s;
    out->solve_s = C.solve_s;
    if (C.built) {
      out->operator_bytes = fsi::operator_bytes(C);
      out->precond_bytes = fsi::precond_bytes(C, C.precision == 1 ? 4 : 8);
    }
    out->relres_hist = C.hist.empty() ? nullptr : C.hist.data();
    out->hist_len = (int)C.hist.size();
    out->kernel_launches = C.last_launches;
    out->learned_accepted = C.last_accepted;
    out->reorth_passes = C.last_reorth;
  }
  if (rc != FSI_OK) return rc;
  if (status == fsi::ENOTCONV_) C.err = "FGMRES reached maxit before rtol";
  if (status == fsi::EBREAKDOWN_) C.err = "Arnoldi breakdown before rtol";
  if (status == fsi::ENONFINITE_) C.err = "non-finite iterate";
  return status;
}

void fsi_free(fsi_ctx* ctx) { delete ctx; }

const char* fsi_last_error(const fsi_ctx* ctx) {
  if (!ctx) return g_setup_error.c_str();
  return ctx->C.err.c_str();
}

int fsi_apply_operator(fsi_ctx* ctx, const double* x_dev, double* y_dev) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::require(x_dev && y_dev, "null vector");
    fsi::apply_operator(ctx->C, x_dev, y_dev);
  });
}

int fsi_apply_block(fsi_ctx* ctx, int which, const double* in_dev, double* out_dev) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::Context& C = ctx->C;
    fsi::require(C.built, "fsi_apply_block before fsi_precond_build");
    fsi::require(in_dev && out_dev, "null vector");
    fsi::require(which >= 0 && which <= 7, "unknown block");
    const int64_t* o = C.off;
    const int64_t len[8] = {o[1] - o[0], o[2] - o[1], o[4] - o[3], o[5] - o[4], o[3] - o[2], o[3] - o[1],
                            o[5] - o[3], C.n};
    if (C.precision == 1) {
      auto& W = C.pw32;
      fsi::cast<double, float>(len[which], in_dev, W.in.p, C.s);
      fsi::apply_block<float>(C, which, W.in.p, W.out.p);
      fsi::cast<float, double>(len[which], W.out.p, out_dev, C.s);
    } else {
      fsi::apply_block<double>(C, which, in_dev, out_dev);
    }
  });
}

int fsi_smoother_step(fsi_ctx* ctx, int which, int level, int reps, double* bytes_per_step) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::Context& C = ctx->C;
    fsi::require(C.built, "fsi_smoother_step before fsi_precond_build");
    fsi::require(which >= 0 && which <= 3 && reps >= 0, "bad arguments");
    const double b = C.precision == 1 ? fsi::amg_smoother_steps<float>(C.H[which], level, reps, C.s)
                                      : fsi::amg_smoother_steps<double>(C.H[which], level, reps, C.s);
    if (bytes_per_step) *bytes_per_step = b;
  });
}

int fsi_amg_info(fsi_ctx* ctx, int which, int level, int64_t info[6], double* lambda) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::Context& C = ctx->C;
    fsi::require(C.built, "fsi_amg_info before fsi_precond_build");
    fsi::require(which >= 0 && which <= 3 && info, "bad arguments");
    fsi::Hierarchy& H = C.H[which];
    fsi::require(level >= 0 && level < (int)H.levels.size(), "level out of range");
    const fsi::AmgLevel& L = H.levels[level];
    info[0] = (int64_t)H.levels.size();
    info[1] = L.A.nbr;
    info[2] = L.A.br;
    info[3] = L.A.nnzb;
    info[4] = (level + 1 < (int)H.levels.size()) ? L.nagg : 0;
    info[5] = H.ncoarse;
    if (lambda) *lambda = L.lam;
  });
}

int fsi_amg_export(fsi_ctx* ctx, int which, int level, int what, void* dst) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::Context& C = ctx->C;
    fsi::require(C.built, "fsi_amg_export before fsi_precond_build");
    fsi::require(which >= 0 && which <= 3 && dst, "bad arguments");
    fsi::Hierarchy& H = C.H[which];
    fsi::require(level >= 0 && level < (int)H.levels.size(), "level out of range");
    const fsi::AmgLevel& L = H.levels[level];
    const bool has_p = level + 1 < (int)H.levels.size();
    auto cp = [&](const void* src, size_t bytes) {
      if (bytes) FSI_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, C.s));
    };
    switch (what) {
      case 0: fsi::require(has_p, "no aggregates on the coarsest level"); cp(L.agg.p, sizeof(int) * L.A.nbr); break;
      case 1: cp(L.A.rowptr.p, sizeof(int) * (L.A.nbr + 1)); break;
      case 2: cp(L.A.colind.p, sizeof(int) * L.A.nnzb); break;
      case 3: cp(L.A.v64.p, sizeof(double) * L.A.nnzb * L.A.br * L.A.bc); break;
      case 4: fsi::require(has_p, "no P on the coarsest level"); cp(L.P.rowptr.p, sizeof(int) * (L.P.nbr + 1)); break;
      case 5: fsi::require(has_p, "no P on the coarsest level"); cp(L.P.colind.p, sizeof(int) * L.P.nnzb); break;
      case 6: fsi::require(has_p, "no P on the coarsest level");
              cp(L.P.v64.p, sizeof(double) * L.P.nnzb * L.P.br * L.P.bc); break;
      case 7: fsi::require(has_p, "no P on the coarsest level"); *static_cast<int64_t*>(dst) = L.P.nnzb; break;
      default: throw fsi::Error(fsi::EINVAL_, "unknown export");
    }
    FSI_CUDA(cudaStreamSynchronize(C.s));
  });
}

int fsi_learned_setup(fsi_ctx* ctx, int64_t n_nodes, const int32_t* node_dof, const int32_t* patch) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    drop_graph(ctx->C);
    fsi::learned_set_geometry(ctx->C.learned, ctx->C.n, n_nodes, node_dof, patch, ctx->C.s);
  });
}

int fsi_learned_load(fsi_ctx* ctx, const char* path) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::require(path != nullptr, "null path");
    drop_graph(ctx->C);
    fsi::learned_load_file(ctx->C.learned, path, ctx->C.s);
  });
}

int fsi_learned_set_weights(fsi_ctx* ctx, const float* sigma_in, const float* sigma_out, const uint16_t* params) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::require(sigma_in && sigma_out && params, "null argument");
    drop_graph(ctx->C);
    fsi::learned_set_weights(ctx->C.learned, sigma_in, sigma_out, params, ctx->C.s);
  });
}

int fsi_learned_apply(fsi_ctx* ctx, const double* r_dev, double* c_dev) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::Learned& L = ctx->C.learned;
    fsi::require(L.n_nodes > 0 && L.has_weights, "fsi_learned_apply needs fsi_learned_setup and weights");
    fsi::require(r_dev && c_dev, "null vector");
    fsi::mlp_apply(fsi::learned_geom(L, ctx->C.off), L.w16.p, r_dev, c_dev, ctx->C.s);
  });
}

int fsi_learned_features(fsi_ctx* ctx, const double* r_dev, float* feat_dev, float* rho_dev) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::Learned& L = ctx->C.learned;
    fsi::require(L.n_nodes > 0, "fsi_learned_features needs fsi_learned_setup");
    fsi::require(r_dev && feat_dev && rho_dev, "null vector");
    fsi::mlp_features(fsi::learned_geom(L, ctx->C.off), r_dev, feat_dev, rho_dev, ctx->C.s);
  });
}

int fsi_set_learned_accept(fsi_ctx* ctx, double tau) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::require(tau > 0.0 && tau <= 1.0, "learned_accept must be in (0, 1]");
    drop_graph(ctx->C);
    ctx->C.prm.learned_accept = tau;
  });
}

int fsi_set_flags(fsi_ctx* ctx, int flags) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    constexpr int fixed = FSI_NO_RIGID_MODES | FSI_CLUSTER_COARSE | FSI_NO_PDL | FSI_GRID_COARSE;
    constexpr int known = FSI_X0_GIVEN | FSI_USE_GRAPHS | FSI_NO_RIGID_MODES | FSI_CLUSTER_COARSE | FSI_LEARNED |
                          FSI_NO_PDL | FSI_GRID_COARSE | FSI_FLUID_GMRES | FSI_MLP_CUDA_CORES;
    fsi::require((flags & ~known) == 0, "unknown flag bits");
    fsi::require((flags & fixed) == (ctx->C.prm.flags & fixed),
                 "FSI_NO_RIGID_MODES, FSI_CLUSTER_COARSE, FSI_GRID_COARSE and FSI_NO_PDL are fixed at fsi_setup");
    ctx->C.prm.flags = flags;
  });
}

int fsi_debug_inject(fsi_ctx* ctx, int mask) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::require((mask & ~(fsi::kInjectCoarseBarrier | fsi::kInjectMlpCommit)) == 0, "unknown injection bits");
    drop_graph(ctx->C);   // the captured iteration holds the launch arguments of its capture
    ctx->C.prm.inject = mask;
  });
}

int fsi_check_device_errors(fsi_ctx* ctx) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::Context& C = ctx->C;
    FSI_CUDA(cudaStreamSynchronize(C.s));
    std::string what;
    if (C.built && (C.prm.flags & FSI_GRID_COARSE)) {
      bool failed = false;
      for (auto& H : C.H) failed = fsi::coarse_failed(H, C.s) || failed;
      if (failed) what += " a grid barrier of the coarse-level kernel;";
    }
    if (fsi::spmv_stage_failed(C.s)) what += " a staged Chebyshev step;";
    if (C.learned.counters.p) {
      int e = 0;
      FSI_CUDA(cudaMemcpy(&e, C.learned.counters.p + 2, sizeof(int), cudaMemcpyDeviceToHost));
      if (e) {
        FSI_CUDA(cudaMemset(C.learned.counters.p + 2, 0, sizeof(int)));
        what += " the tensor-core MLP;";
      }
    }
    if (!what.empty())
      throw fsi::Error(fsi::ECUDA_, "bounded waits timed out in" + what + " those results are not valid");
  });
}

int fsi_set_harvest(fsi_ctx* ctx, double* buf_dev, int nvec) {
  if (!ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::require(nvec >= 0, "nvec must be >= 0");
    if (!buf_dev || nvec == 0) {
      ctx->C.harvest = nullptr;
      ctx->C.harvest_n = 0;
    } else {
      ctx->C.harvest = buf_dev;
      ctx->C.harvest_n = nvec;
    }
  });
}

void fsi_default_train_params(fsi_train_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->lr = 1e-3;
  p->beta1 = 0.9;
  p->beta2 = 0.999;
  p->eps = 1e-8;
  p->weight_decay = 0.0;
  p->seed = 0;
  p->init_out_scale = 0.01;
  p->dim = 2;
  for (int k = 0; k < 5; ++k) p->sigma_in[k] = p->sigma_out[k] = 1.0f;
}

int fsi_trainer_create(fsi_trainer** out, const fsi_train_params* p) {
  if (!out) return FSI_EINVAL;
  *out = nullptr;
  fsi_trainer* tr = nullptr;
  try {
    tr = new fsi_trainer();
  } catch (...) {
    return FSI_ENOMEM;
  }
  int rc = guarded(nullptr, [&] {
    fsi_train_params def;
    fsi_default_train_params(&def);
    const fsi_train_params& q = p ? *p : def;
    fsi::TrainParams tp;
    tp.lr = q.lr; tp.beta1 = q.beta1; tp.beta2 = q.beta2; tp.eps = q.eps; tp.weight_decay = q.weight_decay;
    tp.seed = q.seed;
    tp.dim = q.dim;
    tp.init_out_scale = q.init_out_scale;
    for (int k = 0; k < 5; ++k) { tp.sig_in[k] = q.sigma_in[k]; tp.sig_out[k] = q.sigma_out[k]; }
    fsi::trainer_init(tr->T, tp);
  });
  if (rc != FSI_OK) {
    delete tr;
    return rc;
  }
  *out = tr;
  return FSI_OK;
}

int fsi_trainer_step(fsi_trainer* tr, fsi_ctx* ctx, const double* rprime_dev, double* loss) {
  if (!tr || !ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::require(rprime_dev != nullptr, "null vector");
    const double L = fsi::trainer_step(tr->T, ctx->C, rprime_dev);
    if (loss) *loss = L;
  });
}

int fsi_trainer_loss(fsi_trainer* tr, fsi_ctx* ctx, const double* rprime_dev, double* loss) {
  if (!tr || !ctx) return FSI_EINVAL;
  return guarded(ctx, [&] {
    fsi::require(rprime_dev != nullptr, "null vector");
    const double L = fsi::trainer_step(tr->T, ctx->C, rprime_dev, false);
    if (loss) *loss = L;
  });
}

int fsi_trainer_update(fsi_trainer* tr, fsi_ctx* ctx, double lr) {
  if (!tr || !ctx) return FSI_EINVAL;
  return guarded(ctx, [&] { fsi::trainer_update(tr->T, ctx->C.s, lr); });
}

int fsi_trainer_set_master(fsi_trainer* tr, const float* params) {
  if (!tr || !params) return FSI_EINVAL;
  return guarded(nullptr, [&] { fsi::trainer_set_master(tr->T, params); });
}

int fsi_trainer_get(fsi_trainer* tr, float* master, uint16_t* params_bf16, float* grad) {
  if (!tr) return FSI_EINVAL;
  return guarded(nullptr, [&] {
    FSI_CUDA(cudaDeviceSynchronize());
    const size_t np = (size_t)tr->T.n_params();
    if (master) FSI_CUDA(cudaMemcpy(master, tr->T.master.p, sizeof(float) * np, cudaMemcpyDeviceToHost));
    if (params_bf16) FSI_CUDA(cudaMemcpy(params_bf16, tr->T.w16.p, sizeof(uint16_t) * np, cudaMemcpyDeviceToHost));
    if (grad) FSI_CUDA(cudaMemcpy(grad, tr->T.grad.p, sizeof(float) * np, cudaMemcpyDeviceToHost));
  });
}

int fsi_trainer_save(fsi_trainer* tr, const char* path) {
  if (!tr || !path) return FSI_EINVAL;
  return guarded(nullptr, [&] {
    std::vector<uint16_t> h((size_t)tr->T.n_params());
    FSI_CUDA(cudaDeviceSynchronize());
    FSI_CUDA(cudaMemcpy(h.data(), tr->T.w16.p, sizeof(uint16_t) * h.size(), cudaMemcpyDeviceToHost));
    fsi::learned_save_file(path, tr->T.prm.dim, tr->T.prm.sig_in, tr->T.prm.sig_out, h.data());
  });
}

void fsi_trainer_free(fsi_trainer* tr) { delete tr; }

}  // extern "C"

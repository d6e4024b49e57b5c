// Learned correction stage of the FGMRES solve (the learned form; an extra
// smoothing step after the Alg. 2 preconditioner, not part of the paper).
//
// Per Q2 node a of a D-dimensional mesh (D = 2, 3), with its 3^D lattice patch N(a)
// and the C = 2D+1 components v (D), u (D), p of a node:
//   x_{s,k} = r'[dof_k(N_s(a))] / sigma_in[class]   (0 if absent)
//   rho_a   = sqrt(mean of the 3^D C squares)
//   f_a     = [x / rho_a, one-hot lattice parity (2^D), solid / v fixed / u fixed / interface (4)]
//   y_a     = W3^T gelu(W2^T gelu(W1^T f_a + b1) + b2) + b3        (53 -> 64 -> 64 -> 5 in 2D,
//                                                                   201 -> 64 -> 64 -> 7 in 3D)
//   c[dof_k(a)] = y_{a,k} rho_a sigma_out[class]     (0 on fixed rows and at rho_a = 0)
// Weights are bfloat16, products and sums FP32; the correction is written in FP64.
//
// Training minimises the residual left by the correction, ||r' - A c(r')||^2 / ||r'||^2
// (the error e - c of the pair (r', e = A^-1 r') measured in the residual norm that
// FGMRES's acceptance test compares), by backpropagation through the MLP with the
// gradient dL/dc = -2 A^T (r' - A c) / ||r'||^2, and AdamW on FP32 master weights.
#pragma once
#include "common.cuh"

#include <cstdint>

namespace fsi {

// Layout of the per-node MLP on a D-dimensional mesh; the parameter vector is
// W1 [kIn][kHidden], b1, W2 [kHidden][kHidden], b2, W3 [kHidden][kOut], b3.
template <int D>
struct Net {
  static_assert(D == 2 || D == 3, "2D or 3D meshes");
  static constexpr int kComp = 2 * D + 1;             // v (D), u (D), p
  static constexpr int kSlots = D == 2 ? 9 : 27;      // 3^D lattice neighbours
  static constexpr int kPatch = kSlots * kComp;
  static constexpr int kPar = 1 << D;                 // lattice parity classes
  static constexpr int kIn = kPatch + kPar + 4, kHidden = 64, kOut = kComp;
  static constexpr int kW1 = 0, kB1 = kW1 + kIn * kHidden, kW2 = kB1 + kHidden, kB2 = kW2 + kHidden * kHidden,
                       kW3 = kB2 + kHidden, kB3 = kW3 + kHidden * kOut, kParams = kB3 + kOut;
};
inline int mlp_params(int dim) { return dim == 3 ? Net<3>::kParams : Net<2>::kParams; }
inline int mlp_inputs(int dim) { return dim == 3 ? Net<3>::kIn : Net<2>::kIn; }

// The 2D layout under its own names (the tensor-core kernel is 2D only).
constexpr int kMlpIn = Net<2>::kIn, kMlpHidden = Net<2>::kHidden, kMlpOut = Net<2>::kOut,
              kMlpPatch = Net<2>::kPatch, kMlpSlots = Net<2>::kSlots;
constexpr int kW1 = Net<2>::kW1, kB1 = Net<2>::kB1, kW2 = Net<2>::kW2, kB2 = Net<2>::kB2, kW3 = Net<2>::kW3,
              kB3 = Net<2>::kB3, kMlpParams = Net<2>::kParams;
static_assert(kMlpParams == 7941 && Net<3>::kParams == 17543, "parameter counts");

// Node flags (fourth entry of a node's int4 record); the four flag inputs of the
// MLP are bits 0..3 in this order, the lattice parity bits i, j, k odd are 4, 5, 7.
enum NodeFlags {
  NF_SOLID = 1, NF_VFIX = 2, NF_UFIX = 4, NF_IFACE = 8, NF_IODD = 16, NF_JODD = 32, NF_PFIX = 64, NF_KODD = 128
};

// Everything the per-node kernels read besides the vectors (passed by value).
struct MlpGeom {
  int dim = 2;
  int64_t n_nodes = 0;
  const int4* node_dof = nullptr;   // {first v DOF, first u DOF, p DOF or -1, flags}
  const int* patch = nullptr;       // 3^dim per node, -1 outside the mesh
  int64_t off1 = 0, off2 = 0, off3 = 0, off4 = 0;   // class boundaries s_v, s_u, f_v, f_p
  float sig_in[5] = {1, 1, 1, 1, 1};
  float inv_in[5] = {1, 1, 1, 1, 1};   // 1 / sig_in
  float sig_out[5] = {1, 1, 1, 1, 1};
  int* err = nullptr;                  // set to 1 by the tensor-core MLP when a wait gives up
};

// The stage as one context holds it.
struct Learned {
  int dim = 2;                 // the mesh's; fixes the MLP's layout (Net<dim>)
  int64_t n_nodes = 0;
  DBuf<int4> node_dof;
  DBuf<int> patch;
  DBuf<uint16_t> w16;          // Net<dim>::kParams bfloat16 parameters
  float sig_in[5] = {1, 1, 1, 1, 1}, sig_out[5] = {1, 1, 1, 1, 1};
  bool has_weights = false;
  DBuf<double> rp, c, t;       // r', correction, A c (length n)
  DBuf<double> part;           // 2 x kRedBlocks reduction partials
  DBuf<int> counters;          // [0] accept flag of the current iteration, [1] corrections accepted,
                               // [2] tensor-core MLP error flag (sticky until a solve reports it)
};

// Validate and upload the node map (host arrays) of a system with n DOFs (L.dim set).
void learned_set_geometry(Learned& L, int64_t n, int64_t n_nodes, const int32_t* node_dof, const int32_t* patch,
                          cudaStream_t s);
// Set weights (host bfloat16 parameters, Net<L.dim>::kParams, and class scales).
void learned_set_weights(Learned& L, const float* sig_in, const float* sig_out, const uint16_t* params,
                         cudaStream_t s);
// Read a weights file (8-byte magic "FSIMLP01", int32 n_in n_hidden n_out 0,
// float32 sigma_in[5] sigma_out[5], then the bfloat16 parameters, little endian).
void learned_load_file(Learned& L, const char* path, cudaStream_t s);
void learned_save_file(const char* path, int dim, const float* sig_in, const float* sig_out,
                       const uint16_t* params);
MlpGeom learned_geom(const Learned& L, const int64_t off[6]);

// c = MLP(r'), every DOF of c written: on the tensor cores (mlp_tc.cu) when the
// thread's mlp_tensor_cores() knob is set, g.err is given and the mesh is 2D, else
// on the CUDA cores.
void mlp_apply(const MlpGeom& g, const uint16_t* w16, const double* rp, double* c, cudaStream_t s);
// The tensor-core form: tcgen05.mma (kind::tf32) with the activations split into
// two TF32 terms, FP32 accumulation; *err = 1 if a wait for the MMAs gave up.
void mlp_apply_tc(const MlpGeom& g, const uint16_t* w16, const double* rp, double* c, int* err, cudaStream_t s);
// Feature rows (node-major [n_nodes][Net<g.dim>::kIn]) and rho of r'.
void mlp_features(const MlpGeom& g, const double* rp, float* F, float* rho, cudaStream_t s);

// FGMRES stage pieces (the column index j is read on the device):
// rp = V_j - w and per-block sums of rp^2 into part[0, kRedBlocks)
void learned_residual(int64_t n, const double* V, int64_t ldv, const int* jdev, const double* w, double* rp,
                      double* part, cudaStream_t s);
// per-block sums of (rp - t)^2 into part[kRedBlocks, 2 kRedBlocks); then the
// accept flag (sum_b < tau^2 sum_a, both finite) into counters[0], counters[1] += flag
void learned_decide(int64_t n, const double* rp, const double* t, double tau, double* part, int* counters,
                    cudaStream_t s);
// if counters[0]: Z_j += c, w += t
void learned_commit(int64_t n, const int* counters, const double* c, const double* t, double* Z, int64_t ldz,
                    const int* jdev, double* w, cudaStream_t s);
// buf[j*n + i] = V_j[i] - w[i] for j < nvec (harvest of the preconditioned residuals)
void harvest_residual(int64_t n, const double* V, int64_t ldv, const int* jdev, const double* w, double* buf,
                      int nvec, cudaStream_t s);

// ---------------------------------------------------------------- training
struct TrainParams {
  int dim = 2;                    // mesh dimension of the contexts trained on
  double lr = 1e-3, beta1 = 0.9, beta2 = 0.999, eps = 1e-8, weight_decay = 0.0;
  uint64_t seed = 0;
  double init_out_scale = 0.01;   // last layer initialised this much smaller than Glorot
  float sig_in[5] = {1, 1, 1, 1, 1}, sig_out[5] = {1, 1, 1, 1, 1};
};

struct Trainer {
  TrainParams prm;
  int64_t cap_nodes = 0, cap_n = 0;
  DBuf<float> master, m, v, grad;  // Net<prm.dim>::kParams each
  DBuf<uint16_t> w16;
  DBuf<float> F, rho, H1, H2, dY, dH1, dH2;   // column-major: row k of node a at [k * cap_nodes + a]
  DBuf<float> partial;
  DBuf<double> c, t, res, g, part, scal;
  int grads = 0;        // gradient contributions since the last update
  int64_t steps = 0;    // AdamW steps taken
  double* pinned = nullptr;
  int n_params() const { return mlp_params(prm.dim); }
  ~Trainer();
};

}  // namespace fsi

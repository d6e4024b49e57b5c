// Learned correction stage: per-node MLP inference, the FGMRES accept/fallback
// step, residual harvest, and the training kernels (forward with stored
// activations, backward through the MLP, weight-gradient sums, AdamW).
#include "learned.cuh"
#include "solver.cuh"
#include "vec.cuh"
#include "spmv.cuh"

#include <cmath>
#include <cstring>
#include <fstream>
#include <vector>

namespace fsi {

namespace {

constexpr int kNodeThreads = 128;
template <int D>
constexpr int params_padded() { return (Net<D>::kParams + 3) / 4 * 4; }
static_assert(kB1 % 4 == 0 && kW2 % 4 == 0 && kB2 % 4 == 0 && kW3 % 4 == 0, "float4 rows (2D)");
static_assert(Net<3>::kB1 % 4 == 0 && Net<3>::kW2 % 4 == 0 && Net<3>::kB2 % 4 == 0 && Net<3>::kW3 % 4 == 0,
              "float4 rows (3D)");

__host__ __device__ inline float bf16_to_f32(uint16_t h) {
#ifdef __CUDA_ARCH__
  return __uint_as_float((uint32_t)h << 16);
#else
  uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

__host__ __device__ inline uint16_t f32_to_bf16(float f) {   // round to nearest, ties to even
#ifdef __CUDA_ARCH__
  uint32_t u = __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
#endif
  const uint32_t lsb = (u >> 16) & 1u;
  return (uint16_t)((u + 0x7FFFu + lsb) >> 16);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

__device__ __forceinline__ int cls_of(const MlpGeom& g, int64_t d) {
  return (d >= g.off1) + (d >= g.off2) + (d >= g.off3) + (d >= g.off4);
}

// a[k] for a per-class array held in the kernel parameters
__device__ __forceinline__ float pick5(const float (&a)[5], int k) {
  return k == 0 ? a[0] : k == 1 ? a[1] : k == 2 ? a[2] : k == 3 ? a[3] : a[4];
}

template <int D>
__device__ __forceinline__ void load_weights(float* W, const uint16_t* __restrict__ w16) {
  for (int i = threadIdx.x; i < Net<D>::kParams; i += blockDim.x) W[i] = bf16_to_f32(w16[i]);
  __syncthreads();
}

enum { MODE_APPLY = 0, MODE_FEATURES = 1, MODE_TRAIN = 2 };

// Lattice parity class of a node: (i odd) + 2 (j odd) [+ 4 (k odd)].
template <int D>
__device__ __forceinline__ int parity_of(int fl) {
  const int p = ((fl >> 4) & 1) | (((fl >> 5) & 1) << 1);
  return D == 3 ? p | (((fl >> 7) & 1) << 2) : p;
}

// One thread per node: gather the patch, normalise, run the MLP (MODE_APPLY,
// MODE_TRAIN) and scatter the correction; MODE_TRAIN also stores the features
// and pre-activations column-major (row k of node a at [k * ld + a]).
//
// Dynamic shared memory: the weights as FP32 (params_padded<D>() floats), then
// one column per thread (act[k * kNodeThreads + t]) holding the hidden
// activations and, in MODE_FEATURES / MODE_TRAIN, first the gathered patch.  The
// layers loop over their inputs (read from the thread's column) with the 64
// accumulators in registers, so the kernel body stays small enough for the
// instruction cache.  MODE_APPLY folds the patch into layer 1 as it gathers it
// (W1^T (x / rho) = (sum_i x_i W1[i]) / rho), so its column is 64 rows: 2D 64 KB
// (three CTAs per SM), 3D 102 KB (two).  3D training: 163 KB (one).
template <int D, int MODE>
constexpr int act_rows() {
  return MODE != MODE_APPLY && Net<D>::kPatch > Net<D>::kHidden ? Net<D>::kPatch : Net<D>::kHidden;
}
template <int D, int MODE>
constexpr size_t mlp_smem() {
  return sizeof(float) * ((size_t)params_padded<D>() + (size_t)act_rows<D, MODE>() * kNodeThreads);
}

// The node record of patch entry q (q = -1: outside the mesh, no DOFs).
__device__ __forceinline__ int4 node_rec(const MlpGeom& g, int q) {
  return q >= 0 ? g.node_dof[q] : make_int4(-1, -1, -1, 0);
}

// Issue the loads of one patch node's r' values (raw FP64) and class scales.
template <int D>
__device__ __forceinline__ void load_node_vals(const MlpGeom& g, const double* __restrict__ rp, int4 r,
                                               double (&ev)[2 * D + 1], float (&sc)[3]) {
#pragma unroll
  for (int k = 0; k < 2 * D + 1; ++k) ev[k] = 0.0;
  sc[0] = sc[1] = sc[2] = 0.f;
  if (r.x >= 0) {
    sc[0] = pick5(g.inv_in, cls_of(g, r.x));
    sc[1] = pick5(g.inv_in, cls_of(g, r.y));
#pragma unroll
    for (int k = 0; k < D; ++k) {
      ev[k] = rp[r.x + k];
      ev[D + k] = rp[r.y + k];
    }
    if (r.z >= 0) {
      sc[2] = pick5(g.inv_in, cls_of(g, r.z));
      ev[2 * D] = rp[r.z];
    }
  }
}

// (MODE_FEATURES ends each node after the features: the layers below are then
// unreachable, which the front end would report once per instantiation)
#pragma nv_diag_suppress 128
template <int D, int MODE>
__global__ void __launch_bounds__(kNodeThreads) k_mlp(MlpGeom g, const uint16_t* __restrict__ w16,
                                                      const double* __restrict__ rp, double* __restrict__ c,
                                                      float* __restrict__ F, float* __restrict__ rho_out,
                                                      float* __restrict__ H1, float* __restrict__ H2, int64_t ld) {
  using N = Net<D>;
  constexpr int kC = N::kComp, kH = N::kHidden;
  extern __shared__ __align__(16) float smem[];
  float* W = smem;
  float* act = smem + params_padded<D>();
  const int t = threadIdx.x;
  // the weights do not depend on earlier kernels: load them before waiting for the previous one
  if (MODE != MODE_FEATURES) load_weights<D>(W, w16);
  dep_wait();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // the block loops in lockstep so that the weights stay loaded; idle threads skip the work
  const int64_t nb = (g.n_nodes + blockDim.x - 1) / blockDim.x * blockDim.x;
  for (int64_t a0 = blockIdx.x * (int64_t)blockDim.x; a0 < nb; a0 += stride) {
    const int64_t a = a0 + t;
    if (a >= g.n_nodes) continue;
    const int4 me = g.node_dof[a];
    const int fl = me.w;
    const int par = parity_of<D>(fl);
    float h[kH];
    float rho, inv_rho;
    if constexpr (MODE == MODE_APPLY) {
      // gather and layer 1 in one pass, software-pipelined: while slot s's kC x 64
      // FMAs run, the r' values of slot s+1, the node record of slot s+2 and the
      // patch entry of slot s+3 are in flight
      const int* pa = g.patch + a * N::kSlots;
#pragma unroll
      for (int j = 0; j < kH; ++j) h[j] = 0.f;
      float ss = 0.f;
      double ev[kC];
      float sc[3];
      load_node_vals<D>(g, rp, node_rec(g, pa[0]), ev, sc);
      int4 r1 = node_rec(g, pa[1]);
      int q2 = pa[2];
#pragma unroll 1
      for (int s = 0; s < N::kSlots; ++s) {
        double evn[kC];
        float scn[3];
        load_node_vals<D>(g, rp, r1, evn, scn);                 // slot s+1 (r1.x = -1 past the end)
        const int4 r2 = node_rec(g, q2);                         // slot s+2
        const int q3 = s + 3 < N::kSlots ? pa[s + 3] : -1;       // slot s+3
        float e[kC];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          e[k] = (float)ev[k] * sc[0];
          e[D + k] = (float)ev[D + k] * sc[1];
        }
        e[2 * D] = (float)ev[2 * D] * sc[2];
        float sl = e[0] * e[0];
#pragma unroll
        for (int k = 1; k < kC; ++k) sl += e[k] * e[k];
        ss += sl;
        const float4* w4 = reinterpret_cast<const float4*>(W + N::kW1 + kC * s * kH);
#pragma unroll
        for (int k = 0; k < kC; ++k) {
          const float xi = e[k];
#pragma unroll
          for (int q = 0; q < kH / 4; ++q) {
            const float4 w = w4[k * (kH / 4) + q];
            h[4 * q + 0] += xi * w.x; h[4 * q + 1] += xi * w.y; h[4 * q + 2] += xi * w.z; h[4 * q + 3] += xi * w.w;
          }
        }
#pragma unroll
        for (int k = 0; k < kC; ++k) ev[k] = evn[k];
        sc[0] = scn[0]; sc[1] = scn[1]; sc[2] = scn[2];
        r1 = r2;
        q2 = q3;
      }
      rho = sqrtf(ss * (1.0f / N::kPatch));
      inv_rho = rho > 0.f ? 1.0f / rho : 0.f;
      // h = (sum_i x_i W1[i]) / rho + b1 + the one-hot row + the flag rows
      const float* wp = W + N::kW1 + (N::kPatch + par) * kH;
#pragma unroll
      for (int j = 0; j < kH; ++j) h[j] = h[j] * inv_rho + (W[N::kB1 + j] + wp[j]);
    } else {
      // gather x (unnormalised) into the thread's column and sum its squares
      float ss = 0.f;
#pragma unroll(D == 2 ? 9 : 3)
      for (int s = 0; s < N::kSlots; ++s) {
        const int q = g.patch[a * N::kSlots + s];
        float e[kC];
#pragma unroll
        for (int k = 0; k < kC; ++k) e[k] = 0.f;
        if (q >= 0) {
          const int4 r = g.node_dof[q];
          const float iv = pick5(g.inv_in, cls_of(g, r.x));
          const float iu = pick5(g.inv_in, cls_of(g, r.y));
#pragma unroll
          for (int k = 0; k < D; ++k) {
            e[k] = (float)rp[r.x + k] * iv;
            e[D + k] = (float)rp[r.y + k] * iu;
          }
          if (r.z >= 0) e[2 * D] = (float)rp[r.z] * pick5(g.inv_in, cls_of(g, r.z));
        }
        float sl = e[0] * e[0];
#pragma unroll
        for (int k = 1; k < kC; ++k) sl += e[k] * e[k];
        ss += sl;
#pragma unroll
        for (int k = 0; k < kC; ++k) act[(kC * s + k) * kNodeThreads + t] = e[k];
      }
      rho = sqrtf(ss * (1.0f / N::kPatch));
      inv_rho = rho > 0.f ? 1.0f / rho : 0.f;
      if constexpr (MODE == MODE_FEATURES) {
        float* row = F + a * N::kIn;
        for (int k = 0; k < N::kPatch; ++k) row[k] = act[k * kNodeThreads + t] * inv_rho;
#pragma unroll
        for (int k = 0; k < N::kPar; ++k) row[N::kPatch + k] = (k == par) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) row[N::kPatch + N::kPar + k] = ((fl >> k) & 1) ? 1.f : 0.f;
        rho_out[a] = rho;
        continue;
      }
      for (int k = 0; k < N::kPatch; ++k) F[k * ld + a] = act[k * kNodeThreads + t] * inv_rho;
#pragma unroll
      for (int k = 0; k < N::kPar; ++k) F[(N::kPatch + k) * ld + a] = (k == par) ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) F[(N::kPatch + N::kPar + k) * ld + a] = ((fl >> k) & 1) ? 1.f : 0.f;
      rho_out[a] = rho;
      // layer 1: h = W1^T f + b1 (the one-hot and flag inputs add their weight rows below)
      {
        const float* wp = W + N::kW1 + (N::kPatch + par) * kH;
#pragma unroll
        for (int j = 0; j < kH; ++j) h[j] = W[N::kB1 + j] + wp[j];
      }
#pragma unroll 1
      for (int i = 0; i < N::kPatch; ++i) {
        const float xi = act[i * kNodeThreads + t] * inv_rho;
        const float4* w4 = reinterpret_cast<const float4*>(W + N::kW1 + i * kH);
#pragma unroll
        for (int q = 0; q < kH / 4; ++q) {
          const float4 w = w4[q];
          h[4 * q + 0] += xi * w.x; h[4 * q + 1] += xi * w.y; h[4 * q + 2] += xi * w.z; h[4 * q + 3] += xi * w.w;
        }
      }
    }
    const bool live = rho > 0.f;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      if ((fl >> k) & 1) {   // flag inputs: NF_SOLID, NF_VFIX, NF_UFIX, NF_IFACE are bits 0..3
        const float4* w4 = reinterpret_cast<const float4*>(W + N::kW1 + (N::kPatch + N::kPar + k) * kH);
#pragma unroll
        for (int q = 0; q < kH / 4; ++q) {
          const float4 w = w4[q];
          h[4 * q + 0] += w.x; h[4 * q + 1] += w.y; h[4 * q + 2] += w.z; h[4 * q + 3] += w.w;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kH; ++j) {
      act[j * kNodeThreads + t] = h[j];
      if (MODE == MODE_TRAIN) H1[j * ld + a] = h[j];
    }
#pragma unroll 1
    for (int j = 0; j < kH; ++j) act[j * kNodeThreads + t] = gelu(act[j * kNodeThreads + t]);
    // layer 2: h = W2^T gelu(h1) + b2
#pragma unroll
    for (int j = 0; j < kH; ++j) h[j] = W[N::kB2 + j];
#pragma unroll 1
    for (int i = 0; i < kH; ++i) {
      const float hv = act[i * kNodeThreads + t];
      const float4* w4 = reinterpret_cast<const float4*>(W + N::kW2 + i * kH);
#pragma unroll
      for (int q = 0; q < kH / 4; ++q) {
        const float4 w = w4[q];
        h[4 * q + 0] += hv * w.x; h[4 * q + 1] += hv * w.y; h[4 * q + 2] += hv * w.z; h[4 * q + 3] += hv * w.w;
      }
    }
#pragma unroll
    for (int j = 0; j < kH; ++j) {
      act[j * kNodeThreads + t] = h[j];
      if (MODE == MODE_TRAIN) H2[j * ld + a] = h[j];
    }
    // layer 3: y = W3^T gelu(h2) + b3
    float y[N::kOut];
#pragma unroll
    for (int o = 0; o < N::kOut; ++o) y[o] = W[N::kB3 + o];
#pragma unroll 1
    for (int j = 0; j < kH; ++j) {
      const float a2 = gelu(act[j * kNodeThreads + t]);
      const float* w3 = W + N::kW3 + j * N::kOut;
#pragma unroll
      for (int o = 0; o < N::kOut; ++o) y[o] += a2 * w3[o];
    }
    // scatter c = y rho sigma_out on the node's free DOFs
    const double rr = (double)rho;
    const double sv = live && !(fl & NF_VFIX) ? rr * (double)pick5(g.sig_out, cls_of(g, me.x)) : 0.0;
    const double su = live && !(fl & NF_UFIX) ? rr * (double)pick5(g.sig_out, cls_of(g, me.y)) : 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      c[me.x + k] = sv != 0.0 ? (double)y[k] * sv : 0.0;
      c[me.y + k] = su != 0.0 ? (double)y[D + k] * su : 0.0;
    }
    if (me.z >= 0) {
      const double sp = live && !(fl & NF_PFIX) ? rr * (double)pick5(g.sig_out, cls_of(g, me.z)) : 0.0;
      c[me.z] = sp != 0.0 ? (double)y[2 * D] * sp : 0.0;
    }
  }
}

#pragma nv_diag_default 128

template <int D, int MODE>
void launch_mlp(const MlpGeom& g, const uint16_t* w16, const double* rp, double* c, float* F, float* rho,
                float* H1, float* H2, int64_t ld, cudaStream_t s) {
  constexpr size_t smem = mlp_smem<D, MODE>();
  static std::atomic<unsigned long long> attr{0};   // the opt-in above 48 KB, per instantiation and device
  once_per_device(attr, [](int) {
    FSI_CUDA(cudaFuncSetAttribute(k_mlp<D, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  });
  // one wave of the CTAs that fit an SM (228 KB of shared memory, 1 KB reserved
  // per CTA): the weights are loaded once per CTA
  constexpr int per_sm = (int)((228u * 1024u) / (smem + 1024u)) < 1 ? 1 : (int)((228u * 1024u) / (smem + 1024u));
  int64_t b = (g.n_nodes + kNodeThreads - 1) / kNodeThreads;
  if (b > (int64_t)device_sms() * per_sm) b = (int64_t)device_sms() * per_sm;
  launch_k(k_mlp<D, MODE>, (int)(b < 1 ? 1 : b), kNodeThreads, smem, s, g, w16, rp, c, F, rho, H1, H2, ld);
}

// Backward through the MLP for one node: dY from dL/dc, then dH2 and dH1.  Shared
// memory holds the parameters from W2 on (W2, b2, W3, b3), the only ones read.
template <int D>
__global__ void __launch_bounds__(kNodeThreads) k_mlp_bwd(MlpGeom g, const uint16_t* __restrict__ w16,
                                                          const double* __restrict__ gc, const float* __restrict__ rho_s,
                                                          const float* __restrict__ H1, const float* __restrict__ H2,
                                                          float* __restrict__ dY, float* __restrict__ dH1,
                                                          float* __restrict__ dH2, int64_t ld) {
  using N = Net<D>;
  constexpr int kH = N::kHidden, kO = N::kOut, kTail = N::kParams - N::kW2;
  __shared__ __align__(16) float W[(kTail + 3) / 4 * 4];
  for (int i = threadIdx.x; i < kTail; i += blockDim.x) W[i] = bf16_to_f32(w16[N::kW2 + i]);
  __syncthreads();
  const float* W2 = W;
  const float* W3 = W + (N::kW3 - N::kW2);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < g.n_nodes; a += stride) {
    const int4 me = g.node_dof[a];
    const int fl = me.w;
    const double rr = (double)rho_s[a];
    const bool live = rr > 0.0;
    float dy[kO];
#pragma unroll
    for (int o = 0; o < kO; ++o) dy[o] = 0.f;
    if (live) {
      if (!(fl & NF_VFIX)) {
        const double sv = rr * (double)pick5(g.sig_out, cls_of(g, me.x));
#pragma unroll
        for (int k = 0; k < D; ++k) dy[k] = (float)(gc[me.x + k] * sv);
      }
      if (!(fl & NF_UFIX)) {
        const double su = rr * (double)pick5(g.sig_out, cls_of(g, me.y));
#pragma unroll
        for (int k = 0; k < D; ++k) dy[D + k] = (float)(gc[me.y + k] * su);
      }
      if (me.z >= 0 && !(fl & NF_PFIX))
        dy[2 * D] = (float)(gc[me.z] * rr * (double)pick5(g.sig_out, cls_of(g, me.z)));
    }
#pragma unroll
    for (int o = 0; o < kO; ++o) dY[o * ld + a] = dy[o];
    float d2[kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) {
      float s = 0.f;
#pragma unroll
      for (int o = 0; o < kO; ++o) s += W3[j * kO + o] * dy[o];
      d2[j] = s * gelu_grad(H2[j * ld + a]);
      dH2[j * ld + a] = d2[j];
    }
#pragma unroll 1
    for (int i = 0; i < kH; ++i) {
      const float4* w4 = reinterpret_cast<const float4*>(W2 + i * kH);
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < kH / 4; ++q) {
        const float4 w = w4[q];
        s += w.x * d2[4 * q] + w.y * d2[4 * q + 1] + w.z * d2[4 * q + 2] + w.w * d2[4 * q + 3];
      }
      dH1[i * ld + a] = s * gelu_grad(H1[i * ld + a]);
    }
  }
}

// partial[b][(P+bias) x Q] = sum over block b's nodes of [X; 1] Y^T, the ones row
// only when bias is set (X: P <= 64 rows, optionally through gelu; Y: Q <= 64
// rows; column-major with leading dimension ld).  A layer with more than 64
// inputs is taken in chunks of 64 rows, the last one with the bias row.
constexpr int kOuterThreads = 256, kOuterRows = 64;
template <bool GX>
__global__ void __launch_bounds__(kOuterThreads) k_outer(int P, int bias, int Q, const float* __restrict__ X,
                                                         const float* __restrict__ Y, int64_t ld, int64_t n,
                                                         int64_t chunk, float* __restrict__ partial) {
  __shared__ float xs[kOuterRows][33];
  __shared__ float ys[kOuterRows][33];
  const int t = threadIdx.x, tq = t & 15, tp = t >> 4;
  const int R = P + bias;   // rows of the partial; p = tp + 16 kk covers up to 80
  float acc[5][4];
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[k][u] = 0.f;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  for (int64_t base = lo; base < hi; base += 32) {
    const int cnt = (int)(hi - base < 32 ? hi - base : 32);
    __syncthreads();
    for (int e = t; e < P * 32; e += kOuterThreads) {
      const int r = e >> 5, k = e & 31;
      float v = k < cnt ? X[r * ld + base + k] : 0.f;
      if (GX) v = gelu(v);
      xs[r][k] = v;
    }
    for (int e = t; e < Q * 32; e += kOuterThreads) {
      const int r = e >> 5, k = e & 31;
      ys[r][k] = k < cnt ? Y[r * ld + base + k] : 0.f;
    }
    __syncthreads();
    for (int k = 0; k < cnt; ++k) {
      float yv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = tq * 4 + u;
        yv[u] = q < Q ? ys[q][k] : 0.f;
      }
#pragma unroll
      for (int kk = 0; kk < 5; ++kk) {
        const int p = tp + 16 * kk;
        const float xv = p < P ? xs[p][k] : (p < R ? 1.f : 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[kk][u] += xv * yv[u];
      }
    }
  }
  float* out = partial + (size_t)blockIdx.x * R * Q;
#pragma unroll
  for (int kk = 0; kk < 5; ++kk)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int p = tp + 16 * kk, q = tq * 4 + u;
      if (p < R && q < Q) out[p * Q + q] = acc[kk][u];
    }
}

// grad[param(p, q)] += sum_b partial[b][p][q] in block order (FP64 sum); rows
// p < P are the weights at wofs + p Q + q, row P (when bias) the biases at bofs + q
__global__ void k_reduce_grad(const float* __restrict__ partial, int G, int P, int bias, int Q, int wofs, int bofs,
                              float* __restrict__ grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = (P + bias) * Q;
  if (e >= total) return;
  double s = 0.0;
  for (int b = 0; b < G; ++b) s += (double)partial[(size_t)b * total + e];
  const int p = e / Q, q = e % Q;
  const int idx = p < P ? wofs + p * Q + q : bofs + q;
  grad[idx] += (float)s;
}

__global__ void k_adamw(int np, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                        float* __restrict__ grad, uint16_t* __restrict__ w16, float lr, float b1, float b2, float eps,
                        float wd, float bc1, float bc2, float inv_count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = grad[i] * inv_count;
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mhat = mi / bc1, vhat = vi / bc2;
  const float wi = w[i] - lr * (mhat / (sqrtf(vhat) + eps) + wd * w[i]);
  w[i] = wi;
  w16[i] = f32_to_bf16(wi);
  grad[i] = 0.f;
}

// ---------------------------------------------------------------- FGMRES stage
constexpr int kRT = kRedThreads;

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (threadIdx.x < (blockDim.x >> 5)) v = sh[threadIdx.x];
  if (w == 0)
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// rp = V_j - w; part[blk] = sum of rp^2 over the block's contiguous chunk
__global__ void __launch_bounds__(kRT) k_learned_residual(int64_t n, const double* __restrict__ V, int64_t ldv,
                                                          const int* __restrict__ jdev, const double* __restrict__ w,
                                                          double* __restrict__ rp, double* __restrict__ part) {
  dep_wait();
  __shared__ double sh[32];
  const double* v = V + (int64_t)(*jdev) * ldv;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double r = v[i] - w[i];
    rp[i] = r;
    acc += r * r;
  }
  acc = block_sum_d(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// part[blk] = sum of (rp - t)^2; optionally res = rp - t
__global__ void __launch_bounds__(kRT) k_diff_sq(int64_t n, const double* __restrict__ rp,
                                                 const double* __restrict__ t, double* __restrict__ res,
                                                 double* __restrict__ part) {
  dep_wait();
  __shared__ double sh[32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double d = rp[i] - t[i];
    if (res) res[i] = d;
    acc += d * d;
  }
  acc = block_sum_d(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// sums of both partial arrays (fixed order); accept iff ||rp - t||^2 < tau^2 ||rp||^2
__global__ void __launch_bounds__(kRT) k_learned_decide(const double* __restrict__ part, int np, double tau2,
                                                        int* counters) {
  dep_wait();
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    a += part[k];
    b += part[np + k];
  }
  a = block_sum_d(a, sh);
  b = block_sum_d(b, sh);
  if (threadIdx.x == 0) {
    const int acc = (isfinite(a) && isfinite(b) && b < tau2 * a) ? 1 : 0;
    counters[0] = acc;
    counters[1] += acc;
  }
}

__global__ void k_learned_commit(int64_t n, const int* __restrict__ counters, const double* __restrict__ c,
                                 const double* __restrict__ t, double* __restrict__ Z, int64_t ldz,
                                 const int* __restrict__ jdev, double* __restrict__ w) {
  dep_wait();
  if (counters[0] == 0) return;
  double* z = Z + (int64_t)(*jdev) * ldz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    z[i] += c[i];
    w[i] += t[i];
  }
}

__global__ void k_harvest(int64_t n, const double* __restrict__ V, int64_t ldv, const int* __restrict__ jdev,
                          const double* __restrict__ w, double* __restrict__ buf, int nvec) {
  dep_wait();
  const int j = *jdev;
  if (j >= nvec) return;
  const double* v = V + (int64_t)j * ldv;
  double* out = buf + (int64_t)j * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v[i] - w[i];
}

// loss pieces: scal[0] = sum a, scal[1] = sum b, scal[2] = -2 / scal[0]
__global__ void __launch_bounds__(kRT) k_loss_finish(const double* __restrict__ part, int np, double* scal) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    a += part[k];
    b += part[np + k];
  }
  a = block_sum_d(a, sh);
  b = block_sum_d(b, sh);
  if (threadIdx.x == 0) {
    scal[0] = a;
    scal[1] = b;
    scal[2] = a > 0.0 ? -2.0 / a : 0.0;
  }
}

__global__ void k_scale_dev(int64_t n, const double* __restrict__ alpha, double* __restrict__ x) {
  const double a = *alpha;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= a;
}

__global__ void k_square_partial(int64_t n, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sh[32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += x[i] * x[i];
  acc = block_sum_d(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

inline int grid_elem(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > device_sms() * 8) b = device_sms() * 8;
  return (int)(b < 1 ? 1 : b);
}

inline int grid_nodes(int64_t n_nodes) {
  int64_t b = (n_nodes + kNodeThreads - 1) / kNodeThreads;
  if (b > device_sms() * 8) b = device_sms() * 8;
  return (int)(b < 1 ? 1 : b);
}

uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace

// ---------------------------------------------------------------- host API
void learned_set_geometry(Learned& L, int64_t n, int64_t n_nodes, const int32_t* node_dof, const int32_t* patch,
                          cudaStream_t s) {
  require(n_nodes > 0 && node_dof && patch, "learned stage: empty node map");
  require(L.dim == 2 || L.dim == 3, "learned stage: 2D or 3D meshes");
  const int D = L.dim, slots = L.dim == 3 ? Net<3>::kSlots : Net<2>::kSlots;
  std::vector<uint8_t> seen((size_t)n, 0);
  auto mark = [&](int64_t d) {
    require(d >= 0 && d < n, "learned stage: node DOF out of range");
    require(!seen[(size_t)d], "learned stage: DOF owned by two nodes");
    seen[(size_t)d] = 1;
  };
  for (int64_t a = 0; a < n_nodes; ++a) {
    const int32_t* r = node_dof + 4 * a;
    for (int k = 0; k < D; ++k) {
      mark((int64_t)r[0] + k);
      mark((int64_t)r[1] + k);
    }
    if (r[2] >= 0) mark(r[2]);
    else require(r[2] == -1, "learned stage: p DOF must be >= 0 or -1");
    for (int k = 0; k < slots; ++k) {
      const int32_t q = patch[(int64_t)slots * a + k];
      require(q >= -1 && q < n_nodes, "learned stage: patch entry out of range");
    }
  }
  for (int64_t d = 0; d < n; ++d) require(seen[(size_t)d], "learned stage: a DOF belongs to no node");
  L.n_nodes = n_nodes;
  L.node_dof.alloc((size_t)n_nodes);
  L.patch.alloc((size_t)n_nodes * slots);
  FSI_CUDA(cudaMemcpyAsync(L.node_dof.p, node_dof, sizeof(int4) * n_nodes, cudaMemcpyHostToDevice, s));
  FSI_CUDA(cudaMemcpyAsync(L.patch.p, patch, sizeof(int) * slots * n_nodes, cudaMemcpyHostToDevice, s));
  L.rp.alloc((size_t)n);
  L.c.alloc((size_t)n);
  L.t.alloc((size_t)n);
  L.part.alloc(2 * kRedBlocks);
  L.counters.alloc(3);
  FSI_CUDA(cudaMemsetAsync(L.counters.p, 0, 3 * sizeof(int), s));
  FSI_CUDA(cudaStreamSynchronize(s));
}

void learned_set_weights(Learned& L, const float* sig_in, const float* sig_out, const uint16_t* params,
                         cudaStream_t s) {
  for (int k = 0; k < 5; ++k) {
    require(std::isfinite(sig_in[k]) && sig_in[k] > 0.f && std::isfinite(sig_out[k]) && sig_out[k] > 0.f,
            "learned stage: class scales must be finite and positive");
    L.sig_in[k] = sig_in[k];
    L.sig_out[k] = sig_out[k];
  }
  const int np = mlp_params(L.dim);
  for (int i = 0; i < np; ++i)
    require(std::isfinite(bf16_to_f32(params[i])), "learned stage: non-finite weight");
  if (L.w16.n != (size_t)np) L.w16.alloc(np);
  FSI_CUDA(cudaMemcpyAsync(L.w16.p, params, sizeof(uint16_t) * np, cudaMemcpyHostToDevice, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  L.has_weights = true;
}

namespace {
const char kMagic[8] = {'F', 'S', 'I', 'M', 'L', 'P', '0', '1'};
}

void learned_load_file(Learned& L, const char* path, cudaStream_t s) {
  std::ifstream f(path, std::ios::binary);
  require((bool)f, std::string("learned stage: cannot open ") + path);
  char magic[8];
  int32_t shape[4];
  float scales[10];
  f.read(magic, 8);
  f.read(reinterpret_cast<char*>(shape), sizeof(shape));
  f.read(reinterpret_cast<char*>(scales), sizeof(scales));
  require((bool)f && std::memcmp(magic, kMagic, 8) == 0, "learned stage: not a weights file");
  const bool d3 = L.dim == 3;
  require(shape[0] == (d3 ? Net<3>::kIn : Net<2>::kIn) && shape[1] == Net<2>::kHidden &&
              shape[2] == (d3 ? Net<3>::kOut : Net<2>::kOut),
          "learned stage: the file's MLP shape does not fit this mesh's dimension");
  std::vector<uint16_t> params((size_t)mlp_params(L.dim));
  f.read(reinterpret_cast<char*>(params.data()), sizeof(uint16_t) * params.size());
  require((bool)f, "learned stage: truncated weights file");
  learned_set_weights(L, scales, scales + 5, params.data(), s);
}

void learned_save_file(const char* path, int dim, const float* sig_in, const float* sig_out,
                       const uint16_t* params) {
  std::ofstream f(path, std::ios::binary | std::ios::trunc);
  require((bool)f, std::string("learned stage: cannot write ") + path);
  const bool d3 = dim == 3;
  const int32_t shape[4] = {d3 ? Net<3>::kIn : Net<2>::kIn, Net<2>::kHidden, d3 ? Net<3>::kOut : Net<2>::kOut, 0};
  f.write(kMagic, 8);
  f.write(reinterpret_cast<const char*>(shape), sizeof(shape));
  f.write(reinterpret_cast<const char*>(sig_in), 5 * sizeof(float));
  f.write(reinterpret_cast<const char*>(sig_out), 5 * sizeof(float));
  f.write(reinterpret_cast<const char*>(params), sizeof(uint16_t) * mlp_params(dim));
  require((bool)f, std::string("learned stage: write failed for ") + path);
}

MlpGeom learned_geom(const Learned& L, const int64_t off[6]) {
  MlpGeom g;
  g.dim = L.dim;
  g.n_nodes = L.n_nodes;
  g.node_dof = L.node_dof.p;
  g.patch = L.patch.p;
  g.off1 = off[1]; g.off2 = off[2]; g.off3 = off[3]; g.off4 = off[4];
  for (int k = 0; k < 5; ++k) {
    g.sig_in[k] = L.sig_in[k];
    g.inv_in[k] = 1.0f / L.sig_in[k];
    g.sig_out[k] = L.sig_out[k];
  }
  g.err = L.counters.p ? L.counters.p + 2 : nullptr;
  return g;
}


void mlp_apply(const MlpGeom& g, const uint16_t* w16, const double* rp, double* c, cudaStream_t s) {
  if (g.dim == 3) {
    launch_mlp<3, MODE_APPLY>(g, w16, rp, c, nullptr, nullptr, nullptr, nullptr, 0, s);
    return;
  }
  if (mlp_tensor_cores() && g.err) {
    mlp_apply_tc(g, w16, rp, c, g.err, s);
    return;
  }
  launch_mlp<2, MODE_APPLY>(g, w16, rp, c, nullptr, nullptr, nullptr, nullptr, 0, s);
}

void mlp_features(const MlpGeom& g, const double* rp, float* F, float* rho, cudaStream_t s) {
  if (g.dim == 3) launch_mlp<3, MODE_FEATURES>(g, nullptr, rp, nullptr, F, rho, nullptr, nullptr, 0, s);
  else launch_mlp<2, MODE_FEATURES>(g, nullptr, rp, nullptr, F, rho, nullptr, nullptr, 0, s);
}

void learned_residual(int64_t n, const double* V, int64_t ldv, const int* jdev, const double* w, double* rp,
                      double* part, cudaStream_t s) {
  launch_k(k_learned_residual, kRedBlocks, kRT, 0, s, n, V, ldv, jdev, w, rp, part);
}

void learned_decide(int64_t n, const double* rp, const double* t, double tau, double* part, int* counters,
                    cudaStream_t s) {
  launch_k(k_diff_sq, kRedBlocks, kRT, 0, s, n, rp, t, (double*)nullptr, part + kRedBlocks);
  launch_k(k_learned_decide, 1, kRT, 0, s, part, kRedBlocks, tau * tau, counters);
}

void learned_commit(int64_t n, const int* counters, const double* c, const double* t, double* Z, int64_t ldz,
                    const int* jdev, double* w, cudaStream_t s) {
  launch_k(k_learned_commit, grid_elem(n), 256, 0, s, n, counters, c, t, Z, ldz, jdev, w);
}

void harvest_residual(int64_t n, const double* V, int64_t ldv, const int* jdev, const double* w, double* buf,
                      int nvec, cudaStream_t s) {
  launch_k(k_harvest, grid_elem(n), 256, 0, s, n, V, ldv, jdev, w, buf, nvec);
}

// ---------------------------------------------------------------- training
Trainer::~Trainer() {
  if (pinned) cudaFreeHost(pinned);
}

void trainer_init(Trainer& T, const TrainParams& p) {
  for (int k = 0; k < 5; ++k)
    require(std::isfinite(p.sig_in[k]) && p.sig_in[k] > 0.f && std::isfinite(p.sig_out[k]) && p.sig_out[k] > 0.f,
            "trainer: class scales must be finite and positive");
  require(p.dim == 2 || p.dim == 3, "trainer: dim must be 2 or 3");
  require(p.lr > 0 && p.beta1 >= 0 && p.beta1 < 1 && p.beta2 >= 0 && p.beta2 < 1 && p.eps > 0 && p.weight_decay >= 0,
          "trainer: bad AdamW parameters");
  T.prm = p;
  // Glorot-uniform weights from a SplitMix64 stream (one draw per parameter
  // index), biases zero, last layer scaled by init_out_scale
  const int np = mlp_params(p.dim);
  std::vector<float> w((size_t)np, 0.f);
  auto fill = [&](int ofs, int fan_in, int fan_out, double scale) {
    const double lim = std::sqrt(6.0 / (fan_in + fan_out)) * scale;
    for (int i = 0; i < fan_in * fan_out; ++i) {
      const uint64_t r = splitmix64((p.seed << 32) + (uint64_t)(ofs + i));
      const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
      w[ofs + i] = (float)((2.0 * u - 1.0) * lim);
    }
  };
  if (p.dim == 3) {
    using N = Net<3>;
    fill(N::kW1, N::kIn, N::kHidden, 1.0);
    fill(N::kW2, N::kHidden, N::kHidden, 1.0);
    fill(N::kW3, N::kHidden, N::kOut, p.init_out_scale);
  } else {
    using N = Net<2>;
    fill(N::kW1, N::kIn, N::kHidden, 1.0);
    fill(N::kW2, N::kHidden, N::kHidden, 1.0);
    fill(N::kW3, N::kHidden, N::kOut, p.init_out_scale);
  }
  T.master.alloc(np);
  T.m.alloc(np);
  T.v.alloc(np);
  T.grad.alloc(np);
  T.w16.alloc(np);
  T.scal.alloc(4);
  T.part.alloc(2 * kRedBlocks);
  if (!T.pinned) FSI_CUDA(cudaMallocHost(&T.pinned, 4 * sizeof(double)));
  trainer_set_master(T, w.data());
}

void trainer_set_master(Trainer& T, const float* w) {
  const int np = T.n_params();
  std::vector<uint16_t> h((size_t)np);
  for (int i = 0; i < np; ++i) {
    require(std::isfinite(w[i]), "trainer: non-finite weight");
    h[i] = f32_to_bf16(w[i]);
  }
  FSI_CUDA(cudaMemcpy(T.master.p, w, sizeof(float) * np, cudaMemcpyHostToDevice));
  FSI_CUDA(cudaMemcpy(T.w16.p, h.data(), sizeof(uint16_t) * np, cudaMemcpyHostToDevice));
  FSI_CUDA(cudaMemset(T.m.p, 0, sizeof(float) * np));
  FSI_CUDA(cudaMemset(T.v.p, 0, sizeof(float) * np));
  FSI_CUDA(cudaMemset(T.grad.p, 0, sizeof(float) * np));
  T.grads = 0;
  T.steps = 0;
}

void apply_operator_t(Context& C, const double* x, double* y) {
  if (!C.At_built) {
    bsr_transpose(C.AVV, C.AVVt, C.s);
    bsr_transpose(C.AVP, C.AVPt, C.s);
    bsr_transpose(C.APV, C.APVt, C.s);
    bsr_transpose(C.APP, C.APPt, C.s);
    FSI_CUDA(cudaStreamSynchronize(C.s));
    C.At_built = true;
  }
  const int64_t nv = C.off[4];
  // A^T = [[AVV^T, APV^T], [AVP^T, APP^T]]
  spmv2_axpby<double>(C.AVVt, x, &C.APVt, x + nv, 1.0, 0.0, y, C.s);
  spmv2_axpby<double>(C.AVPt, x, &C.APPt, x + nv, 1.0, 0.0, y + nv, C.s);
}

namespace {
template <int D>
double trainer_step_d(Trainer& T, Context& C, const double* rp, bool grad) {
  using N = Net<D>;
  Learned& L = C.learned;
  const int64_t n = C.n, nn = L.n_nodes;
  cudaStream_t s = C.s;
  if (T.cap_nodes < nn) {
    T.cap_nodes = nn;
    T.F.alloc((size_t)N::kIn * nn);
    T.rho.alloc((size_t)nn);
    T.H1.alloc((size_t)N::kHidden * nn);
    T.H2.alloc((size_t)N::kHidden * nn);
    T.dY.alloc((size_t)N::kOut * nn);
    T.dH1.alloc((size_t)N::kHidden * nn);
    T.dH2.alloc((size_t)N::kHidden * nn);
  }
  if (T.cap_n < n) {
    T.cap_n = n;
    T.c.alloc((size_t)n);
    T.t.alloc((size_t)n);
    T.res.alloc((size_t)n);
    T.g.alloc((size_t)n);
  }
  MlpGeom g = learned_geom(L, C.off);
  for (int k = 0; k < 5; ++k) {
    g.sig_in[k] = T.prm.sig_in[k];
    g.inv_in[k] = 1.0f / T.prm.sig_in[k];
    g.sig_out[k] = T.prm.sig_out[k];
  }
  const int64_t ld = T.cap_nodes;
  launch_mlp<D, MODE_TRAIN>(g, T.w16.p, rp, T.c.p, T.F.p, T.rho.p, T.H1.p, T.H2.p, ld, s);
  apply_operator(C, T.c.p, T.t.p);
  k_square_partial<<<kRedBlocks, kRT, 0, s>>>(n, rp, T.part.p);
  FSI_CHECK_LAUNCH();
  k_diff_sq<<<kRedBlocks, kRT, 0, s>>>(n, rp, T.t.p, T.res.p, T.part.p + kRedBlocks);
  FSI_CHECK_LAUNCH();
  k_loss_finish<<<1, kRT, 0, s>>>(T.part.p, kRedBlocks, T.scal.p);
  FSI_CHECK_LAUNCH();
  if (!grad) {
    FSI_CUDA(cudaMemcpyAsync(T.pinned, T.scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    return T.pinned[0] > 0.0 ? T.pinned[1] / T.pinned[0] : 0.0;
  }
  k_scale_dev<<<grid_elem(n), 256, 0, s>>>(n, T.scal.p + 2, T.res.p);   // res = -2 (r' - A c) / ||r'||^2
  FSI_CHECK_LAUNCH();
  apply_operator_t(C, T.res.p, T.g.p);                                     // dL/dc
  k_mlp_bwd<D><<<grid_nodes(nn), kNodeThreads, 0, s>>>(g, T.w16.p, T.g.p, T.rho.p, T.H1.p, T.H2.p, T.dY.p, T.dH1.p,
                                                    T.dH2.p, ld);
  FSI_CHECK_LAUNCH();
  // weight gradients: dW1 = [F;1] dH1^T, dW2 = [gelu(H1);1] dH2^T, dW3 = [gelu(H2);1] dY^T
  const int G = (int)std::min<int64_t>(2 * device_sms(), std::max<int64_t>(1, (nn + 255) / 256));
  const int64_t chunk = ((nn + G - 1) / G + 31) / 32 * 32;
  const size_t need = (size_t)G * (kOuterRows + 1) * N::kHidden;
  if (T.partial.n < need) T.partial.alloc(need);
  // layer 1 in chunks of kOuterRows inputs, the bias row with the last chunk
  struct Lyr { int P, Q; const float* X; const float* Y; bool gx; int wofs, bofs; };
  const Lyr lyr[3] = {{N::kIn, N::kHidden, T.F.p, T.dH1.p, false, N::kW1, N::kB1},
                      {N::kHidden, N::kHidden, T.H1.p, T.dH2.p, true, N::kW2, N::kB2},
                      {N::kHidden, N::kOut, T.H2.p, T.dY.p, true, N::kW3, N::kB3}};
  for (const Lyr& l : lyr) {
    for (int p0 = 0; p0 < l.P; p0 += kOuterRows) {
      const int P = std::min(kOuterRows, l.P - p0), bias = p0 + P == l.P ? 1 : 0;
      const float* X = l.X + (int64_t)p0 * ld;
      if (l.gx) k_outer<true><<<G, kOuterThreads, 0, s>>>(P, bias, l.Q, X, l.Y, ld, nn, chunk, T.partial.p);
      else k_outer<false><<<G, kOuterThreads, 0, s>>>(P, bias, l.Q, X, l.Y, ld, nn, chunk, T.partial.p);
      FSI_CHECK_LAUNCH();
      const int total = (P + bias) * l.Q;
      k_reduce_grad<<<div_up(total, 256), 256, 0, s>>>(T.partial.p, G, P, bias, l.Q, l.wofs + p0 * l.Q, l.bofs,
                                                       T.grad.p);
      FSI_CHECK_LAUNCH();
    }
  }
  ++T.grads;
  FSI_CUDA(cudaMemcpyAsync(T.pinned, T.scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  return T.pinned[0] > 0.0 ? T.pinned[1] / T.pinned[0] : 0.0;
}
}  // namespace

double trainer_step(Trainer& T, Context& C, const double* rp, bool grad) {
  require(C.learned.n_nodes > 0, "trainer: fsi_learned_setup has not been called on this context");
  require(C.learned.dim == T.prm.dim, "trainer: the context's mesh dimension differs from the trainer's");
  return T.prm.dim == 3 ? trainer_step_d<3>(T, C, rp, grad) : trainer_step_d<2>(T, C, rp, grad);
}

void trainer_update(Trainer& T, cudaStream_t s, double lr) {
  require(T.grads > 0, "trainer: no gradient accumulated since the last update");
  require(std::isfinite(lr), "trainer: learning rate must be finite");
  if (lr <= 0.0) lr = T.prm.lr;
  ++T.steps;
  const double bc1 = 1.0 - std::pow(T.prm.beta1, (double)T.steps);
  const double bc2 = 1.0 - std::pow(T.prm.beta2, (double)T.steps);
  const int np = T.n_params();
  k_adamw<<<div_up(np, 256), 256, 0, s>>>(np, T.master.p, T.m.p, T.v.p, T.grad.p, T.w16.p,
                                                  (float)lr, (float)T.prm.beta1, (float)T.prm.beta2,
                                                  (float)T.prm.eps, (float)T.prm.weight_decay, (float)bc1, (float)bc2,
                                                  1.0f / (float)T.grads);
  FSI_CHECK_LAUNCH();
  T.grads = 0;
  FSI_CUDA(cudaStreamSynchronize(s));
}

}  // namespace fsi

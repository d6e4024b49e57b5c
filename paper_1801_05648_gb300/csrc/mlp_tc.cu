// Learned-stage MLP inference on the 5th-generation tensor cores (tcgen05).
//
// The same map as k_mlp<MODE_APPLY> (learned.cuh): per Q2 node a, the 45 patch
// residuals scaled by the class scales and the patch RMS rho, then
//   h1 = W1^T f + b1, h2 = W2^T gelu(h1) + b2, y = W3^T gelu(h2) + b3,
//   c[dof_k(a)] = y_k rho sigma_out[class].
// A CTA takes 128 nodes at a time, two threads per node; node row r of the tile is
// accumulator row r, read by the warps that own its 32-lane quarter of tensor memory.
// Each layer is a chain of tcgen05.mma.kind::tf32 (M = 128, N = 64 / 64 / 16,
// K = 8 per instruction) from shared memory into tensor memory:
//   layer 1  K = 56: the 53 inputs (45 patch values, the one-hot lattice parity,
//            the four node flags), a constant 1 whose weight row is b1, two zeros
//   layer 2  K = 64
//   layer 3  K = 64, N = 16 (5 outputs, zero-padded columns)
// Operand precision.  The weights are bfloat16, exact in TF32.  Each activation
// x is split into x_hi = x with its low 13 mantissa bits cleared (exact in TF32)
// and x_lo = x - x_hi, and every layer runs the MMA chain on both (D = A_hi W +
// A_lo W): the products keep ~22 significant bits, as FP32 FMAs would, and the
// tensor core accumulates in FP32.
// Operand layout: the canonical K-major layout without swizzling: 8-row x 16-byte
// core matrices, consecutive along K 128 bytes apart (leading-byte offset) and
// along the rows 2048 bytes apart (stride-byte offset, the 64-column capacity of
// every operand tile).
// Every wait on the MMA-completion barrier is bounded (about a second of clock);
// a timeout sets *err, the CTA waits once more (bounded) for its MMAs and frees
// its tensor memory before it returns.
#include "learned.cuh"

#include <cstring>

namespace fsi {

namespace {

constexpr int kTcRows = 128;           // nodes per tile = MMA M
constexpr int kTcThreads = 256;        // two threads per node (see k_mlp_tc)
constexpr int kTcK1 = 56;              // layer-1 K: 53 inputs, the bias column, zero padding
constexpr int kTcN3 = 16;              // layer-3 N (5 outputs, zero-padded)
constexpr uint32_t kLbo = 128;         // bytes between core matrices along K
constexpr uint32_t kSbo = 2048;        // bytes between 8-row groups (64 fp32 columns of capacity)
constexpr uint32_t kTmemCols = 128;    // D1 / D3 in columns [0, 64), D2 in [64, 128)

// dynamic shared memory map (bytes)
constexpr uint32_t kOffAhi = 0, kOffAlo = 32768, kOffB1 = 65536, kOffB2 = 81920, kOffB3 = 98304;
constexpr uint32_t kOffB2v = 102400;                     // b2 (64)
constexpr uint32_t kOffB3v = kOffB2v + 64 * 4;           // b3 (16, padded)
constexpr uint32_t kOffBar = kOffB3v + 16 * 4;           // mbarrier (8 bytes)
constexpr uint32_t kOffTmem = kOffBar + 8;               // tensor-memory base written by tcgen05.alloc
constexpr uint32_t kOffSs = kOffTmem + 8;                // partial sums of squares, 2 x 128 floats
constexpr uint32_t kTcSmem = kOffSs + 2 * 128 * 4;

__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)(r >> 3) * kSbo + (uint32_t)(k >> 2) * kLbo + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLbo >> 4) << 16) | ((uint64_t)(kSbo >> 4) << 32) |
         (1ull << 46);   // descriptor version 1; base offset 0; no swizzling
}

// instruction descriptor: D FP32, A and B TF32, both K-major, M = 128
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's row
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Bounded wait for the completion of phase `parity` of the barrier: false after
// about 2e9 clocks without it.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 2000000000ll) return false;
  }
}

__device__ __forceinline__ float tc_gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float bf16f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

__device__ __forceinline__ int cls_in(const MlpGeom& g, int64_t d) {
  return (d >= g.off1) + (d >= g.off2) + (d >= g.off3) + (d >= g.off4);
}
__device__ __forceinline__ float pick(const float (&a)[5], int k) {
  return k == 0 ? a[0] : k == 1 ? a[1] : k == 2 ? a[2] : k == 3 ? a[3] : a[4];
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// columns col..col+3 (col a multiple of 4) of row `row` -> (hi, lo) in the two A
// tiles; one 16-byte store each, so the 8 rows of a quarter warp fill 128
// consecutive bytes (no bank conflicts)
__device__ __forceinline__ void put4(unsigned char* sm, int row, int col, float a, float b, float c, float d) {
  const float4 hi = make_float4(tf32_hi(a), tf32_hi(b), tf32_hi(c), tf32_hi(d));
  *reinterpret_cast<float4*>(sm + kOffAhi + core_off(row, col)) = hi;
  *reinterpret_cast<float4*>(sm + kOffAlo + core_off(row, col)) = make_float4(a - hi.x, b - hi.y, c - hi.z, d - hi.w);
}

// one layer's MMA chain on (A_hi, A_lo) x B into the accumulator at dcol; issued by one thread
// (commit = false only under fault injection: the wait on the barrier then runs out)
__device__ __forceinline__ void issue_layer(uint32_t sbase, uint32_t boff, uint32_t tmem, uint32_t dcol, int ksteps,
                                            int n, uint32_t bar, bool commit = true) {
  const uint32_t id = idesc_tf32(n);
  for (int s = 0; s < ksteps; ++s)
    tc_mma(tmem + dcol, smem_desc(sbase + kOffAhi + 2u * kLbo * s), smem_desc(sbase + boff + 2u * kLbo * s), id,
           s > 0);
  for (int s = 0; s < ksteps; ++s)
    tc_mma(tmem + dcol, smem_desc(sbase + kOffAlo + 2u * kLbo * s), smem_desc(sbase + boff + 2u * kLbo * s), id, 1);
  if (commit) tc_commit(bar);
}

// 256 threads: thread t works on node row t & 127 of the tile; the two halves (t < 128
// and t >= 128) split every per-node step.  Warp w reads tensor-memory lane quarter
// w & 3 (warps w and w + 4 share it and take different columns).
//   gather     half 0: patch slots 0-3 (columns 0-19); half 1: slots 4-8 (20-44), the
//              one-hot, the flags and the bias column; rho from both halves' partial sums
//   layers 1-2 half 0: hidden columns 0-31; half 1: 32-63
//   layer 3    half 0: the outputs and the scatter
__global__ void __launch_bounds__(kTcThreads, 2) k_mlp_tc(MlpGeom g, const uint16_t* __restrict__ w16,
                                                          const double* __restrict__ rp, double* __restrict__ c,
                                                          int* __restrict__ err, int no_commit) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int t = threadIdx.x, warp = t >> 5;
  const int row = t & (kTcRows - 1), half = t >> 7;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
  const uint32_t bar = sbase + kOffBar;
  float* ssbuf = reinterpret_cast<float*>(sm + kOffSs);   // [2][128] partial sums of squares
  // ---- weights (independent of earlier kernels): B operands N x K, K-major, zero-padded;
  // row 53 of the layer-1 operand is b1 (its input column is the constant 1)
  for (int i = t; i < 64 * 64; i += blockDim.x) {
    const int n = i >> 6, k = i & 63;
    float w1 = 0.f;
    if (k < kMlpIn) w1 = bf16f(w16[kW1 + k * kMlpHidden + n]);
    else if (k == kMlpIn) w1 = bf16f(w16[kB1 + n]);
    *reinterpret_cast<float*>(sm + kOffB1 + core_off(n, k)) = w1;
    *reinterpret_cast<float*>(sm + kOffB2 + core_off(n, k)) = bf16f(w16[kW2 + k * kMlpHidden + n]);
    if (n < kTcN3)
      *reinterpret_cast<float*>(sm + kOffB3 + core_off(n, k)) = n < kMlpOut ? bf16f(w16[kW3 + k * kMlpOut + n]) : 0.f;
  }
  for (int i = t; i < 64; i += blockDim.x) reinterpret_cast<float*>(sm + kOffB2v)[i] = bf16f(w16[kB2 + i]);
  if (t < 16) reinterpret_cast<float*>(sm + kOffB3v)[t] = t < kMlpOut ? bf16f(w16[kB3 + t]) : 0.f;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + kOffTmem),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + kOffTmem);
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's lane quarter
  const uint32_t hcol = 32u * (uint32_t)half;                         // this half's hidden columns
  const float* b2 = reinterpret_cast<const float*>(sm + kOffB2v);
  const float* b3 = reinterpret_cast<const float*>(sm + kOffB3v);
  dep_wait();
  uint32_t phase = 0;
  bool failed = false;
  const int64_t ntiles = (g.n_nodes + kTcRows - 1) / kTcRows;
  // patch slots of this half, and where their values go in the layer-1 operand
  const int s0 = half ? 4 : 0, ns = half ? kMlpSlots - 4 : 4;
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t a = tile * kTcRows + row;
    const bool valid = a < g.n_nodes;
    // ---- gather this half's slots (as k_mlp), partial sum of squares
    int4 me = make_int4(0, 0, -1, 0);
    float x[25];
    float ss = 0.f;
    if (valid) me = g.node_dof[a];
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const int q = (valid && s < ns) ? g.patch[a * kMlpSlots + s0 + s] : -1;
      float e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f, e4 = 0.f;
      if (q >= 0) {
        const int4 r = g.node_dof[q];
        const float iv = pick(g.inv_in, cls_in(g, r.x));
        const float iu = pick(g.inv_in, cls_in(g, r.y));
        e0 = (float)rp[r.x] * iv;
        e1 = (float)rp[r.x + 1] * iv;
        e2 = (float)rp[r.y] * iu;
        e3 = (float)rp[r.y + 1] * iu;
        if (r.z >= 0) e4 = (float)rp[r.z] * pick(g.inv_in, cls_in(g, r.z));
      }
      x[5 * s + 0] = e0; x[5 * s + 1] = e1; x[5 * s + 2] = e2; x[5 * s + 3] = e3; x[5 * s + 4] = e4;
      ss += e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3 + e4 * e4;
    }
    ssbuf[half * kTcRows + row] = ss;
    __syncthreads();
    const float rho = sqrtf((ssbuf[row] + ssbuf[kTcRows + row]) * (1.0f / kMlpPatch));
    const bool live = rho > 0.f;
    const float inv_rho = live ? 1.0f / rho : 0.f;
    const int fl = me.w;
    if (half == 0) {
#pragma unroll
      for (int k = 0; k < 20; k += 4)
        put4(sm, row, k, x[k] * inv_rho, x[k + 1] * inv_rho, x[k + 2] * inv_rho, x[k + 3] * inv_rho);
    } else {
      // columns 20..44, then 45..55: one-hot parity, flags (bits 0..3), the bias input 1,
      // zeros (all exact in TF32, so their low terms are 0); the hidden layers overwrite them
#pragma unroll
      for (int k = 0; k < 24; k += 4)
        put4(sm, row, 20 + k, x[k] * inv_rho, x[k + 1] * inv_rho, x[k + 2] * inv_rho, x[k + 3] * inv_rho);
      const int par = ((fl >> 4) & 1) | (((fl >> 5) & 1) << 1);
      const float oh[4] = {par == 0 ? 1.f : 0.f, par == 1 ? 1.f : 0.f, par == 2 ? 1.f : 0.f, par == 3 ? 1.f : 0.f};
      const float fb[4] = {(float)(fl & 1), (float)((fl >> 1) & 1), (float)((fl >> 2) & 1), (float)((fl >> 3) & 1)};
      put4(sm, row, 44, x[24] * inv_rho, oh[0], oh[1], oh[2]);
      put4(sm, row, 48, oh[3], fb[0], fb[1], fb[2]);
      put4(sm, row, 52, fb[3], 1.f, 0.f, 0.f);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (t == 0) issue_layer(sbase, kOffB1, tmem, 0, kTcK1 / 8, kMlpHidden, bar, !no_commit);
    // ---- layer 1 epilogue: gelu -> layer-2 operand (this half's 32 columns)
    bool ok = bar_wait(bar, phase);
    if (__syncthreads_or(!ok)) { failed = true; break; }
    phase ^= 1u;
    tc_fence_after();
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
      float h[16];
      tc_ld16(trow + hcol + 16u * q, h);
      tc_wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) h[i] = tc_gelu(h[i]);
#pragma unroll
      for (int i = 0; i < 16; i += 4) put4(sm, row, hcol + 16 * q + i, h[i], h[i + 1], h[i + 2], h[i + 3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (t == 0) issue_layer(sbase, kOffB2, tmem, 64, kMlpHidden / 8, kMlpHidden, bar);
    // ---- layer 2 epilogue
    ok = bar_wait(bar, phase);
    if (__syncthreads_or(!ok)) { failed = true; break; }
    phase ^= 1u;
    tc_fence_after();
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
      float h[16];
      tc_ld16(trow + 64u + hcol + 16u * q, h);
      tc_wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) h[i] = tc_gelu(h[i] + b2[hcol + 16 * q + i]);
#pragma unroll
      for (int i = 0; i < 16; i += 4) put4(sm, row, hcol + 16 * q + i, h[i], h[i + 1], h[i + 2], h[i + 3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (t == 0) issue_layer(sbase, kOffB3, tmem, 0, kMlpHidden / 8, kTcN3, bar);
    // ---- layer 3 epilogue: outputs, scatter (half 0)
    ok = bar_wait(bar, phase);
    if (__syncthreads_or(!ok)) { failed = true; break; }
    phase ^= 1u;
    tc_fence_after();
    if (half == 0) {
      float y[16];
      tc_ld16(trow, y);
      tc_wait_ld();
      if (valid) {
        const double rr = (double)rho;
        const double sv = live && !(fl & NF_VFIX) ? rr * (double)pick(g.sig_out, cls_in(g, me.x)) : 0.0;
        const double su = live && !(fl & NF_UFIX) ? rr * (double)pick(g.sig_out, cls_in(g, me.y)) : 0.0;
        c[me.x] = sv != 0.0 ? (double)(y[0] + b3[0]) * sv : 0.0;
        c[me.x + 1] = sv != 0.0 ? (double)(y[1] + b3[1]) * sv : 0.0;
        c[me.y] = su != 0.0 ? (double)(y[2] + b3[2]) * su : 0.0;
        c[me.y + 1] = su != 0.0 ? (double)(y[3] + b3[3]) * su : 0.0;
        if (me.z >= 0) {
          const double sp = live && !(fl & NF_PFIX) ? rr * (double)pick(g.sig_out, cls_in(g, me.z)) : 0.0;
          c[me.z] = sp != 0.0 ? (double)(y[4] + b3[4]) * sp : 0.0;
        }
      }
    }
    tc_fence_before();
    __syncthreads();     // every row read before the next tile's layer 1 overwrites the accumulators
    tc_fence_after();
  }
  if (failed) {   // `phase` is the phase whose wait gave up
    if (t == 0) atomicExch(err, 1);
    bar_wait(bar, phase);   // the MMAs of the unfinished layer (bounded)
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

void mlp_apply_tc(const MlpGeom& g, const uint16_t* w16, const double* rp, double* c, int* err, cudaStream_t s) {
  require(g.dim == 2, "the tensor-core MLP takes the 2D layout (3x3 patch, 53 inputs)");
  static std::atomic<unsigned long long> attr{0};   // the opt-in above 48 KB, per device
  once_per_device(attr, [](int) {
    FSI_CUDA(cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  });
  if (g.n_nodes <= 0) return;
  const int64_t tiles = (g.n_nodes + kTcRows - 1) / kTcRows;
  int64_t grid = (int64_t)device_sms() * 2;   // two 103-KB CTAs per SM
  if (grid > tiles) grid = tiles;
  launch_k(k_mlp_tc, (int)grid, kTcThreads, kTcSmem, s, g, w16, rp, c, err,
           (fault_inject() & kInjectMlpCommit) ? 1 : 0);
}

}  // namespace fsi

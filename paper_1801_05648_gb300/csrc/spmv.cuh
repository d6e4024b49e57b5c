// Block-sparse (BSR) matrix-vector products with fused epilogues.
//
// A group of `tpr` lanes (1..32, a power of two inside one warp) owns one block
// row: lane l reads blocks l, l+tpr, ... of the row, so the lanes of a group
// stream consecutive blocks (row-major br x bc values, 16-byte vector loads
// whenever the block size allows) and the block-column indices coalesced; the
// x entries are gathered through the read-only path.  Each lane issues several
// blocks' loads before multiplying (bytes in flight hide the DRAM latency).
// Lane 0 loads its row's own epilogue operands first, then the group reduces its
// br partial sums with shuffles and lane 0 applies the epilogue.  The lane count
// is chosen per matrix and precision (see lanes_for in common.cuh).  An optional
// second matrix with the same block rows (e.g. the d x 1 pressure columns next
// to the d x d vector columns of the monolithic operator) is accumulated into
// the same sums, so one pass covers every column class of a row.
#pragma once
#include "common.cuh"

namespace fsi {

// Products and fused multiply-adds with their rounding fixed.  Where a formula has
// two products feeding one sum, the compiler may fuse either of them into an FMA,
// and may choose differently in two kernels that inline the same code; the row
// sums and epilogues below spell out which operations round, so the results do
// not depend on those choices (another kernel computing the same rows in the same
// order, e.g. a variant staged through shared memory, is bit-identical).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class T, int N>
__device__ __forceinline__ void load_stream(const T* __restrict__ p, T* out) {
  if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      double2 v = __ldcs(reinterpret_cast<const double2*>(p) + i);
      out[2 * i] = v.x; out[2 * i + 1] = v.y;
    }
  } else if constexpr (sizeof(T) == 4 && N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      float4 v = __ldcs(reinterpret_cast<const float4*>(p) + i);
      out[4 * i] = v.x; out[4 * i + 1] = v.y; out[4 * i + 2] = v.z; out[4 * i + 3] = v.w;
    }
  } else if constexpr (sizeof(T) == 4 && N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      float2 v = __ldcs(reinterpret_cast<const float2*>(p) + i);
      out[2 * i] = v.x; out[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = __ldcs(p + i);
  }
}

template <class T, int N>
__device__ __forceinline__ void load_gather(const T* __restrict__ p, T* out) {
  if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      double2 v = __ldg(reinterpret_cast<const double2*>(p) + i);
      out[2 * i] = v.x; out[2 * i + 1] = v.y;
    }
  } else if constexpr (sizeof(T) == 4 && N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      float2 v = __ldg(reinterpret_cast<const float2*>(p) + i);
      out[2 * i] = v.x; out[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = __ldg(p + i);
  }
}

// FP64 gathers with the L2 evict-last policy: the gathered vector (71 MB in FP64 on
// the 1024x512 system) then outlives the evict-first matrix stream in L2.  FP64
// launches use them unless the caller turns them off (OuterOperatorScope).
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
template <int N>
__device__ __forceinline__ void load_gather_keep(const double* __restrict__ p, double* out) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 900)
  const uint64_t pol = l2_evict_last_policy();
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i)
      asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
          : "=d"(out[2 * i]), "=d"(out[2 * i + 1])
          : "l"(p + 2 * i), "l"(pol));
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(out[i]) : "l"(p + i), "l"(pol));
  }
#else
  for (int i = 0; i < N; ++i) out[i] = p[i];
#endif
}

// FP32 copies of 3 x 3-block matrices are stored planar (bsr_make_fp32): values
// 0-3 of every block, then values 4-7 of every block, then value 8 of every block,
// so that the lanes of a row group, which read consecutive blocks, issue two
// contiguous 16-byte loads and one contiguous 4-byte load per block.  (A 36-byte
// block read row-major takes nine 4-byte loads whose lanes are 36 bytes apart:
// each touches about nine cache lines, and the L1 tag stage, not DRAM, becomes the
// limit.)  Every other block shape and every FP64 copy is stored row-major.
template <class T, int BR, int BC>
__host__ __device__ constexpr bool planar_blocks() {
  return sizeof(T) == 4 && planar_fp32_shape(BR, BC);
}

// Block k of a matrix with nnzb blocks (row-major block values in `out`), loaded
// with the evict-first policy of the matrix streams.
template <class T, int BR, int BC>
__device__ __forceinline__ void load_block(const T* __restrict__ v, int64_t nnzb, int64_t k, T* out) {
  if constexpr (planar_blocks<T, BR, BC>()) {
    const float4 p = __ldcs(reinterpret_cast<const float4*>(v) + k);
    const float4 q = __ldcs(reinterpret_cast<const float4*>(v + 4 * nnzb) + k);
    out[0] = p.x; out[1] = p.y; out[2] = p.z; out[3] = p.w;
    out[4] = q.x; out[5] = q.y; out[6] = q.z; out[7] = q.w;
    out[8] = __ldcs(v + 8 * nnzb + k);
  } else {
    load_stream<T, BR * BC>(v + k * (BR * BC), out);
  }
}

// ------------------------------------------------------------------ gathers
// x[c] segment of the vector the matrix multiplies.
// KEEP (FP64 only): gather with the L2 evict-last policy.  A template parameter, so
// that kernels without it carry no code (and no registers) for it.
template <class T, int BC, bool KEEP = false>
struct GatherX {
  static constexpr bool kKeep = KEEP;
  const T* x;
  __device__ __forceinline__ void operator()(int c, T* out) const {
    if constexpr (sizeof(T) == 8 && KEEP) load_gather_keep<BC>(x + (size_t)c * BC, out);
    else load_gather<T, BC>(x + (size_t)c * BC, out);
  }
};
// (dinv * b * s)[c] segment: the first Chebyshev iterate from x = 0, formed on the fly.
template <class T, int BC>
struct GatherScaled {
  static constexpr bool kKeep = false;
  const T* b; const T* dinv; T s;
  __device__ __forceinline__ void operator()(int c, T* out) const {
    T bv[BC], dv[BC];
    load_gather<T, BC>(b + (size_t)c * BC, bv);
    load_gather<T, BC>(dinv + (size_t)c * BC, dv);
#pragma unroll
    for (int j = 0; j < BC; ++j) out[j] = mul_rn(mul_rn(dv[j], bv[j]), s);
  }
};

// ------------------------------------------------------------------ epilogues
// Each epilogue loads its row's own operands (load) before the row product is
// accumulated, so those loads overlap the gathers, and combines them (store).

// y = alpha * (A x) + beta * y   (y not read when beta == 0)
template <class T, int BR>
struct EpiAxpby {
  T* y; T alpha; T beta;
  struct Pre { T y[BR]; };
  __device__ __forceinline__ Pre load(int row) const {
    Pre p;
#pragma unroll
    for (int i = 0; i < BR; ++i) p.y[i] = beta != T(0) ? y[(size_t)row * BR + i] : T(0);
    return p;
  }
  __device__ __forceinline__ void store(int row, const T* acc, const Pre& p) const {
#pragma unroll
    for (int i = 0; i < BR; ++i) {
      T v = mul_rn(alpha, acc[i]);
      if (beta != T(0)) v = fma_rn(beta, p.y[i], v);
      y[(size_t)row * BR + i] = v;
    }
  }
};

// r = b - A x
template <class T, int BR>
struct EpiResid {
  const T* b; T* r;
  struct Pre { T b[BR]; };
  __device__ __forceinline__ Pre load(int row) const {
    Pre p;
#pragma unroll
    for (int i = 0; i < BR; ++i) p.b[i] = b[(size_t)row * BR + i];
    return p;
  }
  __device__ __forceinline__ void store(int row, const T* acc, const Pre& p) const {
#pragma unroll
    for (int i = 0; i < BR; ++i) r[(size_t)row * BR + i] = p.b[i] - acc[i];
  }
};

// One Chebyshev step (Saad Alg. 12.1, residual recomputed):
//   r = dinv * (b - A x);  d = c1 * d + c2 * r;  xo = x + d
// d is only touched at the row itself, so it is updated in place; xo must not
// alias x (x is gathered by other rows).  d is not read when c1 == 0.
template <class T, int BR>
struct EpiCheb {
  const T* b; const T* dinv; const T* x; T* d; T* xo; T c1; T c2;
  struct Pre { T b[BR], dinv[BR], x[BR], d[BR]; };
  __device__ __forceinline__ Pre load(int row) const {
    Pre p;
#pragma unroll
    for (int i = 0; i < BR; ++i) {
      const size_t k = (size_t)row * BR + i;
      p.b[i] = b[k];
      p.dinv[i] = dinv[k];
      p.x[i] = x[k];
      p.d[i] = c1 != T(0) ? d[k] : T(0);
    }
    return p;
  }
  __device__ __forceinline__ void store(int row, const T* acc, const Pre& p) const {
#pragma unroll
    for (int i = 0; i < BR; ++i) {
      const size_t k = (size_t)row * BR + i;
      const T r = mul_rn(p.dinv[i], p.b[i] - acc[i]);
      T dn = mul_rn(c2, r);
      if (c1 != T(0)) dn = fma_rn(c1, p.d[i], dn);
      d[k] = dn;
      xo[k] = p.x[i] + dn;
    }
  }
};

// Second Chebyshev step from x = 0 with the first step folded in: the gathered
// vector is x1 = d1 = dinv b / theta (GatherScaled), and
//   r = dinv (b - A x1);  d = c1 d1 + c2 r;  xo = x1 + d.
template <class T, int BR>
struct EpiChebFromZero {
  const T* b; const T* dinv; T* d; T* xo; T inv_theta; T c1; T c2;
  struct Pre { T b[BR], dinv[BR]; };
  __device__ __forceinline__ Pre load(int row) const {
    Pre p;
#pragma unroll
    for (int i = 0; i < BR; ++i) {
      const size_t k = (size_t)row * BR + i;
      p.b[i] = b[k];
      p.dinv[i] = dinv[k];
    }
    return p;
  }
  __device__ __forceinline__ void store(int row, const T* acc, const Pre& p) const {
#pragma unroll
    for (int i = 0; i < BR; ++i) {
      const size_t k = (size_t)row * BR + i;
      const T d1 = mul_rn(mul_rn(p.dinv[i], p.b[i]), inv_theta);
      const T r = mul_rn(p.dinv[i], p.b[i] - acc[i]);
      const T dn = fma_rn(c1, d1, mul_rn(c2, r));
      d[k] = dn;
      xo[k] = d1 + dn;
    }
  }
};

// y = dinv * (A x)  (power iteration on D^-1 A)
template <class T, int BR>
struct EpiDinv {
  const T* dinv; T* y;
  struct Pre { T dinv[BR]; };
  __device__ __forceinline__ Pre load(int row) const {
    Pre p;
#pragma unroll
    for (int i = 0; i < BR; ++i) p.dinv[i] = dinv[(size_t)row * BR + i];
    return p;
  }
  __device__ __forceinline__ void store(int row, const T* acc, const Pre& p) const {
#pragma unroll
    for (int i = 0; i < BR; ++i) y[(size_t)row * BR + i] = mul_rn(p.dinv[i], acc[i]);
  }
};

// ------------------------------------------------------------------ kernel
// Unroll depth: blocks each lane has in flight per trip (register budget): the
// requested depth UREQ (4 or 8) for small blocks, less for large ones; 3 for the
// planar FP32 3 x 3 blocks (64 registers: four 256-thread CTAs per SM instead of
// three at depth 4).  A lane visits its blocks in increasing order at any depth,
// so the depth does not change the sums.
template <class T, int BR, int BC, int UREQ>
__host__ __device__ constexpr int unroll_for() {
  return planar_blocks<T, BR, BC>() ? 3
         : (int)(sizeof(T) * (BR * BC + BC)) <= 24 ? UREQ : ((int)(sizeof(T) * (BR * BC + BC)) <= 64 ? 4 : 2);
}

// acc += sum over the lane's share of row entries [kb, ke) of block * x[col].
// The U column indices and the U blocks are requested together (which entries
// exist follows from the position alone), then the x segments, which need the
// indices: one dependent memory round trip for the matrix data, one for x.
// Column indices are int32 block columns (base 0), or int16 offsets from the
// block row (base = the row) for square matrices whose offsets fit.
template <class T, int BR, int BC, int UREQ, class G, class CI = int>
__device__ __forceinline__ void row_accumulate(const CI* __restrict__ ci, int base, const T* __restrict__ v,
                                               int64_t nnzb, const G& gx, int kb, int ke, int lane, int tpr, T* acc) {
  constexpr int U = unroll_for<T, BR, BC, UREQ>();
  for (int k0 = kb + lane; k0 < ke; k0 += tpr * U) {
    int col[U];
    T blk[U][BR * BC], xv[U][BC];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * tpr;
      if (k < ke) {
        col[u] = base + (int)__ldcs(ci + k);
        load_block<T, BR, BC>(v, nnzb, k, blk[u]);
      } else {
        col[u] = -1;
#pragma unroll
        for (int t = 0; t < BR * BC; ++t) blk[u][t] = T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u * tpr < ke) {
        gx(col[u], xv[u]);
      } else {
#pragma unroll
        for (int t = 0; t < BC; ++t) xv[u][t] = T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int i = 0; i < BR; ++i)
#pragma unroll
        for (int j = 0; j < BC; ++j) acc[i] = fma_rn(blk[u][i * BC + j], xv[u][j], acc[i]);
  }
}

// L2 prefetch of the 16-byte-aligned interior of [p, p + bytes) (one bulk
// prefetch per 64 KB; the unaligned edges are left to the ordinary loads).  (An
// evict-first policy on these prefetches changed no DRAM traffic and cost the 3 x 3
// Chebyshev kernel 6 registers, one CTA per SM.)
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 900)
  const uintptr_t a0 = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  for (uintptr_t a = a0; a < e; a += 65536) {
    const uint32_t n = (uint32_t)(e - a < 65536 ? e - a : 65536);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
  }
#endif
}

// L2 prefetch of the values of blocks [a, b) (three ranges in the planar layout).
template <class T, int BR, int BC>
__device__ __forceinline__ void prefetch_blocks(const T* v, int64_t nnzb, int a, int b) {
  if constexpr (planar_blocks<T, BR, BC>()) {
    prefetch_l2(v + 4 * (int64_t)a, sizeof(T) * 4 * (size_t)(b - a));
    prefetch_l2(v + 4 * nnzb + 4 * (int64_t)a, sizeof(T) * 4 * (size_t)(b - a));
    prefetch_l2(v + 8 * nnzb + a, sizeof(T) * (size_t)(b - a));
  } else {
    prefetch_l2(v + (size_t)a * BR * BC, sizeof(T) * (size_t)(b - a) * BR * BC);
  }
}

// One CTA handles the contiguous block rows [blockIdx.x * rows_per_cta, + rows_per_cta),
// blockDim.x / tpr rows per pass, tpr lanes per row.  With prefetch (> 0, a byte cap),
// thread 0 first asks L2 for the head of the CTA's slice of the (constant) matrix
// arrays, at most `prefetch` bytes of each matrix, before waiting for the previous
// kernel (programmatic dependent launch), so the head streams in while that kernel
// drains and while the CTA works through its first rows.  The cap keeps the lines in
// flight for all resident CTAs well inside L2: a whole 80 KB FP64 slice per CTA
// (about 60 MB for the resident CTAs) was evicted before use and read twice.  Reading the
// row pointers before the wait is only allowed once the matrices are built
// (pre_wait != 0); during set-up the previous kernel may still be writing them.
// Two-matrix launches may take a slot table (ord2, Bsr::ord2): the CTA's slots
// [r0, r1) are then its block rows sorted by length within 32-row windows (the same
// rows when r0 is a multiple of 32, i.e. tpr <= 8), so the rows of a warp have equal
// length and no lane idles while a longer row in its warp finishes.  A slot's record
// replaces the four row-pointer loads; each row is summed exactly as without it.
template <class T, int BR, int BC1, int BC2, class Epi, class G1 = GatherX<T, BC1>, int UREQ = 4, class CI1 = int>
__global__ void __launch_bounds__(256) k_bsr_spmv(int nbr, int tpr, int rows_per_cta, int prefetch, int pre_wait,
    const int4* __restrict__ ord2,
    const int* __restrict__ rp1, const CI1* __restrict__ ci1, const T* __restrict__ v1, int64_t nnzb1, G1 g1,
    const int* __restrict__ rp2, const int* __restrict__ ci2, const T* __restrict__ v2, int64_t nnzb2,
    const T* __restrict__ x2,
    Epi epi) {
  const int r0 = blockIdx.x * rows_per_cta;
  const int r1 = r0 + rows_per_cta < nbr ? r0 + rows_per_cta : nbr;
  if (!pre_wait) dep_wait();
  if (prefetch && threadIdx.x == 0 && r0 < r1) {
    const int a = rp1[r0];
    const int cap1 = prefetch / (int)(BR * BC1 * sizeof(T) + sizeof(CI1));
    const int b = rp1[r1] - a < cap1 ? rp1[r1] : a + cap1;
    prefetch_blocks<T, BR, BC1>(v1, nnzb1, a, b);
    prefetch_l2(ci1 + a, sizeof(CI1) * (size_t)(b - a));
    if constexpr (BC2 > 0) {
      const int a2 = rp2[r0];
      const int cap2 = prefetch / (int)(BR * BC2 * sizeof(T) + sizeof(int));
      const int b2 = rp2[r1] - a2 < cap2 ? rp2[r1] : a2 + cap2;
      prefetch_blocks<T, BR, BC2>(v2, nnzb2, a2, b2);
      prefetch_l2(ci2 + a2, sizeof(int) * (size_t)(b2 - a2));
    }
  }
  if (pre_wait) dep_wait();
  const int per_pass = blockDim.x / tpr;
  const int lane = threadIdx.x & (tpr - 1);
  for (int base = r0; base < r1; base += per_pass) {
    const int slot = base + threadIdx.x / tpr;
    const bool valid = slot < r1;
    int row = slot, kb1 = 0, ke1 = 0, kb2 = 0, ke2 = 0;
    if (valid) {
      if (BC2 > 0 && ord2) {
        const int4 o = __ldg(ord2 + slot);
        row = o.x & 0xFFFFFF;
        kb1 = o.y;
        ke1 = kb1 + (int)((unsigned)o.x >> 24);
        kb2 = o.z;
        ke2 = kb2 + o.w;
      } else {
        kb1 = rp1[row];
        ke1 = rp1[row + 1];
        if constexpr (BC2 > 0) {
          kb2 = rp2[row];
          ke2 = rp2[row + 1];
        }
      }
    }
    T acc[BR];
#pragma unroll
    for (int i = 0; i < BR; ++i) acc[i] = T(0);
    typename Epi::Pre pre;
    if (valid && lane == 0) pre = epi.load(row);
    if (valid) {
      row_accumulate<T, BR, BC1, UREQ, G1, CI1>(ci1, sizeof(CI1) == 4 ? 0 : row, v1, nnzb1, g1, kb1, ke1, lane, tpr,
                                                acc);
      if constexpr (BC2 > 0)
        row_accumulate<T, BR, BC2, UREQ>(ci2, 0, v2, nnzb2, GatherX<T, BC2, G1::kKeep>{x2}, kb2, ke2, lane, tpr,
                                         acc);
    }
    for (int off = tpr >> 1; off > 0; off >>= 1)
#pragma unroll
      for (int i = 0; i < BR; ++i) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], off, tpr);
    if (valid && lane == 0) epi.store(row, acc, pre);
  }
}

// ------------------------------------------------------------------ staged 2 x 2 FP32 steps
// Chebyshev steps (EpiCheb, EpiChebFromZero) on 2 x 2 FP32 blocks with 16-bit column
// offsets, with the offsets staged one chunk ahead.  In k_bsr_spmv a warp's pass makes
// two dependent memory round trips: column offsets (with the blocks), then the x they
// index.  Here a persistent CTA walks chunks of R consecutive block rows (chunk c,
// c + gridDim.x, ...; R = 256 / tpr, one k_bsr_spmv CTA's rows).  While it computes
// chunk i, the TMA engine copies the column offsets of chunk i + 2 into a two-stage
// shared-memory ring (cp.async.bulk from the 8-entry boundary below the chunk's first
// block, 16-byte aligned, completing on the stage's mbarrier), and the chunk's block
// values are bulk-prefetched into L2.  A pass then issues its x gathers and its block
// loads together: one round trip.  Each lane visits the same blocks in the same order
// and rounds the same way as k_bsr_spmv, so the results are bit-identical.  smax bounds
// every chunk's offsets, counted from that 8-entry boundary (bsr_make_delta16).  Every
// wait is bounded (about a second of clock); on a timeout the CTA sets *err, waits
// (bounded) for the copy still in flight and returns.
constexpr int kStageDepth = 2;

__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t parity) {
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

// bytes of one ring stage (column offsets) for chunks of at most smax blocks
__host__ __device__ constexpr size_t stage_bytes(int smax) { return (2 * ((size_t)smax + 8) + 15) & ~(size_t)15; }
// dynamic shared memory of the staged kernel: the ring, then one mbarrier per stage
__host__ __device__ constexpr size_t staged_smem_bytes(int smax) {
  return kStageDepth * stage_bytes(smax) + 8 * kStageDepth;
}

// Thread 0: the column offsets of chunk c into ring stage st, and an L2 prefetch of
// its block values (no-op past the last chunk).
__device__ __forceinline__ void stage_issue(int c, int nchunks, int R, int nbr, int st, uint32_t sbase, int smax,
                                            const int* __restrict__ rp, const int16_t* __restrict__ ci,
                                            const float* __restrict__ v, int* s_a8) {
  if (c >= nchunks) return;
  const int r0 = c * R;
  const int r1 = r0 + R < nbr ? r0 + R : nbr;
  const int a = rp[r0], b = rp[r1];
  const int a8 = a & ~7, b8 = (b + 7) & ~7;
  s_a8[st] = a8;
  const uint32_t cbytes = 2u * (uint32_t)(b8 - a8);
  const uint32_t buf = sbase + (uint32_t)(st * stage_bytes(smax));
  const uint32_t bar = sbase + (uint32_t)(kStageDepth * stage_bytes(smax)) + 8u * st;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(cbytes) : "memory");
  if (cbytes)
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(buf),
                 "l"(ci + a8), "r"(cbytes), "r"(bar)
                 : "memory");
  prefetch_l2(v + 4 * (size_t)a, 16 * (size_t)(b - a));
}

template <class Epi, class G1, int UREQ>
__global__ void __launch_bounds__(256) k_bsr_cheb_staged(int nbr, int tpr, int R, int nchunks, int pre_wait,
                                                         const int* __restrict__ rp, const int16_t* __restrict__ ci,
                                                         const float* __restrict__ v, G1 g1, Epi epi, int smax,
                                                         int* __restrict__ err) {
  constexpr int BR = 2, BC = 2;
  constexpr int U = unroll_for<float, BR, BC, UREQ>();
  extern __shared__ __align__(16) unsigned char stage_sm[];
  __shared__ int s_a8[kStageDepth];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(stage_sm);
  const uint32_t bar0 = sbase + (uint32_t)(kStageDepth * stage_bytes(smax));
  if (threadIdx.x == 0) {
    for (int st = 0; st < kStageDepth; ++st)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u * st) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (!pre_wait) dep_wait();
  if (threadIdx.x == 0)
    for (int st = 0; st < kStageDepth; ++st)
      stage_issue(blockIdx.x + st * gridDim.x, nchunks, R, nbr, st, sbase, smax, rp, ci, v, s_a8);
  __syncthreads();
  if (pre_wait) dep_wait();
  const int lane = threadIdx.x & (tpr - 1);
  for (int i = 0;; ++i) {
    const int c = blockIdx.x + i * gridDim.x;
    if (c >= nchunks) break;
    const int st = i % kStageDepth;
    const int r0 = c * R;
    const int r1 = r0 + R < nbr ? r0 + R : nbr;
    const int row = r0 + threadIdx.x / tpr;     // R = blockDim.x / tpr: one row per lane group
    const bool valid = row < r1;
    typename Epi::Pre pre;
    if (valid && lane == 0) pre = epi.load(row);
    int kb = 0, ke = 0;
    if (valid) { kb = rp[row]; ke = rp[row + 1]; }
    const bool ok = stage_wait(bar0 + 8u * st, (uint32_t)(i / kStageDepth) & 1u);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      // the copies still in flight: this stage's and the other stage's next chunk
      stage_wait(bar0 + 8u * st, (uint32_t)(i / kStageDepth) & 1u);
      if (c + (int)gridDim.x < nchunks)
        stage_wait(bar0 + 8u * ((i + 1) % kStageDepth), (uint32_t)((i + 1) / kStageDepth) & 1u);
      return;
    }
    const int16_t* sc = reinterpret_cast<const int16_t*>(stage_sm + st * stage_bytes(smax));
    const int a8 = s_a8[st];
    float acc[BR] = {0.f, 0.f};
    for (int k0 = kb + lane; k0 < ke; k0 += tpr * U) {
      float4 q[U];
      float xv[U][BC];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = k0 + u * tpr;
        if (k < ke) {
          q[u] = __ldcs(reinterpret_cast<const float4*>(v) + k);
          g1(row + (int)sc[k - a8], xv[u]);
        } else {
          q[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          xv[u][0] = 0.f;
          xv[u][1] = 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        acc[0] = fma_rn(q[u].x, xv[u][0], acc[0]);
        acc[0] = fma_rn(q[u].y, xv[u][1], acc[0]);
        acc[1] = fma_rn(q[u].z, xv[u][0], acc[1]);
        acc[1] = fma_rn(q[u].w, xv[u][1], acc[1]);
      }
    }
    for (int off = tpr >> 1; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < BR; ++q) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], off, tpr);
    if (valid && lane == 0) epi.store(row, acc, pre);
    __syncthreads();   // every lane is done with this stage: refill it
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      stage_issue(c + kStageDepth * (int)gridDim.x, nchunks, R, nbr, st, sbase, smax, rp, ci, v, s_a8);
    }
  }
}

// ------------------------------------------------------------------ host API
// y = alpha * A x + beta * y
template <class T> void spmv_axpby(const Bsr& A, const T* x, T alpha, T beta, T* y, cudaStream_t s);
// y = alpha * (A1 x1 + A2 x2) + beta * y   (A2 may have 0 block rows == none)
template <class T> void spmv2_axpby(const Bsr& A1, const T* x1, const Bsr* A2, const T* x2, T alpha, T beta, T* y, cudaStream_t s);
// r = b - A1 x1 - A2 x2
template <class T> void spmv2_resid(const Bsr& A1, const T* x1, const Bsr* A2, const T* x2, const T* b, T* r, cudaStream_t s);
// Coarse right-hand side of a V-cycle level in one pass: y = RAn x + R b with
// RAn = -(R A), i.e. y = R (b - A x), the restricted residual, without forming
// b - A x (R: k x b blocks, RAn: the same block rows and k x b blocks).
template <class T> void spmv_restrict(const Bsr& R, const T* b, const Bsr& RAn, const T* x, T* y, cudaStream_t s);
// Chebyshev step epilogue (see EpiCheb)
template <class T> void spmv_cheb(const Bsr& A, const T* x, const T* b, const T* dinv, T* d, T* xo, T c1, T c2, cudaStream_t s);
// y = dinv * (A x)
template <class T> void spmv_dinv(const Bsr& A, const T* x, const T* dinv, T* y, cudaStream_t s);
// True (and the flag cleared) if a staged Chebyshev step gave up waiting for its copies
// since the last call; the results of that step are then not valid.
bool spmv_stage_failed(cudaStream_t s);
// Chebyshev steps 1 and 2 from x = 0 in one pass (see EpiChebFromZero)
template <class T> void spmv_cheb_from_zero(const Bsr& A, const T* b, const T* dinv, T* d, T* xo, T inv_theta, T c1,
                                            T c2, cudaStream_t s);

}  // namespace fsi

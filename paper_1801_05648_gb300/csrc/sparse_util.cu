#include "sparse_util.cuh"

#include <climits>

namespace fsi {

namespace {

constexpr int kScanBlock = 1024;

__device__ __forceinline__ long long warp_incl_scan(long long v, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += t;
  }
  return v;
}

// Exclusive scan of a 1024-element tile; writes block totals.
template <class Tin>
__global__ void __launch_bounds__(kScanBlock) k_scan_tile(const Tin* __restrict__ in, long long* __restrict__ out,
                                                          int64_t n, long long* __restrict__ bsum) {
  __shared__ long long wsum[32];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long v = i < n ? (long long)in[i] : 0;
  long long inc = warp_incl_scan(v, lane);
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    long long t = wsum[lane];
    t = warp_incl_scan(t, lane);
    wsum[lane] = t;
  }
  __syncthreads();
  long long base = w ? wsum[w - 1] : 0;
  if (i < n) out[i] = base + inc - v;
  if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = base + inc;
}

__global__ void k_scan_add(long long* __restrict__ out, int64_t n, const long long* __restrict__ boff) {
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
}

// exclusive scan of n long longs/ints into out (n entries); returns total on the host
template <class Tin>
long long scan_ll(const Tin* in, long long* out, int64_t n, cudaStream_t s) {
  if (n == 0) return 0;
  const int nb = div_up(n, kScanBlock);
  DBuf<long long> bsum(nb), boff(nb);
  k_scan_tile<Tin><<<nb, kScanBlock, 0, s>>>(in, out, n, bsum.p);
  FSI_CHECK_LAUNCH();
  long long total;
  if (nb == 1) {
    FSI_CUDA(cudaMemcpyAsync(&total, bsum.p, sizeof(long long), cudaMemcpyDeviceToHost, s));
    FSI_CUDA(cudaStreamSynchronize(s));
    return total;
  }
  total = scan_ll<long long>(bsum.p, boff.p, nb, s);
  k_scan_add<<<nb, kScanBlock, 0, s>>>(out, n, boff.p);
  FSI_CHECK_LAUNCH();
  return total;
}

__global__ void k_ll_to_int(const long long* __restrict__ in, int* __restrict__ out, int64_t n, long long total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int)in[i];
  if (i == n) out[n] = (int)total;
}

__device__ __forceinline__ int lower_bound_i(const int* a, int lo, int hi, int key) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int64_t lower_bound_l(const int* a, int64_t lo, int64_t hi, int key) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// --------------------------------------------------------------- extraction
// One thread per block row: merge the br sorted scalar rows restricted to the
// column window into sorted block columns.
template <bool FILL>
__global__ void k_extract(const int64_t* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ va,
                          int64_t r0, int nbr, int br, int64_t c0, int64_t c1, int bc, int* __restrict__ cnt,
                          const int* __restrict__ orp, int* __restrict__ oci, double* __restrict__ ova) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nbr) return;
  int64_t ptr[6], end[6];
  for (int q = 0; q < br; ++q) {
    const int64_t r = r0 + (int64_t)row * br + q;
    ptr[q] = lower_bound_l(ci, rp[r], rp[r + 1], (int)c0);
    end[q] = lower_bound_l(ci, ptr[q], rp[r + 1], (int)c1);
  }
  int count = 0;
  int64_t outpos = FILL ? orp[row] : 0;
  while (true) {
    int best = INT_MAX;
    for (int q = 0; q < br; ++q)
      if (ptr[q] < end[q]) {
        int b = (int)((ci[ptr[q]] - c0) / bc);
        if (b < best) best = b;
      }
    if (best == INT_MAX) break;
    if (FILL) {
      double* blk = ova + outpos * (int64_t)(br * bc);
      for (int t = 0; t < br * bc; ++t) blk[t] = 0.0;
      oci[outpos] = best;
      for (int q = 0; q < br; ++q)
        while (ptr[q] < end[q] && (int)((ci[ptr[q]] - c0) / bc) == best) {
          blk[q * bc + (int)((ci[ptr[q]] - c0) % bc)] = va[ptr[q]];
          ++ptr[q];
        }
      ++outpos;
    } else {
      for (int q = 0; q < br; ++q)
        while (ptr[q] < end[q] && (int)((ci[ptr[q]] - c0) / bc) == best) ++ptr[q];
    }
    ++count;
  }
  if (!FILL) cnt[row] = count;
}

// --------------------------------------------------------------- add
template <bool FILL>
__global__ void k_add(int nbr, int bsz, const int* __restrict__ arp, const int* __restrict__ aci,
                      const double* __restrict__ ava, const int* __restrict__ brp, const int* __restrict__ bci,
                      const double* __restrict__ bva, double alpha, int* __restrict__ cnt, const int* __restrict__ crp,
                      int* __restrict__ cci, double* __restrict__ cva) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nbr) return;
  int ia = arp[row], ea = arp[row + 1], ib = brp[row], eb = brp[row + 1];
  int count = 0;
  int pos = FILL ? crp[row] : 0;
  while (ia < ea || ib < eb) {
    int ca = ia < ea ? aci[ia] : INT_MAX;
    int cb = ib < eb ? bci[ib] : INT_MAX;
    int c = ca < cb ? ca : cb;
    if (FILL) {
      double* o = cva + (int64_t)pos * bsz;
      for (int t = 0; t < bsz; ++t) o[t] = 0.0;
      if (ca == c) for (int t = 0; t < bsz; ++t) o[t] += ava[(int64_t)ia * bsz + t];
      if (cb == c) for (int t = 0; t < bsz; ++t) o[t] += alpha * bva[(int64_t)ib * bsz + t];
      cci[pos] = c;
      ++pos;
    }
    if (ca == c) ++ia;
    if (cb == c) ++ib;
    ++count;
  }
  if (!FILL) cnt[row] = count;
}

// --------------------------------------------------------------- transpose
__global__ void k_count_cols(int64_t nnzb, const int* __restrict__ ci, int* __restrict__ cnt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnzb) atomicAdd(cnt + ci[k], 1);
}
__global__ void k_row_of_block(int nbr, const int* __restrict__ rp, int* __restrict__ rowof) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nbr) return;
  for (int k = rp[row]; k < rp[row + 1]; ++k) rowof[k] = row;
}
__global__ void k_scatter_t(int64_t nnzb, const int* __restrict__ ci, const int* __restrict__ rowof,
                            const int* __restrict__ trp, int* __restrict__ cursor, int* __restrict__ trow,
                            int* __restrict__ tsrc) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnzb) return;
  const int c = ci[k];
  const int pos = trp[c] + atomicAdd(cursor + c, 1);
  trow[pos] = rowof[k];
  tsrc[pos] = (int)k;
}
// insertion sort of each segment by key (with a payload)
__global__ void k_sort_segments(int nseg, const int* __restrict__ off, int* __restrict__ key, int* __restrict__ pay) {
  const int sgm = blockIdx.x * blockDim.x + threadIdx.x;
  if (sgm >= nseg) return;
  const int lo = off[sgm], hi = off[sgm + 1];
  for (int i = lo + 1; i < hi; ++i) {
    int k = key[i], p = pay ? pay[i] : 0;
    int j = i - 1;
    while (j >= lo && key[j] > k) {
      key[j + 1] = key[j];
      if (pay) pay[j + 1] = pay[j];
      --j;
    }
    key[j + 1] = k;
    if (pay) pay[j + 1] = p;
  }
}
__global__ void k_gather_t(int64_t nnzb, int br, int bc, const int* __restrict__ tsrc, const double* __restrict__ va,
                           double* __restrict__ tva) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnzb) return;
  const double* s = va + (int64_t)tsrc[k] * br * bc;
  double* d = tva + k * br * bc;
  // source block br x bc row-major -> destination bc x br row-major
  for (int i = 0; i < br; ++i)
    for (int j = 0; j < bc; ++j) d[j * br + i] = s[i * bc + j];
}

// --------------------------------------------------------------- SpGEMM
constexpr int kHashSize = 1024;      // per warp, shared memory (2 x 4 x 4 KB per block)
constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ unsigned hash_slot(int key) { return ((unsigned)key * 2654435761u) & (kHashSize - 1); }

// returns 1 when key was newly inserted, 0 when present, -1 when the table is
// full (every slot probed once: the loop always ends)
__device__ __forceinline__ int hash_insert(int* table, int key) {
  unsigned h = hash_slot(key);
  for (int probe = 0; probe < kHashSize; ++probe) {
    int prev = atomicCAS(table + h, -1, key);
    if (prev == -1) return 1;
    if (prev == key) return 0;
    h = (h + 1) & (kHashSize - 1);
  }
  return -1;
}

// Symbolic pass, one warp per row of A.  FILL = false: count unique block
// columns (flag overflow).  FILL = true: write them sorted.
template <bool FILL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_spgemm_sym(int nbr, const int* __restrict__ arp,
                                                                    const int* __restrict__ aci,
                                                                    const int* __restrict__ brp,
                                                                    const int* __restrict__ bci, int* __restrict__ cnt,
                                                                    const int* __restrict__ crp, int* __restrict__ cci,
                                                                    int* __restrict__ overflow) {
  __shared__ int table[kWarpsPerBlock][kHashSize];
  __shared__ int list[kWarpsPerBlock][kHashSize];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kWarpsPerBlock + w;
  if (row >= nbr) return;   // whole warp exits together
  int* tb = table[w];
  for (int t = lane; t < kHashSize; t += 32) tb[t] = -1;
  __syncwarp();
  int inserted = 0, full = 0;
  for (int k = arp[row]; k < arp[row + 1]; ++k) {
    const int kk = aci[k];
    for (int q = brp[kk] + lane; q < brp[kk + 1]; q += 32) {
      const int r = hash_insert(tb, bci[q]);
      if (r < 0) full = 1; else inserted += r;
    }
    __syncwarp();
    // bail out on overflow (table over 3/4 full or a failed insert)
    int tot = inserted;
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, off);
    const int anyfull = __any_sync(0xffffffffu, full);
    if (tot > kHashSize * 3 / 4 || anyfull) {
      if (lane == 0) atomicExch(overflow, 1);
      return;
    }
  }
  for (int off = 16; off > 0; off >>= 1) inserted += __shfl_xor_sync(0xffffffffu, inserted, off);
  if (!FILL) {
    if (lane == 0) cnt[row] = inserted;
    return;
  }
  // compact the table
  int* ls = list[w];
  int base = 0;
  for (int t0 = 0; t0 < kHashSize; t0 += 32) {
    int v = tb[t0 + lane];
    unsigned m = __ballot_sync(0xffffffffu, v != -1);
    if (v != -1) ls[base + __popc(m & ((1u << lane) - 1))] = v;
    base += __popc(m);
  }
  __syncwarp();
  const int out0 = crp[row];
  for (int e = lane; e < base; e += 32) {
    const int v = ls[e];
    int rank = 0;
    for (int f = 0; f < base; ++f) rank += ls[f] < v;
    cci[out0 + rank] = v;
  }
}

template <int BR, int BK, int BC>
__global__ void __launch_bounds__(128) k_spgemm_num(int nbr, const int* __restrict__ arp, const int* __restrict__ aci,
                                                    const double* __restrict__ ava, const int* __restrict__ brp,
                                                    const int* __restrict__ bci, const double* __restrict__ bva,
                                                    const int* __restrict__ crp, const int* __restrict__ cci,
                                                    double* __restrict__ cva) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 4 + w;
  if (row >= nbr) return;
  for (int e = crp[row] + lane; e < crp[row + 1]; e += 32) {
    const int J = cci[e];
    double acc[BR * BC];
#pragma unroll
    for (int t = 0; t < BR * BC; ++t) acc[t] = 0.0;
    for (int k = arp[row]; k < arp[row + 1]; ++k) {
      const int kk = aci[k];
      const int pos = lower_bound_i(bci, brp[kk], brp[kk + 1], J);
      if (pos < brp[kk + 1] && bci[pos] == J) {
        const double* a = ava + (int64_t)k * BR * BK;
        const double* b = bva + (int64_t)pos * BK * BC;
#pragma unroll
        for (int i = 0; i < BR; ++i)
#pragma unroll
          for (int j = 0; j < BC; ++j) {
            double s = acc[i * BC + j];
#pragma unroll
            for (int q = 0; q < BK; ++q) s += a[i * BK + q] * b[q * BC + j];
            acc[i * BC + j] = s;
          }
      }
    }
    double* c = cva + (int64_t)e * BR * BC;
#pragma unroll
    for (int t = 0; t < BR * BC; ++t) c[t] = acc[t];
  }
}

// --------------------------------------------------------------- misc
__global__ void k_scale_rows(int nbr, int br, int bc, const int* __restrict__ rp, double* __restrict__ va,
                             const double* __restrict__ w) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nbr) return;
  for (int k = rp[row]; k < rp[row + 1]; ++k)
    for (int i = 0; i < br; ++i)
      for (int j = 0; j < bc; ++j) va[((int64_t)k * br + i) * bc + j] *= w[(int64_t)row * br + i];
}
__global__ void k_scale_all(int64_t n, double alpha, double* __restrict__ va) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) va[i] *= alpha;
}
__global__ void k_delta16(int nbr, const int* __restrict__ rp, const int* __restrict__ ci, int16_t* __restrict__ d,
                          int* __restrict__ overflow) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nbr) return;
  for (int k = rp[row]; k < rp[row + 1]; ++k) {
    const int off = ci[k] - row;
    if (off < -32768 || off > 32767) { atomicExch(overflow, 1); return; }
    d[k] = (int16_t)off;
  }
}
// Slot table of a two-matrix SpMV (block rows of A1 next to those of A2): within
// each window of 32 block rows, the rows by decreasing A1 length, then decreasing A2
// length, ties in row order; record {row | len1 << 24, first A1 block, first A2 block,
// len2}.  One warp per window ranks its rows by counting.  *bad = 1 if an A1 row is
// longer than 255 blocks (the record cannot hold it).
__global__ void k_pair_order(int nbr, const int* __restrict__ rp1, const int* __restrict__ rp2,
                             int4* __restrict__ ord, int* __restrict__ bad) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int kb1 = 0, kb2 = 0, l1 = -1, l2 = -1;     // lanes past the end rank last and write nothing
  if (row < nbr) {
    kb1 = rp1[row];
    l1 = rp1[row + 1] - kb1;
    kb2 = rp2[row];
    l2 = rp2[row + 1] - kb2;
    if (l1 > 255) atomicExch(bad, 1);
  }
  int rank = 0;
  for (int j = 0; j < 32; ++j) {
    const int a = __shfl_sync(0xffffffffu, l1, j), b = __shfl_sync(0xffffffffu, l2, j);
    rank += (a > l1 || (a == l1 && (b > l2 || (b == l2 && j < lane)))) ? 1 : 0;
  }
  if (row < nbr && l1 <= 255) ord[row - lane + rank] = make_int4((int)row | (l1 << 24), kb1, kb2, l2);
}
__global__ void k_point_diag(int nbr, int b, const int* __restrict__ rp, const int* __restrict__ ci,
                             const double* __restrict__ va, double* __restrict__ diag) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nbr) return;
  const int pos = lower_bound_i(ci, rp[row], rp[row + 1], row);
  const bool has = pos < rp[row + 1] && ci[pos] == row;
  for (int i = 0; i < b; ++i) diag[(int64_t)row * b + i] = has ? va[((int64_t)pos * b + i) * b + i] : 0.0;
}
__global__ void k_invert_nonzero(int64_t n, const double* __restrict__ d, double* __restrict__ o) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = d[i] != 0.0 ? 1.0 / d[i] : 0.0;
}
__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
// FP32 copy of 3 x 3 blocks in the planar layout: value t of block k goes to
// 4k + t (t < 4), 4 nnzb + 4k + t - 4 (t < 8) or 8 nnzb + k (t = 8).
__global__ void k_to_f32_planar9(int64_t nnzb, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * nnzb) return;
  const int64_t k = i / 9;
  const int t = (int)(i - 9 * k);
  const int64_t o = t < 4 ? 4 * k + t : (t < 8 ? 4 * nnzb + 4 * k + (t - 4) : 8 * nnzb + k);
  b[o] = (float)a[i];
}
__global__ void k_to_dense(int nbr, int br, int bc, int ncols, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ va, double* __restrict__ D) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nbr) return;
  for (int k = rp[row]; k < rp[row + 1]; ++k)
    for (int i = 0; i < br; ++i)
      for (int j = 0; j < bc; ++j)
        D[((int64_t)row * br + i) * ncols + (int64_t)ci[k] * bc + j] = va[((int64_t)k * br + i) * bc + j];
}

// Gauss-Jordan elimination with partial pivoting on [M | I] (M is destroyed, X
// becomes M^-1), one launch per pivot column over the whole GPU.  Before step p,
// row p holds the pivot row (swapped in and scaled to a unit pivot) and f holds
// column p; step p eliminates column p from every other row.  The CTA that
// finishes a step last (an atomic ticket taken after a memory fence: nothing
// waits) prepares pivot p + 1.
constexpr int kGjThreads = 256;

// Rows that are entirely zero become identity rows; X = I.
__global__ void k_gj_init(int n, double* __restrict__ M, double* __restrict__ X) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nwarps) {
    bool nz = false;
    for (int c = lane; c < n; c += 32) nz |= M[r * n + c] != 0.0;
    nz = __any_sync(0xffffffffu, nz);
    if (!nz && lane == 0) M[r * n + r] = 1.0;
    for (int c = lane; c < n; c += 32) X[r * n + c] = c == r ? 1.0 : 0.0;
  }
}

// Pivot p: the largest |M[r][p]|, r >= p (ties to the lowest row), swapped into
// row p of M and X, row p scaled by 1 / M[p][p], f = column p.  One CTA; the loads
// bypass L1 (other CTAs wrote the data in the same launch).
__device__ void gj_prepare(int n, int p, double* __restrict__ M, double* __restrict__ X, double* __restrict__ f,
                           int* __restrict__ fail) {
  __shared__ double bval[kGjThreads / 32];
  __shared__ int bidx[kGjThreads / 32];
  __shared__ int piv;
  __shared__ double inv;
  const int tid = threadIdx.x;
  double best = -1.0;
  int bi = p;
  for (int r = p + tid; r < n; r += blockDim.x) {
    const double v = fabs(__ldcg(M + (int64_t)r * n + p));
    if (v > best) { best = v; bi = r; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if ((tid & 31) == 0) { bval[tid >> 5] = best; bidx[tid >> 5] = bi; }
  __syncthreads();
  if (tid == 0) {
    double b = -1.0;
    int i = p;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (bval[w] > b || (bval[w] == b && bidx[w] < i)) { b = bval[w]; i = bidx[w]; }
    piv = i;
    if (!(b > 0.0)) *fail = 1;
  }
  __syncthreads();
  const int pr = piv;
  if (pr != p)
    for (int c = tid; c < n; c += blockDim.x) {
      double* a = M + (int64_t)p * n + c;
      double* b = M + (int64_t)pr * n + c;
      const double t = __ldcg(a); *a = __ldcg(b); *b = t;
      double* xa = X + (int64_t)p * n + c;
      double* xb = X + (int64_t)pr * n + c;
      const double u = __ldcg(xa); *xa = __ldcg(xb); *xb = u;
    }
  __syncthreads();
  if (tid == 0) inv = 1.0 / __ldcg(M + (int64_t)p * n + p);
  __syncthreads();
  const double s = inv;
  for (int c = tid; c < n; c += blockDim.x) {
    M[(int64_t)p * n + c] = __dmul_rn(__ldcg(M + (int64_t)p * n + c), s);
    X[(int64_t)p * n + c] = __dmul_rn(__ldcg(X + (int64_t)p * n + c), s);
  }
  for (int r = tid; r < n; r += blockDim.x) f[r] = r == p ? 0.0 : __ldcg(M + (int64_t)r * n + p);
}

__global__ void __launch_bounds__(kGjThreads) k_gj_first(int n, double* M, double* X, double* f, int* fail) {
  gj_prepare(n, 0, M, X, f, fail);
}

// Step p: row r != p of [M | X] -= f[r] * row p; column p of M becomes e_p.
__global__ void __launch_bounds__(kGjThreads) k_gj_step(int n, int p, double* __restrict__ M,
                                                        double* __restrict__ X, double* __restrict__ f,
                                                        unsigned* __restrict__ ticket, int* __restrict__ fail) {
  __shared__ bool last;
  const int64_t w = 2 * (int64_t)n;
  const int64_t total = (int64_t)n * w;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / w);
    const int c = (int)(t - (int64_t)r * w);
    if (r == p) continue;
    const double fr = f[r];
    if (c < n) {
      double* m = M + (int64_t)r * n + c;
      if (c == p) *m = 0.0;
      else if (fr != 0.0) *m = __fma_rn(-fr, M[(int64_t)p * n + c], *m);
    } else if (fr != 0.0) {
      double* x = X + (int64_t)r * n + (c - n);
      *x = __fma_rn(-fr, X[(int64_t)p * n + (c - n)], *x);
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (p + 1 < n) gj_prepare(n, p + 1, M, X, f, fail);
  if (threadIdx.x == 0) *ticket = 0u;
}

template <class F>
void spgemm_dispatch(int br, int bk, int bc, F&& f) {
#define FSI_G(a, b, c) if (br == a && bk == b && bc == c) { f.template operator()<a, b, c>(); return; }
  // A * P_tent / A * P (b x b times b x k)
  FSI_G(1, 1, 1) FSI_G(2, 2, 2) FSI_G(3, 3, 3) FSI_G(2, 2, 3) FSI_G(3, 3, 6) FSI_G(6, 6, 6)
  // R * (A P)  (k x b times b x k)
  FSI_G(3, 2, 3) FSI_G(6, 3, 6)
  // R * A on the first level of the rigid-body solid hierarchy (k x b times b x b)
  FSI_G(3, 2, 2) FSI_G(6, 3, 3)
  // pressure Schur: (1 x d) * (d x 1)
  FSI_G(1, 2, 1) FSI_G(1, 3, 1)
#undef FSI_G
  throw Error(EINVAL_, "unsupported SpGEMM block shape " + std::to_string(br) + "x" + std::to_string(bk) + "x" +
                           std::to_string(bc));
}

void finalize_rowptr(const int* cnt, Bsr& C, cudaStream_t s) {
  DBuf<long long> tmp(C.nbr + 1);
  long long total = scan_ll<int>(cnt, tmp.p, C.nbr, s);
  require(total < INT_MAX, "sparse matrix too large for 32-bit block indices");
  C.rowptr.alloc(C.nbr + 1);
  k_ll_to_int<<<div_up(C.nbr + 1, 256), 256, 0, s>>>(tmp.p, C.rowptr.p, C.nbr, total);
  FSI_CHECK_LAUNCH();
  C.nnzb = total;
  C.colind.alloc(total > 0 ? total : 1);
  C.v64.alloc(total > 0 ? total * C.br * C.bc : 1);
}

}  // namespace

int64_t exclusive_scan(const int* in, int* out, int64_t n, cudaStream_t s) {
  DBuf<long long> tmp(n + 1);
  long long total = scan_ll<int>(in, tmp.p, n, s);
  require(total < INT_MAX, "scan overflow");
  k_ll_to_int<<<div_up(n + 1, 256), 256, 0, s>>>(tmp.p, out, n, total);
  FSI_CHECK_LAUNCH();
  return total;
}

void extract_bsr(const CsrView& A, int64_t r0, int nbr, int br, int64_t c0, int nbc, int bc, Bsr& out,
                 cudaStream_t s) {
  require(br <= 6, "extract_bsr: block rows > 6");
  out = Bsr();
  out.nbr = nbr; out.nbc = nbc; out.br = br; out.bc = bc;
  DBuf<int> cnt(nbr > 0 ? nbr : 1);
  const int64_t c1 = c0 + (int64_t)nbc * bc;
  if (nbr > 0) {
    k_extract<false><<<div_up(nbr, 128), 128, 0, s>>>(A.rowptr, A.colind, A.vals, r0, nbr, br, c0, c1, bc, cnt.p,
                                                    nullptr, nullptr, nullptr);
    FSI_CHECK_LAUNCH();
  }
  finalize_rowptr(cnt.p, out, s);
  if (nbr > 0) {
    k_extract<true><<<div_up(nbr, 128), 128, 0, s>>>(A.rowptr, A.colind, A.vals, r0, nbr, br, c0, c1, bc, nullptr,
                                                   out.rowptr.p, out.colind.p, out.v64.p);
    FSI_CHECK_LAUNCH();
  }
  set_tpr(out);
}

void bsr_add(const Bsr& A, const Bsr& B, double alpha, Bsr& C, cudaStream_t s) {
  require(A.nbr == B.nbr && A.nbc == B.nbc && A.br == B.br && A.bc == B.bc, "bsr_add: shape mismatch");
  C = Bsr();
  C.nbr = A.nbr; C.nbc = A.nbc; C.br = A.br; C.bc = A.bc;
  DBuf<int> cnt(A.nbr > 0 ? A.nbr : 1);
  const int bsz = A.br * A.bc;
  if (A.nbr > 0) {
    k_add<false><<<div_up(A.nbr, 128), 128, 0, s>>>(A.nbr, bsz, A.rowptr.p, A.colind.p, A.v64.p, B.rowptr.p,
                                                   B.colind.p, B.v64.p, alpha, cnt.p, nullptr, nullptr, nullptr);
    FSI_CHECK_LAUNCH();
  }
  finalize_rowptr(cnt.p, C, s);
  if (A.nbr > 0) {
    k_add<true><<<div_up(A.nbr, 128), 128, 0, s>>>(A.nbr, bsz, A.rowptr.p, A.colind.p, A.v64.p, B.rowptr.p,
                                                  B.colind.p, B.v64.p, alpha, nullptr, C.rowptr.p, C.colind.p,
                                                  C.v64.p);
    FSI_CHECK_LAUNCH();
  }
  set_tpr(C);
}

void bsr_transpose(const Bsr& A, Bsr& C, cudaStream_t s) {
  C = Bsr();
  C.nbr = A.nbc; C.nbc = A.nbr; C.br = A.bc; C.bc = A.br;
  DBuf<int> cnt(C.nbr + 1), cursor(C.nbr + 1);
  FSI_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (C.nbr + 1), s));
  FSI_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(int) * (C.nbr + 1), s));
  if (A.nnzb > 0) {
    k_count_cols<<<div_up(A.nnzb, 256), 256, 0, s>>>(A.nnzb, A.colind.p, cnt.p);
    FSI_CHECK_LAUNCH();
  }
  finalize_rowptr(cnt.p, C, s);
  if (A.nnzb == 0) { set_tpr(C); return; }
  DBuf<int> rowof(A.nnzb), tsrc(A.nnzb);
  k_row_of_block<<<div_up(A.nbr, 128), 128, 0, s>>>(A.nbr, A.rowptr.p, rowof.p);
  FSI_CHECK_LAUNCH();
  k_scatter_t<<<div_up(A.nnzb, 256), 256, 0, s>>>(A.nnzb, A.colind.p, rowof.p, C.rowptr.p, cursor.p, C.colind.p,
                                                 tsrc.p);
  FSI_CHECK_LAUNCH();
  k_sort_segments<<<div_up(C.nbr, 128), 128, 0, s>>>(C.nbr, C.rowptr.p, C.colind.p, tsrc.p);
  FSI_CHECK_LAUNCH();
  k_gather_t<<<div_up(A.nnzb, 256), 256, 0, s>>>(A.nnzb, A.br, A.bc, tsrc.p, A.v64.p, C.v64.p);
  FSI_CHECK_LAUNCH();
  set_tpr(C);
}

void bsr_spgemm(const Bsr& A, const Bsr& B, Bsr& C, cudaStream_t s) {
  require(bsr_spgemm_if_fits(A, B, C, s), "bsr_spgemm: a product row has more than 768 block columns");
}

bool bsr_spgemm_if_fits(const Bsr& A, const Bsr& B, Bsr& C, cudaStream_t s) {
  require(A.bc == B.br && A.nbc == B.nbr, "bsr_spgemm: inner dimensions differ");
  C = Bsr();
  C.nbr = A.nbr; C.nbc = B.nbc; C.br = A.br; C.bc = B.bc;
  DBuf<int> cnt(A.nbr > 0 ? A.nbr : 1), overflow(1);
  FSI_CUDA(cudaMemsetAsync(overflow.p, 0, sizeof(int), s));
  const int grid = div_up(A.nbr, kWarpsPerBlock);
  if (A.nbr > 0) {
    k_spgemm_sym<false><<<grid, kWarpsPerBlock * 32, 0, s>>>(A.nbr, A.rowptr.p, A.colind.p, B.rowptr.p, B.colind.p,
                                                            cnt.p, nullptr, nullptr, overflow.p);
    FSI_CHECK_LAUNCH();
  }
  int of = 0;
  FSI_CUDA(cudaMemcpyAsync(&of, overflow.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  if (of) {
    C = Bsr();
    return false;
  }
  finalize_rowptr(cnt.p, C, s);
  if (A.nbr > 0) {
    k_spgemm_sym<true><<<grid, kWarpsPerBlock * 32, 0, s>>>(A.nbr, A.rowptr.p, A.colind.p, B.rowptr.p, B.colind.p,
                                                           nullptr, C.rowptr.p, C.colind.p, overflow.p);
    FSI_CHECK_LAUNCH();
    spgemm_dispatch(A.br, A.bc, B.bc, [&]<int BR, int BK, int BC>() {
      k_spgemm_num<BR, BK, BC><<<grid, 128, 0, s>>>(A.nbr, A.rowptr.p, A.colind.p, A.v64.p, B.rowptr.p, B.colind.p,
                                                    B.v64.p, C.rowptr.p, C.colind.p, C.v64.p);
      FSI_CHECK_LAUNCH();
    });
  }
  set_tpr(C);
  return true;
}

void sort_segments(int nseg, const int* off, int* key, int* pay, cudaStream_t s) {
  if (nseg <= 0) return;
  k_sort_segments<<<div_up(nseg, 128), 128, 0, s>>>(nseg, off, key, pay);
  FSI_CHECK_LAUNCH();
}

void bsr_scale_rows(Bsr& A, const double* w, cudaStream_t s) {
  if (A.nbr == 0) return;
  k_scale_rows<<<div_up(A.nbr, 128), 128, 0, s>>>(A.nbr, A.br, A.bc, A.rowptr.p, A.v64.p, w);
  FSI_CHECK_LAUNCH();
}

void bsr_scale(Bsr& A, double alpha, cudaStream_t s) {
  const int64_t n = A.nnzb * A.br * A.bc;
  if (n == 0) return;
  k_scale_all<<<div_up(n, 256), 256, 0, s>>>(n, alpha, A.v64.p);
  FSI_CHECK_LAUNCH();
}

void bsr_point_diagonal(const Bsr& A, double* diag, cudaStream_t s) {
  require(A.br == A.bc && A.nbr == A.nbc, "point diagonal of a non-square matrix");
  if (A.nbr == 0) return;
  k_point_diag<<<div_up(A.nbr, 128), 128, 0, s>>>(A.nbr, A.br, A.rowptr.p, A.colind.p, A.v64.p, diag);
  FSI_CHECK_LAUNCH();
}

void invert_nonzero(int64_t n, const double* diag, double* dinv, cudaStream_t s) {
  if (n == 0) return;
  k_invert_nonzero<<<div_up(n, 256), 256, 0, s>>>(n, diag, dinv);
  FSI_CHECK_LAUNCH();
}

void bsr_make_fp32(Bsr& A, cudaStream_t s) {
  const int64_t n = A.nnzb * A.br * A.bc;
  A.v32.alloc(n > 0 ? n : 1);
  if (n > 0) {
    if (planar_fp32_shape(A.br, A.bc))
      k_to_f32_planar9<<<div_up(n, 256), 256, 0, s>>>(A.nnzb, A.v64.p, A.v32.p);
    else
      k_to_f32<<<div_up(n, 256), 256, 0, s>>>(n, A.v64.p, A.v32.p);
    FSI_CHECK_LAUNCH();
  }
}

// Largest slice (in blocks, counted from the 8-entry boundary below it) of the CTAs
// that take R consecutive block rows each: the shared-memory size of the staged
// Chebyshev kernel.
__global__ void k_stage_max(int nbr, const int* __restrict__ rp, int R, int* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t r0 = c * R;
  if (r0 >= nbr) return;
  const int64_t r1 = r0 + R < nbr ? r0 + R : nbr;
  atomicMax(out, rp[r1] - (rp[r0] & ~7));
}

void bsr_make_pair_order(Bsr& A1, const Bsr& A2, cudaStream_t s) {
  A1.ord2.release();
  A1.ord2_rp2 = nullptr;
  if (A1.nbr == 0 || A2.nbr != A1.nbr || A1.nbr >= (1 << 24)) return;
  DBuf<int> bad(1);
  FSI_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  A1.ord2.alloc(A1.nbr);
  k_pair_order<<<div_up(A1.nbr, 256), 256, 0, s>>>(A1.nbr, A1.rowptr.p, A2.rowptr.p, A1.ord2.p, bad.p);
  FSI_CHECK_LAUNCH();
  int h = 0;
  FSI_CUDA(cudaMemcpyAsync(&h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  if (h) A1.ord2.release();
  else A1.ord2_rp2 = A2.rowptr.p;
}

bool bsr_make_delta16(Bsr& A, cudaStream_t s) {
  A.cd16.release();
  A.stage_rows = A.stage_max = 0;
  if (A.nbr == 0 || A.nbr != A.nbc || A.nnzb == 0) return false;
  DBuf<int> of(2);
  FSI_CUDA(cudaMemsetAsync(of.p, 0, 2 * sizeof(int), s));
  // 8 spare entries: the staged kernel copies whole 16-byte groups of offsets
  A.cd16.alloc(A.nnzb + 8);
  FSI_CUDA(cudaMemsetAsync(A.cd16.p + A.nnzb, 0, 8 * sizeof(int16_t), s));
  k_delta16<<<div_up(A.nbr, 128), 128, 0, s>>>(A.nbr, A.rowptr.p, A.colind.p, A.cd16.p, of.p);
  FSI_CHECK_LAUNCH();
  const int R = A.br == 2 && A.bc == 2 ? 256 / A.tpr : 0;
  if (R > 0) {
    k_stage_max<<<div_up(div_up(A.nbr, R), 128), 128, 0, s>>>(A.nbr, A.rowptr.p, R, of.p + 1);
    FSI_CHECK_LAUNCH();
  }
  int h[2] = {0, 0};
  FSI_CUDA(cudaMemcpyAsync(h, of.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  if (h[0]) {
    A.cd16.release();
    return false;
  }
  if (R > 0) {
    A.stage_rows = R;
    A.stage_max = h[1];
  }
  return true;
}

void bsr_to_dense(const Bsr& A, double* dense, cudaStream_t s) {
  const int64_t nr = A.rows(), nc = A.cols();
  FSI_CUDA(cudaMemsetAsync(dense, 0, sizeof(double) * nr * nc, s));
  if (A.nbr == 0) return;
  k_to_dense<<<div_up(A.nbr, 128), 128, 0, s>>>(A.nbr, A.br, A.bc, (int)nc, A.rowptr.p, A.colind.p, A.v64.p, dense);
  FSI_CHECK_LAUNCH();
}

bool dense_inverse(int n, double* M, double* Minv, cudaStream_t s) {
  DBuf<int> fail(1);
  FSI_CUDA(cudaMemsetAsync(fail.p, 0, sizeof(int), s));
  DBuf<double> f(n > 0 ? n : 1);      // released after the synchronisation below
  DBuf<unsigned> ticket(1);
  if (n > 0) {
    FSI_CUDA(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned), s));
    const int sms = device_sms();
    k_gj_init<<<std::min(div_up(n, kGjThreads / 32), 4 * sms), kGjThreads, 0, s>>>(n, M, Minv);
    FSI_CHECK_LAUNCH();
    k_gj_first<<<1, kGjThreads, 0, s>>>(n, M, Minv, f.p, fail.p);
    FSI_CHECK_LAUNCH();
    const int grid = std::min(div_up(2 * (int64_t)n * n, kGjThreads), 2 * sms);
    for (int p = 0; p < n; ++p) {
      k_gj_step<<<grid, kGjThreads, 0, s>>>(n, p, M, Minv, f.p, ticket.p, fail.p);
      FSI_CHECK_LAUNCH();
    }
  }
  int failed = 0;
  FSI_CUDA(cudaMemcpyAsync(&failed, fail.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FSI_CUDA(cudaStreamSynchronize(s));
  return failed == 0;
}

}  // namespace fsi

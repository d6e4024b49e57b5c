// Set-up-time sparse kernels: exclusive scans, BSR extraction from the monolithic
// CSR, sparse add, transpose, and the Galerkin SpGEMM.  All are deterministic:
// outputs have sorted block columns and every value is accumulated in a fixed
// order, independent of thread scheduling.
#pragma once
#include "common.cuh"

namespace fsi {

// Non-owning view of a monolithic CSR matrix in device memory.
struct CsrView {
  int64_t n = 0, nnz = 0;
  const int64_t* rowptr = nullptr;
  const int* colind = nullptr;
  const double* vals = nullptr;
};

// Monolithic CSR on the device (what fsi_setup copies in).
struct Csr {
  int64_t n = 0, nnz = 0;
  DBuf<int64_t> rowptr;
  DBuf<int> colind;
  DBuf<double> vals;
  CsrView view() const { return CsrView{n, nnz, rowptr.p, colind.p, vals.p}; }
};

// out[i] = sum_{k<i} in[i] for i <= n (out has n+1 entries); returns the total.
int64_t exclusive_scan(const int* in, int* out, int64_t n, cudaStream_t s);

// BSR block of the monolithic CSR: scalar rows [r0, r0 + nbr*br), scalar columns
// [c0, c0 + nbc*bc), blocks br x bc (column index (c - c0) / bc).
void extract_bsr(const CsrView& A, int64_t r0, int nbr, int br, int64_t c0, int nbc, int bc, Bsr& out,
                 cudaStream_t s);

// C = A + alpha * B (same block shape and dimensions; pattern = union).
void bsr_add(const Bsr& A, const Bsr& B, double alpha, Bsr& C, cudaStream_t s);

// C = A^T (blocks transposed).
void bsr_transpose(const Bsr& A, Bsr& C, cudaStream_t s);

// C = A * B  (A: br x bk blocks, B: bk x bc blocks), FP64 values.  A product row
// may have at most 768 block columns (FSI_EINVAL otherwise).
void bsr_spgemm(const Bsr& A, const Bsr& B, Bsr& C, cudaStream_t s);
// The same, returning false (C left empty) instead when a row has more columns.
bool bsr_spgemm_if_fits(const Bsr& A, const Bsr& B, Bsr& C, cudaStream_t s);

// Scale the scalar rows of A: A[r, :] *= w[r].
void bsr_scale_rows(Bsr& A, const double* w, cudaStream_t s);

// Scale every FP64 value of A by alpha.
void bsr_scale(Bsr& A, double alpha, cudaStream_t s);

// Point diagonal of a square BSR matrix (scalar entry (r, r)); 0 when absent.
void bsr_point_diagonal(const Bsr& A, double* diag, cudaStream_t s);

// dinv = 1/diag where diag != 0, else 0.
void invert_nonzero(int64_t n, const double* diag, double* dinv, cudaStream_t s);

// Sort each segment [off[i], off[i+1]) of key ascending, carrying pay along
// (pay may be null).  Segments are short (set-up use).
void sort_segments(int nseg, const int* off, int* key, int* pay, cudaStream_t s);

// FP32 copy of the values.
void bsr_make_fp32(Bsr& A, cudaStream_t s);
// 16-bit column offsets (block column - block row) of a square matrix, kept only
// when every offset fits in int16; returns whether they were kept.
bool bsr_make_delta16(Bsr& A, cudaStream_t s);
// Slot table of the two-matrix SpMV of A1 with A2 (same block rows), held by A1
// (Bsr::ord2); left empty when a row of A1 has more than 255 blocks.
void bsr_make_pair_order(Bsr& A1, const Bsr& A2, cudaStream_t s);

// Dense row-major copy (n = nbr*br rows, nbc*bc cols) of a BSR matrix.
void bsr_to_dense(const Bsr& A, double* dense, cudaStream_t s);

// Inverse of an n x n row-major dense matrix M into Minv (Gauss-Jordan with partial
// pivoting, one launch per pivot over the whole GPU; M is destroyed); all-zero rows
// are first replaced by identity rows.  Returns false when a pivot vanishes.
bool dense_inverse(int n, double* M, double* Minv, cudaStream_t s);

}  // namespace fsi

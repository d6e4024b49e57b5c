// Vector kernels of the solve path: BLAS-1 updates, precision casts and
// deterministic two-stage reductions (fixed grid, fixed summation order, so a
// result does not depend on scheduling), plus the tall-skinny products of the
// Gram-Schmidt orthogonalisation.
#pragma once
#include "common.cuh"

namespace fsi {

// Partial sums per reduction: a fixed width, independent of the device, so that a
// sum is formed in the same order everywhere (4 CTAs per SM on a 152-SM GB300).
constexpr int kRedBlocks = 608;
constexpr int kRedThreads = 256;

// y = a x + b y  (y not read when b == 0)
template <class T> void axpby(int64_t n, T a, const T* x, T b, T* y, cudaStream_t s);
// z = a x + b y
template <class T> void axpbyz(int64_t n, T a, const T* x, T b, const T* y, T* z, cudaStream_t s);
// y = x * w (elementwise)
template <class T> void vmul(int64_t n, const T* x, const T* w, T* y, cudaStream_t s);
// y += w * x (elementwise)
template <class T> void vfma(int64_t n, const T* w, const T* x, T* y, cudaStream_t s);
// y = (To) x
template <class Ti, class To> void cast(int64_t n, const Ti* x, To* y, cudaStream_t s);
// out[0] = sum_i x_i y_i (FP64 accumulation), device result; partials has kRedBlocks doubles
template <class T> void dot_dev(int64_t n, const T* x, const T* y, double* partials, double* out, cudaStream_t s);
// host convenience: synchronous dot
template <class T> double dot_host(int64_t n, const T* x, const T* y, double* partials, double* out, cudaStream_t s);

// Gram-Schmidt pieces.  V holds basis vectors of length n with leading dimension
// ldv (vector i at V + i*ldv); the number of active vectors is read on the
// device from *jcount (+ joff), so a captured graph can be replayed for every j.
// h[i] = <V_i, w>, i < *jcount + joff.  With skip != nullptr and *skip != 0 (read on
// the device) the products are not formed and h[i] = 0.
void mdot(int64_t n, const double* V, int64_t ldv, const int* jcount, int joff, const double* w, double* partials,
          double* h, int maxcols, cudaStream_t s, const int* skip = nullptr);
// w -= sign * sum_i h[i] V_i; if nrm_partials != nullptr also writes per-block sums of w^2.
// maxcols bounds the number of vectors (*jcount + joff) for the shared-memory copy
// of h (0: unknown, the unvectorised kernel runs).  Both multi-products use 16-byte
// loads when V's columns and w are 16-byte aligned (ldv even).  With *skip != 0
// nothing is written (w and the partial sums keep their values).
void maxpy(int64_t n, const double* V, int64_t ldv, const int* jcount, int joff, const double* h, double sign,
           double* w, double* nrm_partials, int maxcols, cudaStream_t s, const int* skip = nullptr);
// out = sqrt(sum partials)
void finish_norm(const double* partials, double* out, cudaStream_t s);
// Arnoldi defect: w = V_j - w (j = *jcount), partials = per-block sums of w^2.
void arnoldi_defect(int64_t n, const double* V, int64_t ldv, const int* jcount, double* w, double* partials,
                    cudaStream_t s);
// Second-pass test of Gram-Schmidt (kRedBlocks partial sums of squares of the vector
// after and before one pass): flag[0] = 0 when sum(after) < eta^2 sum(before) (a second
// pass is needed), else 1 (the skip flag of that pass); flag[1] += 1 - flag[0].
void reorth_flag(const double* after, const double* before, double eta, int* flag, cudaStream_t s);

}  // namespace fsi

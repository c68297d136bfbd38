// Dense FP64 linear-algebra launchers used by the SCF driver.
#pragma once
#include <cuda_runtime.h>

namespace hf {

int gemm(int M, int N, int K, double alpha, const double* A, int lda, bool ta, const double* B, int ldb, bool tb,
         double beta, double* C, int ldc, cudaStream_t s);
// Eigen-decomposition of a symmetric n x n matrix by parallel cyclic Jacobi.
// w[ncols]: lowest ncols eigenvalues ascending; Vout[n x ncols] the matching
// eigenvectors as columns.  work: >= 3 m^2 + 514 + m_pad doubles, iwork: >= m_pad
// ints (m = n rounded up to even, m_pad = next power of two >= m).
// Returns 0 converged, 1 not converged within max_sweeps, -1 CUDA error.
int jacobi_eigh(int n, const double* A, double* w, double* Vout, int ncols, double* work, int* iwork, int max_sweeps,
                double tol, int* sweeps_done, cudaStream_t s);
size_t jacobi_work_doubles(int n);
size_t jacobi_work_ints(int n);
int antisym(int n, const double* A, double* E, cudaStream_t s);
int dots(long long len, const double* X, const double* const* Ys_dev, int nk, double* part, double* out,
         cudaStream_t s);
int diis_solve(int m, const double* B, double* coef, int* status, cudaStream_t s);
int lincomb(long long len, int nk, const double* const* Xs_dev, const double* coef, double* out, cudaStream_t s);
int rms_diff(long long len, const double* A, const double* B, double* part, double* out, cudaStream_t s);
int scale_cols(int n, int ncols, const double* U, const double* s, double power, double drop_below, double* out,
               cudaStream_t st);

}  // namespace hf

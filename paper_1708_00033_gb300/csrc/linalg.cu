// Dense FP64 linear algebra of the SCF cycle (Section 3: diagonalise the Fock
// matrix in an orthogonal basis, form the new density):
//   - tiled SIMT FP64 GEMM  C = alpha op(A) op(B) + beta C  (row-major);
//   - parallel cyclic Jacobi eigensolver for symmetric matrices: each round
//     applies N/2 disjoint plane rotations chosen by the round-robin
//     ("circle") ordering, every 2x2 block of A' = J^T A J and every row pair
//     of V' = V J being independent; one launch per round, ping-pong buffers;
//   - small helpers (antisymmetric part, dot products, linear combinations,
//     RMS difference, the Pulay DIIS system solved on the device).
#include <math.h>

#include "linalg.cuh"

namespace hf {

// ------------------------------------------------------------------ GEMM --
constexpr int kTM = 64, kTN = 64, kTK = 16;

// C[M x N] = alpha * op(A)[M x K] * op(B)[K x N] + beta * C, all row-major.
// op(A) = A (lda >= K) or A^T (A stored K x M, lda >= M); same for B.
__global__ void __launch_bounds__(256) k_gemm_f64(int M, int N, int K, double alpha, const double* __restrict__ A,
                                                  int lda, int ta, const double* __restrict__ B, int ldb, int tb,
                                                  double beta, double* __restrict__ C, int ldc)
{
    __shared__ double As[kTK][kTM + 1];
    __shared__ double Bs[kTK][kTN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += kTK) {
        // load As[k][m] = op(A)[m0+m][k0+k]
        for (int e = threadIdx.x; e < kTK * kTM; e += 256) {
            int k, m;
            if (ta) {  // A stored K x M: contiguous in m
                k = e / kTM;
                m = e % kTM;
            } else {  // A stored M x K: contiguous in k
                m = e / kTK;
                k = e % kTK;
            }
            const int gm = m0 + m, gk = k0 + k;
            double v = 0.0;
            if (gm < M && gk < K) v = ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            As[k][m] = v;
        }
        for (int e = threadIdx.x; e < kTK * kTN; e += 256) {
            int k, n;
            if (tb) {  // B stored N x K
                n = e / kTK;
                k = e % kTK;
            } else {  // B stored K x N
                k = e / kTN;
                n = e % kTN;
            }
            const int gn = n0 + n, gk = k0 + k;
            double v = 0.0;
            if (gn < N && gk < K) v = tb ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
            Bs[k][n] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kTK; k++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            double* c = C + (size_t)gm * ldc + gn;
            *c = alpha * acc[i][j] + (beta == 0.0 ? 0.0 : beta * *c);
        }
    }
}

int gemm(int M, int N, int K, double alpha, const double* A, int lda, bool ta, const double* B, int ldb, bool tb,
         double beta, double* C, int ldc, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return 0;
    dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM);
    k_gemm_f64<<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, ta ? 1 : 0, B, ldb, tb ? 1 : 0, beta, C, ldc);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------- Jacobi --
// Round-robin pairing of n (even) indices, round r in [0, n-1), pair k in [0, n/2).
__device__ __forceinline__ void rr_pair(int n, int r, int k, int& p, int& q)
{
    const int m = n - 1;
    if (k == 0) {
        p = m;
        q = r;
    } else {
        p = (r + k) % m;
        q = (r - k + m) % m;
    }
}

// Rotation zeroing A_pq: t = sgn(th) / (|th| + sqrt(1 + th^2)), th = (A_qq - A_pp) / (2 A_pq).
__device__ __forceinline__ void jacobi_cs(const double* __restrict__ A, int n, int p, int q, double& c, double& s)
{
    const double apq = A[(size_t)p * n + q];
    if (apq == 0.0) {
        c = 1.0;
        s = 0.0;
        return;
    }
    const double th = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
    const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
    c = 1.0 / sqrt(1.0 + t * t);
    s = t * c;
}

// Rotations of one round: pair k -> (p, q, c, s), from the matrix at the start of the round.
struct Rot {
    int p, q;
    double c, s;
};

__global__ void k_jacobi_rot(int n, int r, const double* __restrict__ A, Rot* __restrict__ rot)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n / 2) return;
    Rot o;
    rr_pair(n, r, k, o.p, o.q);
    jacobi_cs(A, n, o.p, o.q, o.c, o.s);
    rot[k] = o;
}

// One round: thread (kr, kc) transforms the 2x2 block of rows (p_r, q_r) and
// columns (p_c, q_c) of A into Anew, and the entries (p_r|q_r, p_c|q_c) of V.
__global__ void k_jacobi_round(int n, const Rot* __restrict__ rot, const double* __restrict__ A,
                               double* __restrict__ Anew, double* __restrict__ V)
{
    const int half = n / 2;
    const int kc = blockIdx.x * blockDim.x + threadIdx.x;
    const int kr = blockIdx.y;
    if (kc >= half || kr >= half) return;
    const Rot R = rot[kr], C = rot[kc];
    const int pr = R.p, qr = R.q, pc = C.p, qc = C.q;
    const double cr = R.c, sr = R.s, cc = C.c, sc = C.s;
    const double a = A[(size_t)pr * n + pc], b = A[(size_t)pr * n + qc];
    const double c = A[(size_t)qr * n + pc], d = A[(size_t)qr * n + qc];
    // columns: A J_c
    const double a1 = cc * a - sc * b, b1 = sc * a + cc * b;
    const double c1 = cc * c - sc * d, d1 = sc * c + cc * d;
    // rows: J_r^T (A J_c)
    Anew[(size_t)pr * n + pc] = cr * a1 - sr * c1;
    Anew[(size_t)qr * n + pc] = sr * a1 + cr * c1;
    Anew[(size_t)pr * n + qc] = cr * b1 - sr * d1;
    Anew[(size_t)qr * n + qc] = sr * b1 + cr * d1;
    // V J_c on rows pr and qr
    const double vp0 = V[(size_t)pr * n + pc], vq0 = V[(size_t)pr * n + qc];
    V[(size_t)pr * n + pc] = cc * vp0 - sc * vq0;
    V[(size_t)pr * n + qc] = sc * vp0 + cc * vq0;
    const double vp1 = V[(size_t)qr * n + pc], vq1 = V[(size_t)qr * n + qc];
    V[(size_t)qr * n + pc] = cc * vp1 - sc * vq1;
    V[(size_t)qr * n + qc] = sc * vp1 + cc * vq1;
}

// sum of squares of the off-diagonal and of all entries (two partial arrays)
__global__ void k_offdiag(int n, const double* __restrict__ A, double* __restrict__ part)
{
    __shared__ double so[256], sa[256];
    double o = 0.0, t = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const double v = A[e];
        t += v * v;
        if (e / n != e % n) o += v * v;
    }
    so[threadIdx.x] = o;
    sa[threadIdx.x] = t;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            so[threadIdx.x] += so[threadIdx.x + s];
            sa[threadIdx.x] += sa[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = so[0];
        part[gridDim.x + blockIdx.x] = sa[0];
    }
}

__global__ void k_sum2(int nb, const double* __restrict__ part, double* __restrict__ out)
{
    __shared__ double s0[256], s1[256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += part[i];
        b += part[nb + i];
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            s0[threadIdx.x] += s0[threadIdx.x + s];
            s1[threadIdx.x] += s1[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s0[0];
        out[1] = s1[0];
    }
}

// pad an n x n symmetric matrix to m x m (m = n or n + 1); identity for V
__global__ void k_jacobi_init(int n, int m, const double* __restrict__ src, double* __restrict__ A,
                              double* __restrict__ V, double pad_value)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)m * m) return;
    const int i = (int)(e / m), j = (int)(e % m);
    double v;
    if (i < n && j < n)
        v = 0.5 * (src[(size_t)i * n + j] + src[(size_t)j * n + i]);
    else
        v = (i == j) ? pad_value : 0.0;
    A[e] = v;
    V[e] = (i == j) ? 1.0 : 0.0;
}

// eigenvalues -> sort keys (ascending eigenvalue, then index)
__global__ void k_diag_keys(int m, const double* __restrict__ A, double* __restrict__ key, int* __restrict__ val,
                            int m_pad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m_pad) return;
    if (i < m) {
        key[i] = -A[(size_t)i * m + i];  // descending sort of -lambda = ascending lambda
        val[i] = i;
    } else {
        key[i] = -INFINITY;
        val[i] = 0x7fffffff;
    }
}

// w[j] = lambda of sorted column j; Vout[:, j] = V[:n, perm[j]] for j < ncols
__global__ void k_gather_eig(int n, int m, int ncols, const double* __restrict__ A, const double* __restrict__ V,
                             const int* __restrict__ perm, double* __restrict__ w, double* __restrict__ Vout)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * ncols) return;
    const int i = (int)(e / ncols), j = (int)(e % ncols);
    const int src = perm[j];
    Vout[e] = V[(size_t)i * m + src];
    if (i == 0 && w) w[j] = A[(size_t)src * m + src];
}

int bitonic_sort_desc(double* key, int* val, int n, int n_pad, cudaStream_t s);

// remove value x from perm[0..m) keeping order (single thread; m small enough)
__global__ void k_drop_index(int m, int* perm, int x)
{
    int o = 0;
    for (int i = 0; i < m; i++)
        if (perm[i] != x) perm[o++] = perm[i];
}


int jacobi_eigh(int n, const double* Ain, double* w, double* Vout, int ncols, double* work, int* iwork, int max_sweeps,
                double tol, int* sweeps_done, cudaStream_t s)
{
    // work: 3 m^2 + 2*256 + 2 doubles + m_pad keys; iwork: m_pad ints
    const int m = n + (n & 1);
    if (n <= 0) return 0;
    double* A0 = work;
    double* A1 = A0 + (size_t)m * m;
    double* V = A1 + (size_t)m * m;
    double* part = V + (size_t)m * m;
    double* res = part + 512;
    double* key = res + 2;
    Rot* rot = (Rot*)key;  // m/2 rotations (12 m bytes) in the key area, which the final sort reuses
    // padding eigenvalue: far above the spectrum bound (Gershgorin of |A| <= n max|A|) is not known here;
    // a zero-coupled padding entry only needs to be distinct and is dropped from the output.
    k_jacobi_init<<<(unsigned)(((long long)m * m + 255) / 256), 256, 0, s>>>(n, m, Ain, A0, V, 0.0);
    double* cur = A0;
    double* nxt = A1;
    int sweep = 0;
    double h[2];
    for (sweep = 0; sweep < max_sweeps; sweep++) {
        k_offdiag<<<256, 256, 0, s>>>(m, cur, part);
        k_sum2<<<1, 256, 0, s>>>(256, part, res);
        if (cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
        if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
        if (h[0] <= tol * tol * h[1] || h[0] == 0.0) break;
        for (int r = 0; r < m - 1; r++) {
            // every entry of Anew belongs to exactly one (row pair, column pair) block of this round
            k_jacobi_rot<<<(m / 2 + 127) / 128, 128, 0, s>>>(m, r, cur, rot);
            dim3 grid((m / 2 + 127) / 128, m / 2);
            k_jacobi_round<<<grid, 128, 0, s>>>(m, rot, cur, nxt, V);
            double* t = cur;
            cur = nxt;
            nxt = t;
        }
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    if (sweeps_done) *sweeps_done = sweep;
    size_t mp = 1;
    while (mp < (size_t)m) mp <<= 1;
    k_diag_keys<<<(unsigned)((mp + 255) / 256), 256, 0, s>>>(m, cur, key, iwork, (int)mp);
    if (bitonic_sort_desc(key, iwork, (int)mp, (int)mp, s) != 0) return -1;
    // when n is odd the padding index m-1 carries eigenvalue 0 and must be skipped: drop it from perm
    if (n != m) {
        k_drop_index<<<1, 1, 0, s>>>(m, iwork, m - 1);
    }
    const long long tot = (long long)n * ncols;
    k_gather_eig<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, m, ncols, cur, V, iwork, w, Vout);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return sweep >= max_sweeps ? 1 : 0;
}

// ---------------------------------------------------------------- helpers --
__global__ void k_antisym(int n, const double* __restrict__ A, double* __restrict__ E)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    const int i = (int)(e / n), j = (int)(e % n);
    E[e] = A[e] - A[(size_t)j * n + i];
}

int antisym(int n, const double* A, double* E, cudaStream_t s)
{
    k_antisym<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, s>>>(n, A, E);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// out[k] = <X, Y_k> for k < nk (Y_k = Ys[k]); partial sums in part[nk][256]
__global__ void k_dots(long long len, const double* __restrict__ X, const double* const* __restrict__ Ys,
                       double* __restrict__ part)
{
    __shared__ double sm[256];
    const double* Y = Ys[blockIdx.y];
    double acc = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
        acc += X[e] * Y[e];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = sm[0];
}

__global__ void k_dots_final(int nk, int nb, const double* __restrict__ part, double* __restrict__ out)
{
    const int k = blockIdx.x;
    __shared__ double sm[256];
    double a = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += part[k * nb + i];
    sm[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && k < nk) out[k] = sm[0];
}

int dots(long long len, const double* X, const double* const* Ys_dev, int nk, double* part, double* out,
         cudaStream_t s)
{
    dim3 grid(128, nk);
    k_dots<<<grid, 256, 0, s>>>(len, X, Ys_dev, part);
    k_dots_final<<<nk, 256, 0, s>>>(nk, 128, part, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Pulay DIIS: B[m x m] (Gram of error vectors) -> solve [B -1; -1 0][c; l] = [0; -1]
// by Gaussian elimination with partial pivoting (one thread, m <= 16).
// status: 0 ok, 1 singular.
__global__ void k_diis_solve(int m, const double* __restrict__ B, double* __restrict__ coef, int* __restrict__ status)
{
    double a[17][18];
    const int n = m + 1;
    for (int i = 0; i < m; i++) {
        for (int j = 0; j < m; j++) a[i][j] = B[i * m + j];
        a[i][m] = -1.0;
        a[i][n] = 0.0;
    }
    for (int j = 0; j < m; j++) a[m][j] = -1.0;
    a[m][m] = 0.0;
    a[m][n] = -1.0;
    // scale rows of the Gram block by its largest diagonal to keep pivots moderate
    double dmax = 0.0;
    for (int i = 0; i < m; i++) dmax = fmax(dmax, fabs(a[i][i]));
    if (dmax > 0.0)
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++) a[i][j] /= dmax;
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (fabs(a[piv][c]) < 1e-300) {
            *status = 1;
            return;
        }
        if (piv != c)
            for (int k = 0; k <= n; k++) {
                const double t = a[c][k];
                a[c][k] = a[piv][k];
                a[piv][k] = t;
            }
        for (int r = c + 1; r < n; r++) {
            const double f = a[r][c] / a[c][c];
            for (int k = c; k <= n; k++) a[r][k] -= f * a[c][k];
        }
    }
    double x[17];
    for (int r = n - 1; r >= 0; r--) {
        double v = a[r][n];
        for (int k = r + 1; k < n; k++) v -= a[r][k] * x[k];
        x[r] = v / a[r][r];
    }
    for (int i = 0; i < m; i++) coef[i] = x[i];
    *status = 0;
}

int diis_solve(int m, const double* B, double* coef, int* status, cudaStream_t s)
{
    k_diis_solve<<<1, 1, 0, s>>>(m, B, coef, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// out = sum_k coef[k] * Xs[k]
__global__ void k_lincomb(long long len, int nk, const double* const* __restrict__ Xs, const double* __restrict__ coef,
                          double* __restrict__ out)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    double v = 0.0;
    for (int k = 0; k < nk; k++) v += coef[k] * Xs[k][e];
    out[e] = v;
}

int lincomb(long long len, int nk, const double* const* Xs_dev, const double* coef, double* out, cudaStream_t s)
{
    k_lincomb<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, nk, Xs_dev, coef, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// RMS of A - B into out[0] (partials in part[256])
__global__ void k_sqdiff(long long len, const double* __restrict__ A, const double* __restrict__ B,
                         double* __restrict__ part)
{
    __shared__ double sm[256];
    double acc = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
        const double d = A[e] - B[e];
        acc += d * d;
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_rms_final(long long len, const double* __restrict__ part, double* __restrict__ out)
{
    __shared__ double sm[256];
    sm[threadIdx.x] = part[threadIdx.x];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sqrt(sm[0] / (double)len);
}

int rms_diff(long long len, const double* A, const double* B, double* part, double* out, cudaStream_t s)
{
    k_sqdiff<<<256, 256, 0, s>>>(len, A, B, part);
    k_rms_final<<<1, 256, 0, s>>>(len, part, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// X = U diag(f(s)) U^T helper: Us[:, j] = U[:, j] * scale(s_j), zero for dropped vectors
__global__ void k_scale_cols(int n, int ncols, const double* __restrict__ U, const double* __restrict__ s,
                             double power, double drop_below, double* __restrict__ out)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * ncols) return;
    const int j = (int)(e % ncols);
    const double sj = s[j];
    out[e] = sj > drop_below ? U[e] * pow(sj, power) : 0.0;
}

int scale_cols(int n, int ncols, const double* U, const double* s, double power, double drop_below, double* out,
               cudaStream_t st)
{
    k_scale_cols<<<(unsigned)(((long long)n * ncols + 255) / 256), 256, 0, st>>>(n, ncols, U, s, power, drop_below, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hf

namespace hf {
size_t jacobi_work_doubles(int n)
{
    const size_t m = (size_t)(n + (n & 1));
    size_t mp = 1;
    while (mp < m) mp <<= 1;
    return 3 * m * m + 514 + mp + 2 * m;
}
size_t jacobi_work_ints(int n)
{
    const size_t m = (size_t)(n + (n & 1));
    size_t mp = 1;
    while (mp < m) mp <<= 1;
    return mp;
}
}  // namespace hf

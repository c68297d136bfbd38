// Fock-matrix assembly around the ERI kernels (the 2e-Fock reduction and
// flush of Algorithms 1-3, ddi_gsumf + buffer flushes):
//   P' = n P n             density in the library's raw component normalisation
//                          (n = Cartesian component factors), with a finiteness
//                          and symmetry check of P;
//   J = n (Jt + Jt^T) n / 2, K = n (Kt + Kt^T) n / 2, F = H + J - K/2;
//   E_elec = 1/2 sum P (H + F), reduced in a fixed order.
#include <math.h>

#include <algorithm>

#include "eri_common.cuh"
#include "setup.cuh"

namespace hf {

__global__ void k_scale_density(int N, const double* __restrict__ P, const double* __restrict__ n,
                                double* __restrict__ P64, float* __restrict__ P32, int* __restrict__ bad)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * N) return;
    const int i = (int)(t / N), j = (int)(t % N);
    const double v = P[t], w = P[(size_t)j * N + i];
    if (!isfinite(v) || fabs(v - w) > 1e-12 * fmax(1.0, fabs(v))) atomicOr(bad, 1);
    const double s = n[i] * n[j] * v;
    P64[t] = s;
    if (P32) P32[t] = (float)s;
}

__global__ void k_assemble(int N, const double* __restrict__ Jt, const double* __restrict__ Kt,
                           const double* __restrict__ n, const double* __restrict__ H, double* __restrict__ J,
                           double* __restrict__ K, double* __restrict__ F, const int* __restrict__ bad)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * N || (bad && *bad)) return;
    const int i = (int)(t / N), j = (int)(t % N);
    const size_t tt = (size_t)j * N + i;
    const double s = 0.5 * n[i] * n[j];
    const double jv = s * (Jt[t] + Jt[tt]);
    const double kv = s * (Kt[t] + Kt[tt]);
    if (J) J[t] = jv;
    if (K) K[t] = kv;
    if (F) F[t] = H[t] + jv - 0.5 * kv;
}

__global__ void k_energy_partial(long long n, const double* __restrict__ P, const double* __restrict__ H,
                                 const double* __restrict__ F, double* __restrict__ partial)
{
    __shared__ double sm[256];
    double e = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        e += P[t] * (H[t] + F[t]);
    sm[threadIdx.x] = e;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

__global__ void k_energy_final(int nb, const double* __restrict__ partial, double* __restrict__ out)
{
    __shared__ double sm[256];
    double e = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) e += partial[b];
    sm[threadIdx.x] = e;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = 0.5 * sm[0];
}

// dsh[i][j] = max |P_mu nu| over the (i, j) shell block
__global__ void k_shell_block_max(int n_sh, int N, const int* __restrict__ l, const int* __restrict__ bf0,
                                  const double* __restrict__ P, float* __restrict__ dsh)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_sh * n_sh) return;
    const int i = (int)(t / n_sh), j = (int)(t % n_sh);
    const int ni = (l[i] + 1) * (l[i] + 2) / 2, nj = (l[j] + 1) * (l[j] + 2) / 2;
    double m = 0.0;
    for (int a = 0; a < ni; a++)
        for (int b = 0; b < nj; b++) m = fmax(m, fabs(P[(size_t)(bf0[i] + a) * N + bf0[j] + b]));
    dsh[t] = (float)m;
}

int launch_shell_block_max(int n_sh, int N, const int* l, const int* bf0, const double* P, float* dsh, cudaStream_t s)
{
    const long long n = (long long)n_sh * n_sh;
    if (n > 0) k_shell_block_max<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n_sh, N, l, bf0, P, dsh);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// C = A + alpha * B (N x N)
__global__ void k_axpby(long long n, const double* __restrict__ A, double alpha, const double* __restrict__ B,
                        double* __restrict__ C)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) C[t] = A[t] + alpha * B[t];
}

int launch_axpby(long long n, const double* A, double alpha, const double* B, double* C, cudaStream_t s)
{
    if (n > 0) k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, A, alpha, B, C);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// out[t] = sum over the copies of in[c * NN + t]: the reduction of per-block accumulator copies
__global__ void k_sum_copies(int n_copies, long long nn, const double* __restrict__ in, double* __restrict__ out)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < n_copies; c++) s += in[(size_t)c * nn + t];
        out[t] = s;
    }
}

int launch_sum_copies(int n_copies, long long nn, const double* in, double* out, int num_sms, cudaStream_t s)
{
    if (nn > 0) {
        const long long blocks = std::min<long long>((nn + 255) / 256, (long long)num_sms * 8);
        k_sum_copies<<<(unsigned)blocks, 256, 0, s>>>(n_copies, nn, in, out);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_scale_density(int N, const double* P, const double* comp_norm, double* P64, float* P32, int* bad,
                         cudaStream_t s)
{
    const long long n = (long long)N * N;
    if (n > 0) k_scale_density<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(N, P, comp_norm, P64, P32, bad);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_assemble(int N, const double* Jt, const double* Kt, const double* comp_norm, const double* H, double* J,
                    double* K, double* F, const int* bad, cudaStream_t s)
{
    const long long n = (long long)N * N;
    if (n > 0) k_assemble<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(N, Jt, Kt, comp_norm, H, J, K, F, bad);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// F = H + J - K/2 from already symmetrised J and K (the assembly of a sharded build after the sum over
// shards); *bad is set when J or K holds a non-finite value.
__global__ void k_fock_from_jk(long long n, const double* __restrict__ H, const double* __restrict__ J,
                               const double* __restrict__ K, double* __restrict__ F, int* __restrict__ bad)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double j = J[t], k = K[t];
    if (!isfinite(j) || !isfinite(k)) atomicOr(bad, 1);
    F[t] = H[t] + j - 0.5 * k;
}

int launch_fock_from_jk(long long n, const double* H, const double* J, const double* K, double* F, int* bad,
                        cudaStream_t s)
{
    if (n > 0) k_fock_from_jk<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, H, J, K, F, bad);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// partial must hold 256 doubles
int launch_energy(int N, const double* P, const double* H, const double* F, double* partial, double* out,
                  cudaStream_t s)
{
    k_energy_partial<<<256, 256, 0, s>>>((long long)N * N, P, H, F, partial);
    k_energy_final<<<1, 256, 0, s>>>(256, partial, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hf

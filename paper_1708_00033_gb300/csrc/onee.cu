// One-electron part of the Fock matrix (Section 3: the O(N^2) term, computed
// once per geometry): overlap S, kinetic T and nuclear attraction V, H = T + V,
// and the nuclear repulsion energy.
//
//   S: Obara-Saika 1-D recurrence s_{i+1,j} = PA s_ij + (i s_{i-1,j} + j s_{i,j-1}) / 2p
//      (and the same with PB on the second index), s_00 = sqrt(pi/p) exp(-mu X_AB^2);
//   T: one half of the gradient overlap, per direction
//      t_ij = (i j s_{i-1,j-1} - 2b i s_{i-1,j+1} - 2a j s_{i+1,j-1} + 4ab s_{i+1,j+1}) / 2;
//   V: Obara-Saika auxiliaries [e|0]^(m) with [0|0]^(m) = 2pi/p K F_m(p |PC|^2),
//      [e+1_i]^(m) = PA_i [e]^(m) - PC_i [e]^(m+1) + e_i/2p ([e-1_i]^(m) - [e-1_i]^(m+1)),
//      then the binomial shift (a|b) = sum_k C(b,k) AB^(b-k) (a+k|0) per direction.
#include <math.h>

#include "eri_common.cuh"
#include "setup.cuh"

namespace hf {

namespace {

__device__ __forceinline__ int ncomp(int l) { return (l + 1) * (l + 2) / 2; }

__device__ __forceinline__ void comp_pow(int l, int c, int& x, int& y, int& z)
{
    int k = 0;
    for (int a = l; a >= 0; a--)
        for (int b = l - a; b >= 0; b--) {
            if (k == c) {
                x = a;
                y = b;
                z = l - a - b;
                return;
            }
            k++;
        }
    x = y = z = 0;
}

// position of the exponent triple e = (x, y, z), |e| = t <= 4, in a packed list ordered by |e|,
// then by x descending, then by y descending (35 entries for |e| <= 4)
__device__ __forceinline__ int eidx(int x, int y, int z)
{
    const int t = x + y + z, r = t - x;
    return t * (t + 1) * (t + 2) / 6 + r * (r + 1) / 2 + z;
}

__device__ __forceinline__ double binom(int n, int k)
{
    return (n == 2 && k == 1) ? 2.0 : 1.0;  // n <= 2
}

}  // namespace

// one thread per unordered shell pair (i >= j); writes the (i, j) block of S
// and H and its transpose.  Primitive pairs whose Gaussian-product factor
// exp(-ab/(a+b) |AB|^2) is below exp(-60) ~ 9e-27 are skipped: with
// normalised coefficients below 1e3, 2 pi / p below 30, a total nuclear
// charge below 1e5 and polynomial factors below 1e6 their contribution to
// any element stays below 1e-12 of the 1e-11 parity tolerance.
__global__ void k_one_electron(int n_sh, int n_atoms, int N, const int* __restrict__ l, const int* __restrict__ atom,
                               const int* __restrict__ bf0, const int* __restrict__ nprim,
                               const int* __restrict__ prim0, const double* __restrict__ exps,
                               const double* __restrict__ cn, const double* __restrict__ xyz,
                               const double* __restrict__ Z, const double* __restrict__ comp_norm,
                               const double* __restrict__ boys64, double* __restrict__ S, double* __restrict__ H)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_sh * (n_sh + 1) / 2) return;
    long long ii = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (ii * (ii + 1) / 2 > t) ii--;
    while ((ii + 1) * (ii + 2) / 2 <= t) ii++;
    const int i = (int)ii, j = (int)(t - ii * (ii + 1) / 2);
    const int la = l[i], lb = l[j];
    const int na = ncomp(la), nb = ncomp(lb);
    const double A[3] = {xyz[3 * atom[i]], xyz[3 * atom[i] + 1], xyz[3 * atom[i] + 2]};
    const double B[3] = {xyz[3 * atom[j]], xyz[3 * atom[j] + 1], xyz[3 * atom[j] + 2]};
    double sblk[36], hblk[36];
    for (int c = 0; c < 36; c++) sblk[c] = hblk[c] = 0.0;
    const int Lab = la + lb;
    for (int ka = 0; ka < nprim[i]; ka++)
        for (int kb = 0; kb < nprim[j]; kb++) {
            const double a = exps[prim0[i] + ka], b = exps[prim0[j] + kb];
            const double cc = cn[prim0[i] + ka] * cn[prim0[j] + kb];
            const double p = a + b, mu = a * b / p, o2p = 0.5 / p;
            const double R2ab = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) +
                                (A[2] - B[2]) * (A[2] - B[2]);
            if (mu * R2ab > 60.0) continue;
            double P[3], PA[3], PB[3];
            double s[3][4][4];  // s[dir][i][j], i <= la+1, j <= lb+1
            for (int d = 0; d < 3; d++) {
                P[d] = (a * A[d] + b * B[d]) / p;
                PA[d] = P[d] - A[d];
                PB[d] = P[d] - B[d];
                const double X = A[d] - B[d];
                for (int u = 0; u < 4; u++)
                    for (int v = 0; v < 4; v++) s[d][u][v] = 0.0;
                s[d][0][0] = sqrt(M_PI / p) * exp(-mu * X * X);
                for (int u = 0; u <= la + 1; u++)
                    for (int v = 0; v <= lb + 1; v++) {
                        if (u == 0 && v == 0) continue;
                        if (u > 0)
                            s[d][u][v] = PA[d] * s[d][u - 1][v] +
                                         o2p * ((u - 1) * (u >= 2 ? s[d][u - 2][v] : 0.0) + v * (v >= 1 ? s[d][u - 1][v - 1] : 0.0));
                        else
                            s[d][u][v] = PB[d] * s[d][u][v - 1] + o2p * (v - 1) * (v >= 2 ? s[d][u][v - 2] : 0.0);
                    }
            }
            // nuclear-attraction auxiliaries [e|0]^(m), e up to Lab (<= 4), m up to Lab; their m = 0
            // level, weighted by the nuclear charges, is summed over the nuclei first, and the
            // binomial shift to (a|b) (linear in [e|0]) is applied once per primitive pair
            double ts[35];  // sum over nuclei of Z_C [e|0]^(0), packed by eidx
            for (int c = 0; c < 35; c++) ts[c] = 0.0;
            const double K = exp(-mu * R2ab);
            const double pre = 2.0 * M_PI / p * K;
            for (int nuc = 0; nuc < n_atoms; nuc++) {
                const double PC[3] = {P[0] - xyz[3 * nuc], P[1] - xyz[3 * nuc + 1], P[2] - xyz[3 * nuc + 2]};
                double F[5];
                boys_eval<4>(p * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]), boys64, F);
                // th[m][eidx(e)], |e| <= Lab - m
                double th[5][35];
                for (int m = 0; m <= Lab; m++) th[m][0] = pre * F[m];
                for (int tot = 1; tot <= Lab; tot++)
                    for (int m = 0; m <= Lab - tot; m++)
                        for (int x = tot; x >= 0; x--)
                            for (int y = tot - x; y >= 0; y--) {
                                const int z = tot - x - y;
                                int e[3] = {x, y, z};
                                const int d = x > 0 ? 0 : (y > 0 ? 1 : 2);
                                int e1[3] = {x, y, z};
                                e1[d]--;
                                const int i1 = eidx(e1[0], e1[1], e1[2]);
                                double v = PA[d] * th[m][i1] - PC[d] * th[m + 1][i1];
                                if (e1[d] > 0) {
                                    int e2[3] = {e1[0], e1[1], e1[2]};
                                    e2[d]--;
                                    const int i2 = eidx(e2[0], e2[1], e2[2]);
                                    v += e1[d] * o2p * (th[m][i2] - th[m + 1][i2]);
                                }
                                th[m][eidx(e[0], e[1], e[2])] = v;
                            }
                const double zc = Z[nuc];
                const int ne = (Lab + 1) * (Lab + 2) * (Lab + 3) / 6;
                for (int c = 0; c < ne; c++) ts[c] += zc * th[0][c];
            }
            // (a|b) = sum_k C(b,k) (A-B)^(b-k) [a+k|0] per direction
            double ABp[3][3];
            for (int d = 0; d < 3; d++) {
                ABp[d][0] = 1.0;
                ABp[d][1] = A[d] - B[d];
                ABp[d][2] = ABp[d][1] * ABp[d][1];
            }
            double V[36];  // (a|b) for this primitive pair, summed over nuclei
            for (int ca = 0; ca < na; ca++) {
                int ax, ay, az;
                comp_pow(la, ca, ax, ay, az);
                for (int cb = 0; cb < nb; cb++) {
                    int bx, by, bz;
                    comp_pow(lb, cb, bx, by, bz);
                    double acc = 0.0;
                    for (int kx = 0; kx <= bx; kx++)
                        for (int ky = 0; ky <= by; ky++)
                            for (int kz = 0; kz <= bz; kz++) {
                                const double w = binom(bx, kx) * binom(by, ky) * binom(bz, kz) * ABp[0][bx - kx] *
                                                 ABp[1][by - ky] * ABp[2][bz - kz];
                                acc += w * ts[eidx(ax + kx, ay + ky, az + kz)];
                            }
                    V[ca * nb + cb] = -acc;
                }
            }
            for (int ca = 0; ca < na; ca++) {
                int p3a[3];
                comp_pow(la, ca, p3a[0], p3a[1], p3a[2]);
                for (int cb = 0; cb < nb; cb++) {
                    int p3b[3];
                    comp_pow(lb, cb, p3b[0], p3b[1], p3b[2]);
                    double sd[3], td[3];
                    for (int d = 0; d < 3; d++) {
                        const int u = p3a[d], v = p3b[d];
                        sd[d] = s[d][u][v];
                        double tv = 4.0 * a * b * s[d][u + 1][v + 1];
                        if (u > 0) tv -= 2.0 * b * u * s[d][u - 1][v + 1];
                        if (v > 0) tv -= 2.0 * a * v * s[d][u + 1][v - 1];
                        if (u > 0 && v > 0) tv += u * v * s[d][u - 1][v - 1];
                        td[d] = 0.5 * tv;
                    }
                    sblk[ca * nb + cb] += cc * sd[0] * sd[1] * sd[2];
                    hblk[ca * nb + cb] += cc * (td[0] * sd[1] * sd[2] + sd[0] * td[1] * sd[2] + sd[0] * sd[1] * td[2] +
                                                V[ca * nb + cb]);
                }
            }
        }
    for (int ca = 0; ca < na; ca++)
        for (int cb = 0; cb < nb; cb++) {
            const int r = bf0[i] + ca, c = bf0[j] + cb;
            const double nrm = comp_norm[r] * comp_norm[c];
            if (S) S[(size_t)r * N + c] = S[(size_t)c * N + r] = nrm * sblk[ca * nb + cb];
            if (H) H[(size_t)r * N + c] = H[(size_t)c * N + r] = nrm * hblk[ca * nb + cb];
        }
}

__global__ void k_nuclear_repulsion(int n_atoms, const double* __restrict__ xyz, const double* __restrict__ Z,
                                    double* __restrict__ out)
{
    // single block, fixed-order reduction
    __shared__ double sm[256];
    double e = 0.0;
    for (int a = threadIdx.x; a < n_atoms; a += blockDim.x)
        for (int b = 0; b < a; b++) {
            const double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1],
                         dz = xyz[3 * a + 2] - xyz[3 * b + 2];
            e += Z[a] * Z[b] / sqrt(dx * dx + dy * dy + dz * dz);
        }
    sm[threadIdx.x] = e;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

int launch_one_electron(int n_sh, int n_atoms, int N, const int* l, const int* atom, const int* bf0,
                        const int* nprim, const int* prim0, const double* exps, const double* cn,
                        const double* xyz, const double* Z, const double* comp_norm, const double* boys64,
                        double* S, double* H, cudaStream_t s)
{
    const long long n = (long long)n_sh * (n_sh + 1) / 2;
    if (n > 0)
        k_one_electron<<<(unsigned)((n + 63) / 64), 64, 0, s>>>(n_sh, n_atoms, N, l, atom, bf0, nprim, prim0, exps, cn,
                                                              xyz, Z, comp_norm, boys64, S, H);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_nuclear_repulsion(int n_atoms, const double* xyz, const double* Z, double* out, cudaStream_t s)
{
    k_nuclear_repulsion<<<1, 256, 0, s>>>(n_atoms, xyz, Z, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hf

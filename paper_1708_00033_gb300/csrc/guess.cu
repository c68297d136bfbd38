// Learned initial guess: a small MLP maps per-atom-pair geometric features
// to the corresponding block of the density matrix.  Training and inference
// run in these kernels: BF16 weights (with FP32 master copies for Adam),
// FP32 activations and FP32 accumulation.
//
//   features (16): R, u_x, u_y, u_z, the 9 products u_i u_j, one-hot of the
//                  element pair (O-O, O-H, H-H); u = (r_b - r_a) / R, zero
//                  for on-site pairs (a == b, R = 0)
//   network:       16 -> 256 (SiLU) -> 256 (SiLU) -> 325 = 225 (O-O head)
//                  + 75 (O-H head) + 25 (H-H head); a sample's loss only sees
//                  its own head
//   density:       each unordered pair's predicted block is placed at
//                  P[a, b] (and its transpose at P[b, a]); on-site blocks are
//                  symmetrised; P is finally scaled so that tr(PS) = N_e.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "hf_internal.h"

namespace hf {
namespace {

constexpr int kFeat = 16;
constexpr int kWidth = 256;
constexpr int kOut = 325;
__host__ __device__ __forceinline__ int head_off(int h) { return h == 0 ? 0 : (h == 1 ? 225 : 300); }
__host__ __device__ __forceinline__ int head_rows(int h) { return h == 2 ? 5 : 15; }
__host__ __device__ __forceinline__ int head_cols(int h) { return h == 0 ? 15 : 5; }

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ float ld(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p, size_t i) { return __bfloat162float(p[i]); }

// C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias[N]) with optional SiLU; FP32
// accumulation.  A is FP32; B is FP32 or BF16.  If Z != nullptr the
// pre-activation is stored there and C receives SiLU(Z).  beta = 1 adds into C.
template <typename TB>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda, int ta,
                                               const TB* __restrict__ B, int ldb, int tb, const float* __restrict__ bias,
                                               float* __restrict__ Z, float* __restrict__ C, int ldc, int act, int beta)
{
    __shared__ float As[16][65];
    __shared__ float Bs[16][65];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int k, m;
            if (ta) {
                k = e / 64;
                m = e % 64;
            } else {
                m = e / 16;
                k = e % 16;
            }
            const int gm = m0 + m, gk = k0 + k;
            As[k][m] = (gm < M && gk < K) ? (ta ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk]) : 0.0f;
        }
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int k, n;
            if (tb) {
                n = e / 16;
                k = e % 16;
            } else {
                k = e / 64;
                n = e % 64;
            }
            const int gn = n0 + n, gk = k0 + k;
            Bs[k][n] = (gn < N && gk < K) ? (tb ? ld(B, (size_t)gn * ldb + gk) : ld(B, (size_t)gk * ldb + gn)) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
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
            float v = acc[i][j] + (bias ? bias[gn] : 0.0f);
            const size_t o = (size_t)gm * ldc + gn;
            if (Z) Z[o] = v;
            if (act) v = silu(v);
            C[o] = beta ? C[o] + v : v;
        }
    }
}

template <typename TB>
void sgemm(int M, int N, int K, const float* A, int lda, bool ta, const TB* B, int ldb, bool tb, const float* bias,
           float* Z, float* C, int ldc, bool act, bool beta, cudaStream_t s)
{
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_sgemm<TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, bias, Z, C, ldc, act ? 1 : 0, beta ? 1 : 0);
}

// dY = 2 (Y - T) mask / count, loss partials
__global__ void k_mse(long long n, const float* __restrict__ Y, const float* __restrict__ T,
                      const float* __restrict__ mask, float inv_count, float* __restrict__ dY,
                      double* __restrict__ part)
{
    __shared__ double sm[256];
    double acc = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float d = (Y[e] - T[e]) * mask[e];
        dY[e] = 2.0f * d * inv_count;
        acc += (double)d * d;
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_sum_parts(int nb, const double* __restrict__ part, float scale, float* __restrict__ out)
{
    __shared__ double sm[256];
    double a = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += part[i];
    sm[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)(sm[0] * scale);
}

// g *= dsilu(Z) elementwise
__global__ void k_dsilu(long long n, const float* __restrict__ Z, float* __restrict__ G)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) G[e] *= dsilu(Z[e]);
}

// db[j] = sum_i dY[i, j]
__global__ void k_colsum(int n, int m, const float* __restrict__ dY, float* __restrict__ db)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    float a = 0.0f;
    for (int i = 0; i < n; i++) a += dY[(size_t)i * m + j];
    db[j] = a;
}

// Adam on FP32 master weights, BF16 working copy refreshed
__global__ void k_adam(long long n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wb, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gg;
    const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    const float wn = w[e] - lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    w[e] = wn;
    if (wb) wb[e] = __float2bfloat16(wn);
}

__global__ void k_to_bf16(long long n, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) wb[e] = __float2bfloat16(w[e]);
}

// per unordered atom pair (a <= b): features and block placement
struct PairMeta {
    int row0, col0;  // first basis function of the block's row atom and column atom
    int head;        // 0 O-O, 1 O-H (O rows), 2 H-H
    int onsite;
};

__device__ __forceinline__ int element_class(int Z) { return Z == 8 ? 0 : (Z == 1 ? 1 : -1); }

__global__ void k_guess_features(int n_atoms, const double* __restrict__ xyz, const int* __restrict__ Z,
                                 const int* __restrict__ atom_bf0, float* __restrict__ X,
                                 PairMeta* __restrict__ meta, int* __restrict__ bad)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long np = (long long)n_atoms * (n_atoms + 1) / 2;
    if (t >= np) return;
    long long ii = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (ii * (ii + 1) / 2 > t) ii--;
    while ((ii + 1) * (ii + 2) / 2 <= t) ii++;
    int a = (int)(t - ii * (ii + 1) / 2), b = (int)ii;  // a <= b
    int ca = element_class(Z[a]), cb = element_class(Z[b]);
    if (ca < 0 || cb < 0) {
        atomicOr(bad, 1);
        ca = cb = 1;
    }
    if (ca == 1 && cb == 0) {  // O-H blocks have the O atom first
        const int t2 = a;
        a = b;
        b = t2;
        ca = 0;
        cb = 1;
    }
    float u[3] = {0.f, 0.f, 0.f}, R = 0.f;
    if (a != b) {
        const double d0 = xyz[3 * b] - xyz[3 * a], d1 = xyz[3 * b + 1] - xyz[3 * a + 1], d2 = xyz[3 * b + 2] - xyz[3 * a + 2];
        const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        R = (float)r;
        u[0] = (float)(d0 / r);
        u[1] = (float)(d1 / r);
        u[2] = (float)(d2 / r);
    }
    float* x = X + t * kFeat;
    x[0] = R;
    x[1] = u[0];
    x[2] = u[1];
    x[3] = u[2];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) x[4 + 3 * i + j] = u[i] * u[j];
    const int head = ca == 0 ? (cb == 0 ? 0 : 1) : 2;
    x[13] = head == 0;
    x[14] = head == 1;
    x[15] = head == 2;
    PairMeta pm;
    pm.row0 = atom_bf0[a];
    pm.col0 = atom_bf0[b];
    pm.head = head;
    pm.onsite = a == b;
    meta[t] = pm;
}

// place each pair's predicted block; on-site blocks symmetrised
__global__ void k_guess_scatter(long long np, int N, const float* __restrict__ Y, const PairMeta* __restrict__ meta,
                                double* __restrict__ P)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const PairMeta pm = meta[t];
    const int h = pm.head, nr = head_rows(h), nc = head_cols(h);
    const float* y = Y + t * kOut + head_off(h);
    for (int r = 0; r < nr; r++)
        for (int c = 0; c < nc; c++) {
            double v = y[r * nc + c];
            if (pm.onsite) v = 0.5 * (v + (double)y[c * nc + r]);
            P[(size_t)(pm.row0 + r) * N + pm.col0 + c] = v;
            P[(size_t)(pm.col0 + c) * N + pm.row0 + r] = v;
        }
}

// Training targets of every atom pair: T[t][head block] = the pair's block of P, mask 1 there, 0 elsewhere.
__global__ void k_guess_targets(long long np, int N, const double* __restrict__ P, const PairMeta* __restrict__ meta,
                                float* __restrict__ T, float* __restrict__ mask)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np * kOut) return;
    const long long t = e / kOut;
    const int o = (int)(e - t * kOut);
    const PairMeta pm = meta[t];
    const int h = pm.head, o0 = head_off(h), nc = head_cols(h);
    const int r = (o - o0) / nc, c = (o - o0) % nc;
    const bool in = o >= o0 && o < o0 + head_rows(h) * nc;
    T[e] = in ? (float)P[(size_t)(pm.row0 + r) * N + pm.col0 + c] : 0.0f;
    mask[e] = in ? 1.0f : 0.0f;
}

// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014) applied to seed + (i + 1) * golden gamma.
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long i)
{
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Minibatch of step k: sample j is row splitmix64(seed, k * batch + j) mod n of the dataset.
__global__ void k_draw_batch(long long n, int batch, unsigned long long seed, long long step,
                             const float* __restrict__ X, const float* __restrict__ T, const float* __restrict__ M,
                             float* __restrict__ Xb, float* __restrict__ Tb, float* __restrict__ Mb)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)batch * kOut) return;
    const int j = (int)(e / kOut), o = (int)(e % kOut);
    const long long row = (long long)(splitmix64(seed, (unsigned long long)(step * batch + j)) % (unsigned long long)n);
    Tb[e] = T[row * kOut + o];
    Mb[e] = M[row * kOut + o];
    if (o < kFeat) Xb[(size_t)j * kFeat + o] = X[row * kFeat + o];
}

__global__ void k_trace_ps(int N, const double* __restrict__ P, const double* __restrict__ S, double* __restrict__ part)
{
    __shared__ double sm[256];
    double acc = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)N * N;
         e += (long long)gridDim.x * blockDim.x)
        acc += P[e] * S[e];  // tr(PS) = sum_ij P_ij S_ji, S symmetric
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_scale_density_to(int N, const double* __restrict__ part, double n_el, double* __restrict__ P,
                                   int* __restrict__ bad)
{
    __shared__ double tr;
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < 256; i++) a += part[i];
        tr = a;
        if (!(a > 0.0) || !isfinite(a)) atomicOr(bad, 2);
    }
    __syncthreads();
    const double f = (tr > 0.0 && isfinite(tr)) ? n_el / tr : 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)N * N;
         e += (long long)gridDim.x * blockDim.x) {
        const double v = P[e] * f;
        if (!isfinite(v)) atomicOr(bad, 4);
        P[e] = v;
    }
}

int gfail(int code, const std::string& msg)
{
    set_error(code, msg);
    return code;
}

struct GuessDevice {
    int prev = -1;
    explicit GuessDevice(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~GuessDevice()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace hf

using namespace hf;

struct hf_model {
    hf_ctx* ctx = nullptr;
    // FP32 master weights, BF16 copies, gradients, Adam moments: W1 [256x16], b1, W2 [256x256], b2, W3 [325x256], b3
    DevBuf w, wb, g, m, v;
    long long n_params = 0;
    long long off[6] = {};
    int step = 0;
    // activation workspace
    DevBuf Z1, H1, Z2, H2, Y, dY, dH, dZ, part, lossbuf;
    DevBuf Xb, Tb, Mb;  // minibatch drawn by hf_guess_train
    long long cap = 0, bcap = 0;
    int reserve(long long n)
    {
        if (n <= cap) return HF_OK;
        const long long c = std::max(n, 1024LL);
        int rc;
        if ((rc = Z1.alloc(sizeof(float) * c * kWidth)) || (rc = H1.alloc(sizeof(float) * c * kWidth)) ||
            (rc = Z2.alloc(sizeof(float) * c * kWidth)) || (rc = H2.alloc(sizeof(float) * c * kWidth)) ||
            (rc = Y.alloc(sizeof(float) * c * kOut)) || (rc = dY.alloc(sizeof(float) * c * kOut)) ||
            (rc = dH.alloc(sizeof(float) * c * kWidth)) || (rc = dZ.alloc(sizeof(float) * c * kWidth)))
            return rc;
        cap = c;
        return HF_OK;
    }
    float* W(int i) { return w.as<float>() + off[i]; }
    __nv_bfloat16* Wb(int i) { return wb.as<__nv_bfloat16>() + off[i]; }
    float* G(int i) { return g.as<float>() + off[i]; }
};

static const long long kSizes[6] = {(long long)kWidth * kFeat, kWidth, (long long)kWidth * kWidth, kWidth,
                                    (long long)kOut * kWidth, kOut};

static int forward(hf_model* M, int n, const float* X, cudaStream_t st)
{
    sgemm<__nv_bfloat16>(n, kWidth, kFeat, X, kFeat, false, M->Wb(0), kFeat, true, M->W(1), M->Z1.as<float>(),
                         M->H1.as<float>(), kWidth, true, false, st);
    sgemm<__nv_bfloat16>(n, kWidth, kWidth, M->H1.as<float>(), kWidth, false, M->Wb(2), kWidth, true, M->W(3),
                         M->Z2.as<float>(), M->H2.as<float>(), kWidth, true, false, st);
    sgemm<__nv_bfloat16>(n, kOut, kWidth, M->H2.as<float>(), kWidth, false, M->Wb(4), kWidth, true, M->W(5), nullptr,
                         M->Y.as<float>(), kOut, false, false, st);
    return cudaGetLastError() == cudaSuccess ? HF_OK : cuda_status(cudaGetLastError(), "guess forward");
}

// gradients of loss = sum(mask (Y - T)^2) / count into M->g
static int backward(hf_model* M, int n, const float* X, const float* T, const float* mask, float* loss,
                    cudaStream_t st, float* loss_dev = nullptr)
{
    // loss = (1/n) sum_samples sum_outputs mask (Y - T)^2, masks being 0/1 per output
    const long long ny = (long long)n * kOut;
    const float inv = 1.0f / (float)n;
    k_mse<<<128, 256, 0, st>>>(ny, M->Y.as<float>(), T, mask, inv, M->dY.as<float>(), M->part.as<double>());
    if (loss || loss_dev)
        k_sum_parts<<<1, 256, 0, st>>>(128, M->part.as<double>(), inv, loss_dev ? loss_dev : M->lossbuf.as<float>());
    // layer 3
    sgemm<float>(kOut, kWidth, n, M->dY.as<float>(), kOut, true, M->H2.as<float>(), kWidth, false, nullptr, nullptr,
                 M->G(4), kWidth, false, false, st);
    k_colsum<<<(kOut + 127) / 128, 128, 0, st>>>(n, kOut, M->dY.as<float>(), M->G(5));
    sgemm<__nv_bfloat16>(n, kWidth, kOut, M->dY.as<float>(), kOut, false, M->Wb(4), kWidth, false, nullptr, nullptr,
                         M->dH.as<float>(), kWidth, false, false, st);
    k_dsilu<<<(unsigned)(((long long)n * kWidth + 255) / 256), 256, 0, st>>>((long long)n * kWidth, M->Z2.as<float>(),
                                                                           M->dH.as<float>());
    // layer 2
    sgemm<float>(kWidth, kWidth, n, M->dH.as<float>(), kWidth, true, M->H1.as<float>(), kWidth, false, nullptr, nullptr,
                 M->G(2), kWidth, false, false, st);
    k_colsum<<<(kWidth + 127) / 128, 128, 0, st>>>(n, kWidth, M->dH.as<float>(), M->G(3));
    sgemm<__nv_bfloat16>(n, kWidth, kWidth, M->dH.as<float>(), kWidth, false, M->Wb(2), kWidth, false, nullptr,
                         nullptr, M->dZ.as<float>(), kWidth, false, false, st);
    k_dsilu<<<(unsigned)(((long long)n * kWidth + 255) / 256), 256, 0, st>>>((long long)n * kWidth, M->Z1.as<float>(),
                                                                           M->dZ.as<float>());
    // layer 1
    sgemm<float>(kWidth, kFeat, n, M->dZ.as<float>(), kWidth, true, X, kFeat, false, nullptr, nullptr, M->G(0), kFeat,
                 false, false, st);
    k_colsum<<<(kWidth + 127) / 128, 128, 0, st>>>(n, kWidth, M->dZ.as<float>(), M->G(1));
    if (loss && !loss_dev) {
        HF_CUDA(cudaMemcpyAsync(loss, M->lossbuf.p, sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    return cudaGetLastError() == cudaSuccess ? HF_OK : cuda_status(cudaGetLastError(), "guess backward");
}

// One Adam step (beta 0.9 / 0.999, eps 1e-8) on the gradients in M->g with learning rate lr.
static void adam_step(hf_model* M, float lr, cudaStream_t st)
{
    M->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f / (1.0f - powf(b1, (float)M->step)), c2 = 1.0f / (1.0f - powf(b2, (float)M->step));
    k_adam<<<(unsigned)((M->n_params + 255) / 256), 256, 0, st>>>(M->n_params, M->w.as<float>(), M->g.as<float>(),
                                                                  M->m.as<float>(), M->v.as<float>(),
                                                                  M->wb.as<__nv_bfloat16>(), lr, b1, b2, 1e-8f, c1, c2);
}

extern "C" {

int hf_model_create(hf_ctx* ctx, const float* init_weights, hf_model** out)
{
    if (!ctx || !init_weights || !out) return gfail(HF_E_INVALID, "hf_model_create: NULL argument");
    *out = nullptr;
    GuessDevice gd(ctx->device);
    hf_model* M = new hf_model();
    M->ctx = ctx;
    long long o = 0;
    for (int i = 0; i < 6; i++) {
        M->off[i] = o;
        o += kSizes[i];
    }
    M->n_params = o;
    int rc;
    if ((rc = M->w.alloc(sizeof(float) * o)) || (rc = M->wb.alloc(sizeof(__nv_bfloat16) * o)) ||
        (rc = M->g.alloc(sizeof(float) * o)) || (rc = M->m.alloc(sizeof(float) * o)) ||
        (rc = M->v.alloc(sizeof(float) * o)) || (rc = M->part.alloc(sizeof(double) * 256)) ||
        (rc = M->lossbuf.alloc(sizeof(float) * 4))) {
        delete M;
        return rc;
    }
    cudaStream_t st = ctx->stream;
    HF_CUDA(cudaMemcpyAsync(M->w.p, init_weights, sizeof(float) * o, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemsetAsync(M->m.p, 0, sizeof(float) * o, st));
    HF_CUDA(cudaMemsetAsync(M->v.p, 0, sizeof(float) * o, st));
    k_to_bf16<<<(unsigned)((o + 255) / 256), 256, 0, st>>>(o, M->w.as<float>(), M->wb.as<__nv_bfloat16>());
    HF_CUDA(cudaStreamSynchronize(st));
    *out = M;
    return HF_OK;
}

void hf_model_destroy(hf_model* M)
{
    if (!M) return;
    GuessDevice gd(M->ctx->device);
    cudaStreamSynchronize(M->ctx->stream);
    delete M;
}

int64_t hf_model_num_params(void) { return kSizes[0] + kSizes[1] + kSizes[2] + kSizes[3] + kSizes[4] + kSizes[5]; }

int hf_model_get_weights(hf_model* M, float* w, float* grad)
{
    if (!M) return gfail(HF_E_INVALID, "hf_model_get_weights: NULL model");
    GuessDevice gd(M->ctx->device);
    cudaStream_t st = M->ctx->stream;
    if (w) HF_CUDA(cudaMemcpyAsync(w, M->w.p, sizeof(float) * M->n_params, cudaMemcpyDeviceToHost, st));
    if (grad) HF_CUDA(cudaMemcpyAsync(grad, M->g.p, sizeof(float) * M->n_params, cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    return HF_OK;
}

int hf_model_forward(hf_model* M, int n, const float* X, float* Y, int flags)
{
    if (!M || !X || !Y || n <= 0) return gfail(HF_E_INVALID, "hf_model_forward: bad arguments");
    GuessDevice gd(M->ctx->device);
    cudaStream_t st = M->ctx->stream;
    int rc = M->reserve(n);
    if (rc != HF_OK) return rc;
    const bool dev = (flags & HF_PTR_DEVICE) != 0;
    DevBuf Xd;
    const float* xp = X;
    if (!dev) {
        if ((rc = Xd.alloc(sizeof(float) * (size_t)n * kFeat))) return rc;
        HF_CUDA(cudaMemcpyAsync(Xd.p, X, sizeof(float) * (size_t)n * kFeat, cudaMemcpyHostToDevice, st));
        xp = Xd.as<float>();
    }
    if ((rc = forward(M, n, xp, st)) != HF_OK) return rc;
    HF_CUDA(cudaMemcpyAsync(Y, M->Y.p, sizeof(float) * (size_t)n * kOut,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    return HF_OK;
}

int hf_model_train_step(hf_model* M, int n, const float* X, const float* T, const float* mask, float lr,
                        float* loss, int flags)
{
    if (!M || !X || !T || !mask || n <= 0) return gfail(HF_E_INVALID, "hf_model_train_step: bad arguments");
    GuessDevice gd(M->ctx->device);
    cudaStream_t st = M->ctx->stream;
    int rc = M->reserve(n);
    if (rc != HF_OK) return rc;
    if (!(flags & HF_PTR_DEVICE)) return gfail(HF_E_INVALID, "hf_model_train_step: device pointers required");
    if ((rc = forward(M, n, X, st)) != HF_OK) return rc;
    if ((rc = backward(M, n, X, T, mask, loss, st)) != HF_OK) return rc;
    if (lr > 0.0f) adam_step(M, lr, st);
    HF_CUDA(cudaStreamSynchronize(st));
    HF_CUDA(cudaGetLastError());
    return HF_OK;
}

int hf_guess_train(hf_model* M, int64_t n, const float* X, const float* T, const float* mask,
                   const hf_train_opts* opts, float* losses, int flags)
{
    if (!M || !X || !T || !mask || !opts || n <= 0) return gfail(HF_E_INVALID, "hf_guess_train: bad arguments");
    if (!(flags & HF_PTR_DEVICE)) return gfail(HF_E_INVALID, "hf_guess_train: the dataset must be in device memory");
    if (opts->steps <= 0 || opts->batch < 0 || !(opts->lr >= 0.0f) || !isfinite(opts->lr))
        return gfail(HF_E_INVALID, "hf_guess_train: bad options");
    GuessDevice gd(M->ctx->device);
    cudaStream_t st = M->ctx->stream;
    const int batch = (int)std::min<int64_t>(opts->batch > 0 ? opts->batch : 2048, n);
    const float lr = opts->lr > 0.0f ? opts->lr : 1e-3f;
    int rc = M->reserve(batch);
    if (rc != HF_OK) return rc;
    if (batch > M->bcap) {
        if ((rc = M->Xb.alloc(sizeof(float) * (size_t)batch * kFeat)) ||
            (rc = M->Tb.alloc(sizeof(float) * (size_t)batch * kOut)) ||
            (rc = M->Mb.alloc(sizeof(float) * (size_t)batch * kOut))) {
            M->bcap = 0;
            return rc;
        }
        M->bcap = batch;
    }
    DevBuf ldev;
    if ((rc = ldev.alloc(sizeof(float) * (size_t)opts->steps))) return rc;
    const long long ne = (long long)batch * kOut;
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < opts->steps; k++) {
        k_draw_batch<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(n, batch, (unsigned long long)opts->seed, k, X, T,
                                                                  mask, M->Xb.as<float>(), M->Tb.as<float>(),
                                                                  M->Mb.as<float>());
        if ((rc = forward(M, batch, M->Xb.as<float>(), st)) != HF_OK) return rc;
        if ((rc = backward(M, batch, M->Xb.as<float>(), M->Tb.as<float>(), M->Mb.as<float>(), nullptr, st,
                           ldev.as<float>() + k)) != HF_OK)
            return rc;
        // cosine decay from lr to 0 over the run
        const float lr_k = (float)(lr * 0.5 * (1.0 + cos(pi * (double)k / (double)opts->steps)));
        if (lr_k > 0.0f) adam_step(M, lr_k, st);
    }
    HF_CUDA(cudaGetLastError());
    if (losses) HF_CUDA(cudaMemcpyAsync(losses, ldev.p, sizeof(float) * (size_t)opts->steps, cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    HF_CUDA(cudaGetLastError());
    return HF_OK;
}

// Check that every atom is H (5 functions) or O (15 functions) with contiguous shells.
static int check_guess_basis(const hf_system* S)
{
    for (int a = 0; a < S->n_atoms; a++) {
        const int z = S->Z_h[a], nb = S->atom_nbf_h[a];
        if (!((z == 8 && nb == 15) || (z == 1 && nb == 5)) || S->atom_bf0_h[a] < 0)
            return gfail(HF_E_UNSUPPORTED, "learned guess: every atom must be O with 15 or H with 5 contiguous "
                                           "Cartesian functions (the synthetic water basis)");
    }
    return HF_OK;
}

// per-pair features of a system: X [n_pairs x 16] floats, meta [n_pairs x 4] ints
// (row atom's first function, column atom's first function, head, on-site flag)
int hf_guess_features(hf_system* S, float* X, int32_t* meta, int64_t* n_pairs, int flags)
{
    if (!S || !n_pairs) return gfail(HF_E_INVALID, "hf_guess_features: NULL argument");
    const long long np = (long long)S->n_atoms * (S->n_atoms + 1) / 2;
    *n_pairs = np;
    if (!X || !meta) return HF_OK;  // size query
    int rc = check_guess_basis(S);
    if (rc != HF_OK) return rc;
    GuessDevice gd(S->device);
    cudaStream_t st = S->stream;
    DevBuf bf0, Zi, bad, Xd, Md;
    if ((rc = bf0.alloc(sizeof(int) * S->n_atoms)) || (rc = Zi.alloc(sizeof(int) * S->n_atoms)) ||
        (rc = bad.alloc(sizeof(int))))
        return rc;
    HF_CUDA(cudaMemcpyAsync(Zi.p, S->Z_h.data(), sizeof(int) * S->n_atoms, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemcpyAsync(bf0.p, S->atom_bf0_h.data(), sizeof(int) * S->n_atoms, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    const bool dev = (flags & HF_PTR_DEVICE) != 0;
    float* xp = X;
    PairMeta* mp = (PairMeta*)meta;
    if (!dev) {
        if ((rc = Xd.alloc(sizeof(float) * np * kFeat)) || (rc = Md.alloc(sizeof(PairMeta) * np))) return rc;
        xp = Xd.as<float>();
        mp = Md.as<PairMeta>();
    }
    k_guess_features<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(S->n_atoms, S->atom_xyz.as<double>(), Zi.as<int>(),
                                                                  bf0.as<int>(), xp, mp, bad.as<int>());
    int hb = 0;
    HF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (!dev) {
        HF_CUDA(cudaMemcpyAsync(X, xp, sizeof(float) * np * kFeat, cudaMemcpyDeviceToHost, st));
        HF_CUDA(cudaMemcpyAsync(meta, mp, sizeof(PairMeta) * np, cudaMemcpyDeviceToHost, st));
    }
    HF_CUDA(cudaStreamSynchronize(st));
    if (hb) return gfail(HF_E_UNSUPPORTED, "hf_guess_features: only H and O atoms are supported");
    return HF_OK;
}

int hf_guess_targets(hf_system* S, const double* P, float* T, float* mask, int flags)
{
    if (!S || !P || !T || !mask) return gfail(HF_E_INVALID, "hf_guess_targets: NULL argument");
    GuessDevice gd(S->device);
    cudaStream_t st = S->stream;
    int64_t np = 0;
    hf_guess_features(S, nullptr, nullptr, &np, 0);
    const int N = S->n_bf;
    const bool dev = (flags & HF_PTR_DEVICE) != 0;
    DevBuf X, meta, Pd, Td, Md;
    int rc;
    if ((rc = X.alloc(sizeof(float) * np * kFeat)) || (rc = meta.alloc(sizeof(PairMeta) * np))) return rc;
    if ((rc = hf_guess_features(S, X.as<float>(), (int32_t*)meta.p, &np, HF_PTR_DEVICE)) != HF_OK) return rc;
    const double* pp = P;
    float *tp = T, *mp = mask;
    if (!dev) {
        if ((rc = Pd.alloc(sizeof(double) * (size_t)N * N)) || (rc = Td.alloc(sizeof(float) * np * kOut)) ||
            (rc = Md.alloc(sizeof(float) * np * kOut)))
            return rc;
        HF_CUDA(cudaMemcpyAsync(Pd.p, P, sizeof(double) * (size_t)N * N, cudaMemcpyHostToDevice, st));
        pp = Pd.as<double>();
        tp = Td.as<float>();
        mp = Md.as<float>();
    }
    const long long ne = np * kOut;
    k_guess_targets<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(np, N, pp, meta.as<PairMeta>(), tp, mp);
    HF_CUDA(cudaGetLastError());
    if (!dev) {
        HF_CUDA(cudaMemcpyAsync(T, tp, sizeof(float) * ne, cudaMemcpyDeviceToHost, st));
        HF_CUDA(cudaMemcpyAsync(mask, mp, sizeof(float) * ne, cudaMemcpyDeviceToHost, st));
    }
    HF_CUDA(cudaStreamSynchronize(st));
    return HF_OK;
}

int hf_guess_predict(hf_model* M, hf_system* S, double* P, int flags)
{
    if (!M || !S || !P) return gfail(HF_E_INVALID, "hf_guess_predict: NULL argument");
    GuessDevice gd(S->device);
    cudaStream_t st = S->stream;
    int64_t np = 0;
    hf_guess_features(S, nullptr, nullptr, &np, 0);
    DevBuf X, meta, Pd, part, bad;
    int rc;
    if ((rc = X.alloc(sizeof(float) * np * kFeat)) || (rc = meta.alloc(sizeof(PairMeta) * np)) ||
        (rc = part.alloc(sizeof(double) * 256)) || (rc = bad.alloc(sizeof(int))))
        return rc;
    if ((rc = hf_guess_features(S, X.as<float>(), (int32_t*)meta.p, &np, HF_PTR_DEVICE)) != HF_OK)
        return rc;
    if ((rc = M->reserve(np)) != HF_OK) return rc;
    if ((rc = forward(M, (int)np, X.as<float>(), st)) != HF_OK) return rc;
    const int N = S->n_bf;
    const bool dev = (flags & HF_PTR_DEVICE) != 0;
    double* pp = P;
    if (!dev) {
        if ((rc = Pd.alloc(sizeof(double) * (size_t)N * N))) return rc;
        pp = Pd.as<double>();
    }
    HF_CUDA(cudaMemsetAsync(pp, 0, sizeof(double) * (size_t)N * N, st));
    HF_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    k_guess_scatter<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(np, N, M->Y.as<float>(), meta.as<PairMeta>(), pp);
    k_trace_ps<<<256, 256, 0, st>>>(N, pp, S->S.as<double>(), part.as<double>());
    k_scale_density_to<<<256, 256, 0, st>>>(N, part.as<double>(), (double)S->n_electrons, pp, bad.as<int>());
    int hb = 0;
    HF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (!dev) HF_CUDA(cudaMemcpyAsync(P, pp, sizeof(double) * (size_t)N * N, cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    HF_CUDA(cudaGetLastError());
    if (hb) return gfail(HF_E_INVALID, "hf_guess_predict: the predicted density is not finite or has tr(PS) <= 0");
    return HF_OK;
}

}  // extern "C"

// Device-side building blocks shared by the generated ERI class kernels.
//
// Shell pairs (Algorithm 1's (i, j) index; Section 4.1's shell footnote) are
// stored once per significant unordered pair, oriented so that l_A >= l_B,
// with one record per primitive pair.  Quartets of one angular class are the
// pairs (bra b, ket k) of two Schwarz-sorted pair lists; bra b owns the ket
// prefix [kstart[b], kstart[b] + offsets[b+1] - offsets[b]), which is how the
// screening of Algorithm 1 (schwartz(i,j,k,l)) becomes a per-bra cut on a list
// sorted by Q_kl.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hf_internal.h"

namespace hf {

template <typename real>
struct PrimPair {
    real p;              // a + b
    real Px, Py, Pz;     // (a A + b B) / p
    real PAx, PAy, PAz;  // P - A
    real K;              // c_a c_b exp(-ab/p |AB|^2) sqrt(2) pi^(5/4) / p
    real oo2p;           // 1 / (2p)
    float B;             // primitive-pair Schwarz bound sqrt(max |[ab|ab]|), normalised components
};

// Ket primitive-pair records as the generated quartet functions read them.
//   KetAos: the pair's own records (PrimPair array at prims + prim0, or a shared-memory copy of them);
//   KetSoa: the ket's column of its class's ket table, a field-major copy of every significant pair's
//           records in class-list order (field f of record i of ket k at f9[(9 i + f) stride + k], bound
//           at fB[i stride + k]): the 32 lanes of a warp, which hold consecutive kets of a class list,
//           read 32 consecutive words per field instead of 32 scattered records.
template <typename real>
struct KetAos {
    const PrimPair<real>* __restrict__ r;
    __device__ __forceinline__ PrimPair<real> rec(int i) const { return r[i]; }
    __device__ __forceinline__ float B(int i) const { return r[i].B; }
};

template <typename real>
struct KetSoa {
    const real* __restrict__ f9;
    const float* __restrict__ fB;
    long long stride;
    __device__ __forceinline__ PrimPair<real> rec(int i) const
    {
        const real* q = f9 + (long long)i * 9 * stride;
        PrimPair<real> x;
        x.p = __ldg(q);
        x.Px = __ldg(q + stride);
        x.Py = __ldg(q + 2 * stride);
        x.Pz = __ldg(q + 3 * stride);
        x.PAx = __ldg(q + 4 * stride);
        x.PAy = __ldg(q + 5 * stride);
        x.PAz = __ldg(q + 6 * stride);
        x.K = __ldg(q + 7 * stride);
        x.oo2p = __ldg(q + 8 * stride);
        x.B = __ldg(fB + (long long)i * stride);
        return x;
    }
    __device__ __forceinline__ float B(int i) const { return __ldg(fB + (long long)i * stride); }
};

// Boys tables in Taylor-coefficient form, so that evaluation is a pure Horner chain:
//   FP64 rows, two regions of one table:
//     A: T_k = k / 512 for k = 0..kBoysRowsA-1 (T < 64): c[m][j] = F_{m+j}(T_k) / j!  (m = 0..8, j = 0..4)
//        at m*5 + j, and e^{-T_k} / j! (j = 0..4) at 45 + j;
//     B: T_k = 2^e (1 + i / 4096), e = 6..31, i = 0..4095 (64 <= T < 2^31): the same coefficients of the
//        asymptotic form F_m(T) = (2m-1)!! / 2^(m+1) sqrt(pi / T^(2m+1)), which is F_m to within half an
//        ulp there (every order's switch point is below 64), with the e^{-T_k} coefficients zero;
//   FP32 rows T_k = k / 32, k = 0..kBoysRows32-1 (T < 60):
//             c[m][j] = F_{m+j}(T_k) / j!  (m = 0..8, j = 0..3) at m*4 + j,
//             e^{-T_k} / j! (j = 0..4) at 36 + j.
// One FP64 table over both regions gives every lane of a warp the same instruction stream whatever its
// T (no Taylor/asymptotic branch to diverge on); the grids are fine so that each Horner chain is short.
// FP64 instructions are the scarce resource of the ERI kernels, table loads are not.
constexpr int kBoysRowsA = 64 * 512 + 1;
constexpr int kBoysBinade0 = 6;    // region B starts at 2^6 = 64
constexpr int kBoysBinades = 26;   // binades 2^6 .. 2^31 (the last one only its first row)
constexpr int kBoysSubBits = 12;   // 4096 rows per binade
constexpr int kBoysRows64 = kBoysRowsA + (kBoysBinades << kBoysSubBits);
constexpr long long kBoysBitsB = 0x4050000000000000LL;    // bit pattern of 64.0
constexpr long long kBoysBitsTop = 0x41E0000000000000LL;  // bit pattern of 2^31
constexpr int kBoysRows32 = 60 * 32 + 1;
constexpr int kBoysStride64 = 50;
constexpr int kBoysStride32 = 44;
constexpr int kBoysExp64 = 45;
constexpr int kBoysExp32 = 36;
constexpr double kBoysTmax = 60.0;

__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }

// Switch points of the asymptotic form F_m(T) ~ (2m-1)!! / 2^(m+1) sqrt(pi / T^(2m+1)), by the highest
// order L evaluated: from these T on, its relative error (the dropped terms carry e^{-T}) is below half
// an ulp for every m <= L, in FP64 (2^-54) and FP32 (2^-25), computed from the incomplete gamma function
// at 40 digits.  FP32: below them the Taylor table, above them the asymptotic form.  FP64: the asymptotic
// rows of the table (region B) start at 64, above every order's switch point.
__host__ __device__ constexpr double boys_switch64(int L)
{
    return L == 0 ? 36.0 : L == 1 ? 40.0 : L == 2 ? 43.0 : L == 3 ? 46.0 : L == 4 ? 49.0 : L == 5 ? 52.0
         : L == 6 ? 54.0 : L == 7 ? 57.0 : 59.0;
}
__host__ __device__ constexpr float boys_switch32(int L)
{
    return L == 0 ? 16.0f : L == 1 ? 19.0f : L == 2 ? 22.0f : L == 3 ? 25.0f : L == 4 ? 27.0f : L == 5 ? 29.0f
         : L == 6 ? 31.0f : L == 7 ? 33.0f : 35.0f;
}

// F_m(T), m = 0..L, FP64.  Taylor expansion about the nearest row T_k of the table (region A: |T - T_k| <=
// 1/1024, five terms, truncation below (1/1024)^5 / 5! < 1e-17 relative, as |F_{m+5}| <= |F_m|; region B:
// |T - T_k| <= T / 8192, where the asymptotic form's fifth-order term is below 2e-17 relative for m <= 8),
// using dF_m/dT = -F_{m+1}, which the asymptotic form obeys as well.  For L >= 2 only F_L is expanded and
// the rest follow from the downward recursion F_m = (2T F_{m+1} + e^{-T}) / (2m+1), with e^{-T} =
// e^{-T_k} e^{T_k - T} expanded the same way (zero in region B).  Region A's row is the integer that
// T*512 + 1.5*2^52 rounds to, read from the low word of the sum; region B's row and T_k come from T's bit
// pattern rounded to 12 mantissa bits.  T >= 2^31 (far beyond any screened quartet) takes the asymptotic
// form directly: F_0 = sqrt(pi/T)/2, F_{m+1} = (2m+1) F_m / (2T).
static_assert(boys_switch64(8) <= 64.0, "region B of the FP64 table must lie above every switch point");
template <int L>
__device__ __forceinline__ void boys_eval(double T, const double* __restrict__ tab, double* F)
{
    const long long bits = __double_as_longlong(T);
    if (bits < kBoysBitsTop) {
        const double big = 6755399441055744.0;  // 1.5 * 2^52
        const double t = fma(T, 512.0, big);
        int k = __double2loint(t);
        double d = fma(t - big, 1.0 / 512.0, -T);  // T_k - T (region A)
        const long long rb = bits + (1LL << (51 - kBoysSubBits));
        const double Tk = __longlong_as_double(rb & ~((1LL << (52 - kBoysSubBits)) - 1));
        const double dB = Tk - T;
        if (bits >= kBoysBitsB) {
            k = kBoysRowsA + (((int)(rb >> 52) - 1023 - kBoysBinade0) << kBoysSubBits)
              + (int)((rb >> (52 - kBoysSubBits)) & ((1 << kBoysSubBits) - 1));
            d = dB;
        }
        const double* __restrict__ r = tab + (size_t)k * kBoysStride64;
        if constexpr (L <= 1) {
#pragma unroll
            for (int m = 0; m <= L; m++) {
                const double* c = r + 5 * m;
                F[m] = c[0] + d * (c[1] + d * (c[2] + d * (c[3] + d * c[4])));
            }
        } else {
            const double* c = r + 5 * L;
            F[L] = c[0] + d * (c[1] + d * (c[2] + d * (c[3] + d * c[4])));
            const double* x = r + kBoysExp64;
            const double e = x[0] + d * (x[1] + d * (x[2] + d * (x[3] + d * x[4])));
            const double t2 = T + T;
#pragma unroll
            for (int m = L - 1; m >= 0; m--) F[m] = (t2 * F[m + 1] + e) * (1.0 / (2 * m + 1));
        }
    } else {
        const double rs = rsqrt(T);
        F[0] = 0.88622692545275801365 * rs;
        if constexpr (L > 0) {
            const double h = 0.5 * rs * rs;
#pragma unroll
            for (int m = 0; m < L; m++) F[m + 1] = F[m] * ((2 * m + 1) * h);
        }
    }
}

// Single-precision variant for the mixed path: four Taylor terms (truncation
// < 3e-9 relative), same recursions, asymptotic from boys_switch32(L).
template <int L>
__device__ __forceinline__ void boys_eval(float T, const float* __restrict__ tab, float* F)
{
    if (T < boys_switch32(L)) {
        const float big = 12582912.0f;  // 1.5 * 2^23
        const float t = fmaf(T, 32.0f, big);
        const int k = __float_as_int(t) - 0x4B400000;
        const float d = fmaf(t - big, 1.0f / 32.0f, -T);
        const float* __restrict__ r = tab + k * kBoysStride32;
        if constexpr (L <= 1) {
#pragma unroll
            for (int m = 0; m <= L; m++) {
                const float* c = r + 4 * m;
                F[m] = c[0] + d * (c[1] + d * (c[2] + d * c[3]));
            }
        } else {
            const float* c = r + 4 * L;
            F[L] = c[0] + d * (c[1] + d * (c[2] + d * c[3]));
            const float* x = r + kBoysExp32;
            const float e = x[0] + d * (x[1] + d * (x[2] + d * (x[3] + d * x[4])));
            const float t2 = T + T;
#pragma unroll
            for (int m = L - 1; m >= 0; m--) F[m] = (t2 * F[m + 1] + e) * (1.0f / (2 * m + 1));
        }
    } else {
        const float rs = rsqrtf(T);
        F[0] = 0.886226925f * rs;
        if constexpr (L > 0) {
            const float h = 0.5f * rs * rs;
#pragma unroll
            for (int m = 0; m < L; m++) F[m + 1] = F[m] * ((2 * m + 1) * h);
        }
    }
}

template <typename real, int L>
__device__ __forceinline__ void boys(real T, const real* __restrict__ tab, real* F)
{
    boys_eval<L>(T, tab, F);
}

__device__ __forceinline__ void red_add(double* p, double v) { atomicAdd(p, v); }

// A - B of a pair in the kernel's arithmetic type (FP32 kernels read the FP32 copies).
template <typename real>
__device__ __forceinline__ real pair_ab(double d, float f)
{
    if constexpr (sizeof(real) == 8)
        return d;
    else
        return f;
}

// Largest b in [0, n) with off[b] <= q (off is non-decreasing, off[0] = 0).
__device__ __forceinline__ int find_bra(const long long* __restrict__ off, int n, long long q)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= q)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Largest b in [lo, hi] with off[b] <= q, given off[lo] <= q (the bra lookup tables bound the range).
__device__ __forceinline__ int find_bra_in(const long long* __restrict__ off, int lo, int hi, long long q)
{
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= q)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

constexpr int kEriThreads = 128;

// Density-weighted screening: a quartet (AB|CD) changes the six Fock blocks of Eq. 1a-1f by at most
// Q_AB Q_CD times the largest |P| of the blocks (CD), (AB), (BD), (AC), (BC), (AD) it is contracted with
// (times 4 for the Coulomb weight); density_block_max returns that largest |P|.  The quartet is skipped
// when 4 Q_AB Q_CD max|P| is below dtau, and its primitive quartets are screened against prim_tau / max|P|,
// so that a build from a small density (a difference of densities) keeps the absolute error bound of
// the build from a density of order one.
template <typename A>
__device__ __forceinline__ float density_block_max(const A& a, const PairHdr& hb, const PairHdr& hk)
{
    const int n = a.n_sh;
    const float* d = a.dsh;
    float m = fmaxf(fmaxf(d[hk.A * n + hk.B], d[hb.A * n + hb.B]), fmaxf(d[hb.B * n + hk.B], d[hb.A * n + hk.A]));
    return fmaxf(m, fmaxf(d[hb.B * n + hk.A], d[hb.A * n + hk.B]));
}

// Number of surviving primitive quartets of a shell quartet (the length of its primitive staircase):
// bra primitive ib pairs with the first c(ib) ket primitives whose bound product reaches ptau, c
// non-increasing as the records are sorted by bound.
template <typename real, typename KV>
__device__ __forceinline__ int staircase_total(const PrimPair<real>* __restrict__ bpp, int nbp, const KV& kv,
                                               int nkp, float ptau)
{
    int total = 0;
    for (int ib = 0, c = nkp; ib < nbp; ib++) {
        const float Bb = bpp[ib].B;
        while (c > 0 && Bb * kv.B(c - 1) < ptau) c--;
        if (c == 0) break;
        total += c;
    }
    return total;
}

// Quartet scheduling inside a warp.  Each warp takes a window of W = R * 32 / GK consecutive quartets of
// the launch (R rounds of 32 / GK quartets), computes every quartet's staircase length, sorts the window by
// it (bitonic sort in the warp's shared memory; key = length << 16 | position) and runs the R rounds in
// sorted order, so that the lanes of a round have primitive loops of similar length and idle less while
// the longest one runs.  R is the largest power of two <= kSortRounds that still gives every warp two
// windows; with R = 1 the window is one round in launch order.
constexpr int kSortRounds = 8;

template <typename real, bool SOA>
__device__ __forceinline__ unsigned quartet_sort_key(const EriArgs& a, const PrimPair<real>* prims, long long q,
                                                     int pos, float ptau)
{
    if (q >= a.n_quartets) return (unsigned)pos;
    const long long c = q >> kChunkShift;
    const int b = a.chunk ? find_bra_in(a.offsets, a.chunk[c], a.chunk[c + 1], q) : find_bra(a.offsets, a.n_bra, q);
    const int k = (int)(q - a.offsets[b]) + (a.kstart ? a.kstart[b] : 0);
    const PairHdr& hb = a.bhdr[b];
    const PairHdr& hk = a.khdr[k];
    int t;
    if constexpr (SOA)
        t = staircase_total(prims + hb.prim0, hb.nprim, KetSoa<real>{(const real*)a.kt + k, a.ktB + k, a.kstride},
                            hk.nprim, ptau);
    else
        t = staircase_total(prims + hb.prim0, hb.nprim, KetAos<real>{prims + hk.prim0}, hk.nprim, ptau);
    return ((unsigned)min(t, 0xFFFF) << 16) | (unsigned)pos;
}

// ascending bitonic sort of n (a power of two) keys by the 32 lanes of one warp
__device__ __forceinline__ void warp_bitonic_sort(unsigned* k, int n, int lane32)
{
    for (int size = 2; size <= n; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane32; i < (n >> 1); i += 32) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const unsigned x = k[lo], y = k[hi];
                if ((x > y) == ((lo & size) == 0)) {
                    k[lo] = y;
                    k[hi] = x;
                }
            }
            __syncwarp();
        }
}

}  // namespace hf

// Kernels and host launchers of one class.  The digestion weight of a unique
// shell quartet is f = 1/((1+d_AB)(1+d_CD)(1+d_AB,CD)).
#define ERI_KERNEL_BODY(QFN, SORT)                                                                           \
    {                                                                                                        \
        if (a.bad && *a.bad) return; /* rejected density: grid-uniform exit, outputs untouched */            \
        const PrimPair<real>* prims = (const PrimPair<real>*)(sizeof(real) == 8 ? a.prims64 : a.prims32);   \
        const real* P = (const real*)(sizeof(real) == 8 ? (const void*)a.P64 : (const void*)a.P32);          \
        const real* bt = (const real*)(sizeof(real) == 8 ? (const void*)a.boys64 : (const void*)a.boys32);  \
        const float ptau = (float)a.prim_tau;                                                                \
        const size_t cofs = a.n_copies > 1 ? (size_t)(blockIdx.x % a.n_copies) * a.copy_stride : 0;          \
        double* const Jt = a.Jt + cofs;                                                                      \
        double* const Kt = a.Kt + cofs;                                                                      \
        unsigned nprimq = 0;                                                                                 \
        constexpr int gpw = 32 / GK;                                                                         \
        constexpr bool kSort = (SORT) && sizeof(real) == 8; /* FP32 launches run in launch order */         \
        constexpr int kWmax = kSort ? kSortRounds * gpw : 1;                                                 \
        __shared__ unsigned skeys[(kEriThreads / 32) * kWmax];                                               \
        unsigned* const wkeys = skeys + (threadIdx.x >> 5) * kWmax;                                          \
        const int lane32 = threadIdx.x & 31;                                                                 \
        const int lane = threadIdx.x & (GK - 1);                                                             \
        const int grp = lane32 / GK;                                                                         \
        const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;                      \
        const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;                                   \
        int R = 1; /* rounds per window (grid-uniform; 1 in kernels compiled without the sort) */            \
        if (kSort && a.sort_work)                                                                            \
            while (R < kSortRounds && (long long)(2 * R) * gpw * nwarps * 2 <= a.n_quartets - a.q_begin) R *= 2; \
        const int W = R * gpw;                                                                               \
        for (long long wb = a.q_begin + warp * W; wb < a.n_quartets; wb += nwarps * W) { /* warp-uniform */  \
            if (kSort && R > 1) {                                                                            \
                for (int pos = lane32; pos < W; pos += 32)                                                   \
                    wkeys[pos] = quartet_sort_key<real, SOA>(a, prims, wb + pos, pos, ptau);                 \
                __syncwarp();                                                                                \
                warp_bitonic_sort(wkeys, W, lane32);                                                         \
            }                                                                                                \
            for (int r = 0; r < R; r++) {                                                                    \
                const int s = r * gpw + grp;                                                                 \
                const long long q = wb + (kSort && R > 1 ? (long long)(wkeys[s] & 0xFFFFu) : (long long)s);  \
                const bool valid = q < a.n_quartets;                                                         \
                PairHdr hb, hk;                                                                              \
                real f = real(1);                                                                            \
                int k = 0;                                                                                   \
                if (valid) {                                                                                 \
                    const long long c = q >> kChunkShift;                                                    \
                    const int b = a.chunk ? find_bra_in(a.offsets, a.chunk[c], a.chunk[c + 1], q)             \
                                          : find_bra(a.offsets, a.n_bra, q);                                 \
                    k = (int)(q - a.offsets[b]) + (a.kstart ? a.kstart[b] : 0);                              \
                    hb = a.bhdr[b];                                                                          \
                    hk = a.khdr[k];                                                                          \
                    if (hb.A == hb.B) f *= real(0.5);                                                        \
                    if (hk.A == hk.B) f *= real(0.5);                                                        \
                    if (a.same && b == k) f *= real(0.5);                                                    \
                } else {                                                                                     \
                    hb = hk = a.bhdr[0];                                                                     \
                }                                                                                            \
                bool live = valid;                                                                           \
                float pt = ptau;                                                                             \
                if (a.dsh) { /* density-weighted screening (warp-uniform branch) */                          \
                    const float dm = valid ? density_block_max(a, hb, hk) : 0.0f;                            \
                    live = valid && 4.0f * (float)(hb.Q * hk.Q) * dm >= a.dtau;                              \
                    pt = ptau / fmaxf(dm, 1e-30f);                                                           \
                }                                                                                            \
                if constexpr (SOA) {                                                                         \
                    const KetSoa<real> kv{(const real*)a.kt + k, a.ktB + k, a.kstride};                      \
                    nprimq += QFN<real, GK>(hb, hk, kv, prims, bt, P, a.N, f, Jt, Kt, nullptr, pt, lane,     \
                                            live);                                                           \
                } else {                                                                                     \
                    const KetAos<real> kv{prims + hk.prim0};                                                 \
                    nprimq += QFN<real, GK>(hb, hk, kv, prims, bt, P, a.N, f, Jt, Kt, nullptr, pt, lane,     \
                                            live);                                                           \
                }                                                                                            \
            }                                                                                                \
            __syncwarp();                                                                                    \
        }                                                                                                    \
        if (a.prim_count) {                                                                                  \
            const unsigned long long w = __reduce_add_sync(0xffffffffu, nprimq);                            \
            if ((threadIdx.x & 31) == 0 && w) atomicAdd(a.prim_count, w);                                    \
        }                                                                                                    \
    }

#define ERI_CLASS_KERNELS(NAME, X, Y, GL)                                                                    \
    template <typename real, int GK, bool SOA>                                                               \
    __global__ void __launch_bounds__(kEriThreads) k_eri_##NAME(const EriArgs a)                            \
    ERI_KERNEL_BODY(quartet_##NAME, true)                                                                    \
    void launch_eri_##NAME(const EriArgs& a, int use_f32, int grid, int block, cudaStream_t s, int lanes)   \
    {                                                                                                        \
        if (use_f32)                                                                                         \
            k_eri_##NAME<float, 1, true><<<grid, block, 0, s>>>(a);                                          \
        else if (lanes > 1)                                                                                  \
            k_eri_##NAME<double, (GL), false><<<grid, block, 0, s>>>(a);                                     \
        else                                                                                                 \
            k_eri_##NAME<double, 1, false><<<grid, block, 0, s>>>(a);                                        \
    }                                                                                                        \
    size_t local_bytes_##NAME()                                                                              \
    {                                                                                                        \
        cudaFuncAttributes fa;                                                                               \
        size_t m = 0;                                                                                        \
        const void* fns[] = {(const void*)k_eri_##NAME<double, 1, false>, (const void*)k_eri_##NAME<double, (GL), false>, \
                             (const void*)k_eri_##NAME<float, 1, true>, (const void*)k_eri_batch_##NAME};   \
        for (const void* fn : fns)                                                                           \
            if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && fa.localSizeBytes > m) m = fa.localSizeBytes; \
        cudaGetLastError();                                                                                  \
        return m;                                                                                            \
    }

// Rys-quadrature variant of a class: the same kernel body around quartet_rys_NAME, FP64 and the ket
// tables only (launch_eri_rys_NAME is given FP64 launches with a.kt set).
#define ERI_RYS_KERNELS(NAME, GL)                                                                            \
    template <typename real, int GK, bool SOA>                                                               \
    __global__ void __launch_bounds__(kEriThreads) k_eri_rys_##NAME(const EriArgs a)                        \
    ERI_KERNEL_BODY(quartet_rys_##NAME, false)                                                               \
    void launch_eri_rys_##NAME(const EriArgs& a, int, int grid, int block, cudaStream_t s, int lanes)       \
    {                                                                                                        \
        if (lanes > 1)                                                                                       \
            k_eri_rys_##NAME<double, (GL), true><<<grid, block, 0, s>>>(a);                                  \
        else                                                                                                 \
            k_eri_rys_##NAME<double, 1, true><<<grid, block, 0, s>>>(a);                                     \
    }                                                                                                        \
    size_t local_bytes_rys_##NAME()                                                                          \
    {                                                                                                        \
        cudaFuncAttributes fa;                                                                               \
        size_t m = 0;                                                                                        \
        if (cudaFuncGetAttributes(&fa, k_eri_rys_##NAME<double, 1, true>) == cudaSuccess) m = fa.localSizeBytes; \
        if (cudaFuncGetAttributes(&fa, k_eri_rys_##NAME<double, (GL), true>) == cudaSuccess && fa.localSizeBytes > m) \
            m = fa.localSizeBytes;                                                                           \
        cudaGetLastError();                                                                                  \
        return m;                                                                                            \
    }

// Schwarz bounds of the pairs of a diagonal class: Q = sqrt(max |(ab|ab)|) of the
// contracted pair (item 0 of each pair) and B = the same bound of each primitive pair
// alone (items 1..a.items-1), one thread per item so that the high-L classes'
// single-thread latency is paid once per pair, not once per primitive pair.
#define SCHWARZ_KERNEL(NAME)                                                                                 \
    __global__ void __launch_bounds__(kEriThreads) k_schwarz_##NAME(const SchwarzArgs a)                    \
    {                                                                                                        \
        const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;                                \
        if (t >= (long long)a.n * a.items) return;                                                           \
        const int pid = a.ids[t / a.items];                                                                  \
        const int item = (int)(t % a.items);                                                                 \
        PairHdr h = a.pairs[pid];                                                                            \
        if (item > h.nprim) return;                                                                          \
        const PrimPair<double>* pr = (const PrimPair<double>*)a.prims64;                                     \
        if (item > 0) { /* bound of one primitive pair alone */                                              \
            h.prim0 += item - 1;                                                                             \
            h.nprim = 1;                                                                                     \
        }                                                                                                    \
        double qm = 0.0;                                                                                     \
        quartet_##NAME<double, 1>(h, h, KetAos<double>{pr + h.prim0}, pr, a.boys64, nullptr, 0, 1.0, nullptr,  \
                                  nullptr, &qm, 0.0f, 0, true);                                              \
        if (item == 0)                                                                                       \
            a.Q[pid] = sqrt(qm);                                                                             \
        else                                                                                                 \
            a.Bprim[h.prim0] = sqrt(qm);                                                                     \
    }                                                                                                        \
    void launch_schwarz_##NAME(const SchwarzArgs& a, int block, cudaStream_t s)                             \
    {                                                                                                        \
        const long long items = (long long)a.n * a.items;                                                    \
        if (items > 0) k_schwarz_##NAME<<<(unsigned)((items + block - 1) / block), block, 0, s>>>(a);        \
    }

// Batched build: one persistent kernel per class over many molecules.  Warps
// take chunks of the batch's quartet index space from a device counter (the
// GPU analogue of the paper's dynamic load balancing, ddi_dlbnext); a quartet
// index resolves to (molecule, bra, ket) by two binary searches.
#define ERI_BATCH_KERNEL(NAME, GL_UNUSED)                                                                           \
    __global__ void __launch_bounds__(256) k_eri_batch_##NAME(const BatchArgs a)                            \
    {                                                                                                        \
        const int wl = threadIdx.x & 31;                                                                     \
        constexpr int GL = 1; /* batches have enough quartets per class for one thread per quartet */        \
        const int lane = 0;                                                                                  \
        const int grp = wl;                                                                                  \
        constexpr int gpw = 32;                                                                              \
        const float ptau = (float)a.prim_tau;                                                                \
        for (;;) {                                                                                           \
            unsigned long long base = 0;                                                                     \
            if (wl == 0) base = atomicAdd(a.counter, (unsigned long long)a.chunk);                          \
            base = __shfl_sync(0xffffffffu, base, 0);                                                        \
            if (base >= (unsigned long long)a.n_total) break;                                                \
            const long long end = min((long long)base + a.chunk, a.n_total);                                 \
            for (long long wq = (long long)base; wq < end; wq += gpw) { /* warp-uniform */                  \
                const long long q = wq + grp;                                                                \
                const bool valid = q < end;                                                                  \
                const int m = find_bra(a.mol_off, a.n_mol, valid ? q : (long long)base);                     \
                const MolClass mc = a.mols[m];                                                               \
                PairHdr hb, hk;                                                                              \
                double f = 1.0;                                                                              \
                if (valid) {                                                                                 \
                    const long long ql = q - a.mol_off[m];                                                   \
                    const int b = find_bra(mc.offsets, mc.n_bra, ql);                                        \
                    const int k = (int)(ql - mc.offsets[b]);                                                 \
                    hb = mc.pairs[mc.bra[b]];                                                                \
                    hk = mc.pairs[mc.ket[k]];                                                                \
                    if (hb.A == hb.B) f *= 0.5;                                                              \
                    if (hk.A == hk.B) f *= 0.5;                                                              \
                    if (mc.same && b == k) f *= 0.5;                                                         \
                } else {                                                                                     \
                    hb = hk = mc.pairs[mc.bra[0]];                                                           \
                }                                                                                            \
                const PrimPair<double>* mp = (const PrimPair<double>*)mc.prims64;                            \
                quartet_##NAME<double, (GL)>(hb, hk, KetAos<double>{mp + hk.prim0}, mp, a.boys64, mc.P64, mc.N, f, \
                                             mc.Jt, mc.Kt, nullptr, ptau, lane, valid);                      \
            }                                                                                                \
        }                                                                                                    \
    }                                                                                                        \
    void launch_eri_batch_##NAME(const BatchArgs& a, int grid, int block, cudaStream_t s)                   \
    {                                                                                                        \
        k_eri_batch_##NAME<<<grid, block, 0, s>>>(a);                                                        \
    }

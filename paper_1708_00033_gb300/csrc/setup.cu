// Per-geometry setup kernels: Boys tables, basis normalisation, shell-pair
// records with primitive-pair data, Cauchy-Schwarz bounds, significant-pair
// lists sorted by (angular class, bound), and the per-class quartet schedule
// (ket prefix per bra, FP64/FP32 split).  Algorithm 1's schwartz(i,j,k,l)
// test and Algorithm 3's (i,j) pre-screen become cuts on these sorted lists.
#include <math.h>

#include "eri_common.cuh"
#include "setup.cuh"

namespace hf {

// ------------------------------------------------------------ Boys table --
// F_m(T_k), m = 0..14, at the grid points T_k = k/512 (FP64 table, T < 64) and k/32 (FP32 table): the series
//   F_M(T) = exp(-T) sum_i (2T)^i / ((2M+1)(2M+3)...(2M+2i+1))
// for the top order (compensated summation of its positive terms), then the
// downward recursion F_m = (2T F_{m+1} + exp(-T)) / (2m+1); stored as the
// Taylor coefficients F_{m+j}(T_k) / j! and exp(-T_k) / j! (layout in eri_common.cuh).
__device__ static void boys_row(double T, double* F, double& e)
{
    const int M = 14;
    double term = 1.0 / (2 * M + 1), sum = term, comp = 0.0;
    for (int i = 1; i < 1000; i++) {
        term *= 2.0 * T / (2 * M + 2 * i + 1);
        const double y = term - comp;
        const double t = sum + y;
        comp = (t - sum) - y;
        sum = t;
        if (term < 1e-21 * sum) break;
    }
    e = exp(-T);
    F[M] = e * sum;
    for (int m = M - 1; m >= 0; m--) F[m] = (2.0 * T * F[m + 1] + e) / (2 * m + 1);
}

__global__ void k_boys_table(double* t64, float* t32)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double F[15], e;
    if (k < kBoysRowsA) {
        boys_row(k / 512.0, F, e);
    } else if (k < kBoysRows64) {
        // region B: the asymptotic form at T_k = 2^e (1 + i / 4096)
        const int r = k - kBoysRowsA;
        const double Tk = ldexp(1.0 + (r & ((1 << kBoysSubBits) - 1)) / (double)(1 << kBoysSubBits),
                                kBoysBinade0 + (r >> kBoysSubBits));
        F[0] = 0.5 * sqrt(M_PI / Tk);
        for (int m = 0; m < 14; m++) F[m + 1] = F[m] * (2 * m + 1) / (2.0 * Tk);
        e = 0.0;
    }
    if (k < kBoysRows64) {
        double* r = t64 + (size_t)k * kBoysStride64;
        double fact = 1.0;
        for (int j = 0; j <= 4; j++) {
            if (j > 0) fact *= j;
            for (int m = 0; m <= 8; m++) r[5 * m + j] = F[m + j] / fact;
            r[kBoysExp64 + j] = e / fact;
        }
    }
    if (k < kBoysRows32) {
        boys_row(k / 32.0, F, e);
        float* q = t32 + (size_t)k * kBoysStride32;
        for (int i = 0; i < kBoysStride32; i++) q[i] = 0.0f;
        double fact = 1.0;
        for (int j = 0; j <= 4; j++) {
            if (j > 0) fact *= j;
            if (j <= 3)
                for (int m = 0; m <= 8; m++) q[4 * m + j] = (float)(F[m + j] / fact);
            q[kBoysExp32 + j] = (float)(e / fact);
        }
    }
}

int build_boys_tables(double* t64, float* t32, cudaStream_t s)
{
    k_boys_table<<<(kBoysRows64 + 127) / 128, 128, 0, s>>>(t64, t32);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ----------------------------------------------------- basis normalisation --
// Shell-level primitive factor (2a/pi)^{3/4} (4a)^{l/2} times the caller's
// coefficient, rescaled so that the contracted function has unit norm.  The
// Cartesian component factor 1/sqrt((2i-1)!!(2j-1)!!(2k-1)!!) is applied to
// P and to J/K outside the ERI kernels (comp_norm).
__global__ void k_shell_coef(int n_sh, const int* __restrict__ l, const int* __restrict__ nprim,
                             const int* __restrict__ prim0, const double* __restrict__ exps,
                             const double* __restrict__ coefs, double* __restrict__ cn)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sh) return;
    const int L = l[s], n = nprim[s], o = prim0[s];
    double ss = 0.0;
    for (int a = 0; a < n; a++)
        for (int b = 0; b < n; b++) {
            const double ea = exps[o + a], eb = exps[o + b];
            ss += coefs[o + a] * coefs[o + b] * pow(2.0 * sqrt(ea * eb) / (ea + eb), L + 1.5);
        }
    const double r = 1.0 / sqrt(ss);
    for (int a = 0; a < n; a++) {
        const double e = exps[o + a];
        cn[o + a] = coefs[o + a] * pow(2.0 * e / M_PI, 0.75) * pow(4.0 * e, 0.5 * L) * r;
    }
}

__global__ void k_comp_norm(int n_sh, const int* __restrict__ l, const int* __restrict__ bf0, double* __restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sh) return;
    const int L = l[s], b = bf0[s];
    if (L < 2) {
        for (int c = 0; c < (L + 1) * (L + 2) / 2; c++) out[b + c] = 1.0;
    } else {  // xx xy xz yy yz zz
        const double r3 = 0.57735026918962576451;
        out[b + 0] = r3;
        out[b + 1] = 1.0;
        out[b + 2] = 1.0;
        out[b + 3] = r3;
        out[b + 4] = 1.0;
        out[b + 5] = r3;
    }
}

// ------------------------------------------------------------- shell pairs --
__device__ __forceinline__ void decode_pair(long long t, int& i, int& j)
{
    long long ii = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (ii * (ii + 1) / 2 > t) ii--;
    while ((ii + 1) * (ii + 2) / 2 <= t) ii++;
    i = (int)ii;
    j = (int)(t - ii * (ii + 1) / 2);
}

__global__ void k_build_pairs(long long n_pairs, int maxpp, const int* __restrict__ l, const int* __restrict__ atom,
                              const int* __restrict__ bf0, const int* __restrict__ nprim, const int* __restrict__ prim0,
                              const double* __restrict__ exps, const double* __restrict__ cn,
                              const double* __restrict__ xyz, PairHdr* __restrict__ pairs,
                              PrimPair<double>* __restrict__ p64, PrimPair<float>* __restrict__ p32,
                              int* __restrict__ pclass)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_pairs) return;
    int i, j;
    decode_pair(t, i, j);
    const int A = l[i] >= l[j] ? i : j;
    const int B = l[i] >= l[j] ? j : i;
    const int la = l[A], lb = l[B];
    const double Ax = xyz[3 * atom[A]], Ay = xyz[3 * atom[A] + 1], Az = xyz[3 * atom[A] + 2];
    const double Bx = xyz[3 * atom[B]], By = xyz[3 * atom[B] + 1], Bz = xyz[3 * atom[B] + 2];
    const double ABx = Ax - Bx, ABy = Ay - By, ABz = Az - Bz;
    const double R2 = ABx * ABx + ABy * ABy + ABz * ABz;
    PairHdr h;
    h.A = A;
    h.B = B;
    h.bfA = bf0[A];
    h.bfB = bf0[B];
    h.prim0 = (int)(t * maxpp);
    h.nprim = nprim[A] * nprim[B];
    h.ABx = ABx;
    h.ABy = ABy;
    h.ABz = ABz;
    h.Q = 0.0;
    h.ABfx = (float)ABx;
    h.ABfy = (float)ABy;
    h.ABfz = (float)ABz;
    pairs[t] = h;
    pclass[t] = la * (la + 1) / 2 + lb;
    const double c52 = sqrt(2.0) * pow(M_PI, 1.25);  // sqrt(2) pi^(5/4)
    int k = 0;
    for (int ka = 0; ka < nprim[A]; ka++) {
        const double a = exps[prim0[A] + ka], ca = cn[prim0[A] + ka];
        for (int kb = 0; kb < nprim[B]; kb++, k++) {
            const double b = exps[prim0[B] + kb], cb = cn[prim0[B] + kb];
            const double p = a + b, ip = 1.0 / p;
            PrimPair<double> r;
            r.p = p;
            r.Px = (a * Ax + b * Bx) * ip;
            r.Py = (a * Ay + b * By) * ip;
            r.Pz = (a * Az + b * Bz) * ip;
            r.PAx = r.Px - Ax;
            r.PAy = r.Py - Ay;
            r.PAz = r.Pz - Az;
            r.K = ca * cb * exp(-a * b * ip * R2) * c52 * ip;
            r.oo2p = 0.5 * ip;
            r.B = 0.0f;  // set by the Schwarz pass; 0 never stops a primitive loop whose threshold is 0
            p64[t * maxpp + k] = r;
            PrimPair<float> f;
            f.p = (float)r.p;
            f.Px = (float)r.Px;
            f.Py = (float)r.Py;
            f.Pz = (float)r.Pz;
            f.PAx = (float)r.PAx;
            f.PAy = (float)r.PAy;
            f.PAz = (float)r.PAz;
            f.K = (float)r.K;
            f.oo2p = (float)r.oo2p;
            f.B = 0.0f;
            p32[t * maxpp + k] = f;
        }
    }
    (void)la;
}

__global__ void k_class_count(long long n, const int* __restrict__ pclass, unsigned long long* __restrict__ cnt)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) atomicAdd(&cnt[pclass[t]], 1ull);
}

// all pairs of one class (unordered list), for the Schwarz pass
__global__ void k_class_scatter_all(long long n, const int* __restrict__ pclass, int X, unsigned* __restrict__ cursor,
                                    int* __restrict__ ids)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && pclass[t] == X) ids[atomicAdd(cursor, 1u)] = (int)t;
}

__global__ void k_copy_q(long long n, const double* __restrict__ Q, PairHdr* __restrict__ pairs)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) pairs[t].Q = Q[t];
}

// max of non-negative doubles via their order-preserving bit patterns
__global__ void k_max_q(long long n, const double* __restrict__ Q, unsigned long long* __restrict__ out)
{
    __shared__ double sm[256];
    double m = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        m = fmax(m, Q[t]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sm[0]));
}

// significant pairs of class X: Q * Qmax >= tau (tau = 0 keeps all)
__global__ void k_class_scatter_sig(long long n, const int* __restrict__ pclass, const double* __restrict__ Q, int X,
                                    double qmax, double tau, unsigned* __restrict__ cursor, double* __restrict__ key,
                                    int* __restrict__ val)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n || pclass[t] != X) return;
    const double q = Q[t];
    if (tau > 0.0 && !(q * qmax >= tau)) return;
    const unsigned pos = atomicAdd(cursor, 1u);
    key[pos] = q;
    val[pos] = (int)t;
}

__global__ void k_fill_pad(int from, int n_pad, double* key, int* val)
{
    const int t = from + blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_pad) {
        key[t] = -1.0;
        val[t] = 0x7fffffff;
    }
}

// one compare-exchange step of a bitonic sort into (key descending, val ascending)
__global__ void k_bitonic_step(double* __restrict__ key, int* __restrict__ val, unsigned n_pad, unsigned j, unsigned k)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    const unsigned l = i ^ j;
    if (l <= i) return;
    const double ki = key[i], kl = key[l];
    const int vi = val[i], vl = val[l];
    const bool l_first = (kl > ki) || (kl == ki && vl < vi);
    const bool asc = (i & k) == 0;
    if (asc ? l_first : !l_first) {
        key[i] = kl;
        key[l] = ki;
        val[i] = vl;
        val[l] = vi;
    }
}

int bitonic_sort_desc(double* key, int* val, int n, int n_pad, cudaStream_t s)
{
    if (n_pad > n) k_fill_pad<<<(n_pad - n + 255) / 256, 256, 0, s>>>(n, n_pad, key, val);
    for (unsigned k = 2; k <= (unsigned)n_pad; k <<= 1)
        for (unsigned j = k >> 1; j > 0; j >>= 1)
            k_bitonic_step<<<(n_pad + 255) / 256, 256, 0, s>>>(key, val, (unsigned)n_pad, j, k);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Attach the primitive-pair bounds and order each pair's primitive pairs by
// bound, largest first, so that the ERI loops can stop at the first
// primitive quartet whose bound product falls below the primitive threshold.
__global__ void k_sort_prims(long long n_pairs, const PairHdr* __restrict__ pairs, const double* __restrict__ Bprim,
                             PrimPair<double>* __restrict__ p64, PrimPair<float>* __restrict__ p32)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_pairs) return;
    const int o = pairs[t].prim0, n = pairs[t].nprim;
    for (int k = 0; k < n; k++) {
        p64[o + k].B = (float)Bprim[o + k];
        p32[o + k].B = (float)Bprim[o + k];
    }
    for (int i = 1; i < n; i++) {  // insertion sort, descending B
        const PrimPair<double> r = p64[o + i];
        const PrimPair<float> f = p32[o + i];
        int j = i - 1;
        while (j >= 0 && p64[o + j].B < r.B) {
            p64[o + j + 1] = p64[o + j];
            p32[o + j + 1] = p32[o + j];
            j--;
        }
        p64[o + j + 1] = r;
        p32[o + j + 1] = f;
    }
}

// Ket table of one pair class: record i of the class's k-th pair (ids[k]) at field-major position
// (9 i + f) stride + k of the FP64 and FP32 field rows, its bound at i stride + k; records past the pair's
// primitive count are zero (bound 0, so every primitive screen skips them).
__global__ void k_ket_table(int n, int maxpp, long long stride, const int* __restrict__ ids,
                            const PairHdr* __restrict__ pairs, const PrimPair<double>* __restrict__ p64,
                            const PrimPair<float>* __restrict__ p32, double* __restrict__ t64, float* __restrict__ t32,
                            float* __restrict__ tB)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * maxpp) return;
    const int i = (int)(t / n), k = (int)(t % n);  // consecutive threads: consecutive kets (coalesced writes)
    const PairHdr h = pairs[ids[k]];
    PrimPair<double> r{};
    PrimPair<float> f{};
    if (i < h.nprim) {
        r = p64[h.prim0 + i];
        f = p32[h.prim0 + i];
    }
    const double v64[9] = {r.p, r.Px, r.Py, r.Pz, r.PAx, r.PAy, r.PAz, r.K, r.oo2p};
    const float v32[9] = {f.p, f.Px, f.Py, f.Pz, f.PAx, f.PAy, f.PAz, f.K, f.oo2p};
#pragma unroll
    for (int x = 0; x < 9; x++) {
        t64[((long long)i * 9 + x) * stride + k] = v64[x];
        t32[((long long)i * 9 + x) * stride + k] = v32[x];
    }
    tB[(long long)i * stride + k] = i < h.nprim ? r.B : 0.0f;
}

// out[k] = pairs[ids[k]]: a class list's pair headers in list order
__global__ void k_gather_headers(int n, const int* __restrict__ ids, const PairHdr* __restrict__ pairs,
                                 PairHdr* __restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = pairs[ids[k]];
}

int launch_gather_headers(int n, const int* ids, const PairHdr* pairs, PairHdr* out, cudaStream_t s)
{
    if (n > 0) k_gather_headers<<<(n + 255) / 256, 256, 0, s>>>(n, ids, pairs, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_ket_table(int n, int maxpp, long long stride, const int* ids, const PairHdr* pairs, const void* p64,
                     const void* p32, double* t64, float* t32, float* tB, cudaStream_t s)
{
    const long long items = (long long)n * maxpp;
    if (items > 0)
        k_ket_table<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(n, maxpp, stride, ids, pairs,
                                                                    (const PrimPair<double>*)p64,
                                                                    (const PrimPair<float>*)p32, t64, t32, tB);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sort_prims(long long n_pairs, const PairHdr* pairs, const double* Bprim, void* p64, void* p32, cudaStream_t s)
{
    if (n_pairs > 0)
        k_sort_prims<<<(unsigned)((n_pairs + 127) / 128), 128, 0, s>>>(n_pairs, pairs, Bprim, (PrimPair<double>*)p64,
                                                                     (PrimPair<float>*)p32);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------- quartet schedule --
// exclusive scan of n counts into out[0..n] (single block, chunked)
__global__ void k_scan(int n, const long long* __restrict__ in, long long* __restrict__ out)
{
    __shared__ long long sm[1024];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long v = i < n ? in[i] : 0;
        sm[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            const long long add = threadIdx.x >= (unsigned)off ? sm[threadIdx.x - off] : 0;
            __syncthreads();
            sm[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n) out[i] = carry + sm[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += sm[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

// --------------------------------------------- all-class scatter and counts --
struct SegBase {
    long long base[8];
};

__global__ void k_fill_keys(long long n, double* __restrict__ key, int* __restrict__ val)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        key[t] = -1.0;
        val[t] = 0x7fffffff;
    }
}

// significant pairs (Q * Qmax >= tau, or all when tau = 0) into their class segment
__global__ void k_sig_scatter(long long n, const int* __restrict__ pclass, const double* __restrict__ Q,
                              const unsigned long long* __restrict__ qmax_bits, double tau, SegBase seg,
                              unsigned* __restrict__ cursor, double* __restrict__ key, int* __restrict__ val)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double q = Q[t];
    if (tau > 0.0) {
        const double qmax = __longlong_as_double((long long)*qmax_bits);
        if (!(q * qmax >= tau)) return;
    }
    const int c = pclass[t];
    const unsigned pos = atomicAdd(&cursor[c], 1u);
    key[seg.base[c] + pos] = q;
    val[seg.base[c] + pos] = (int)t;
}

int launch_sig_scatter(long long n_pairs, long long n_seg, const int* pclass, const double* Q,
                       const unsigned long long* qmax_bits, double tau, const size_t* seg_host, unsigned* cursor,
                       double* key, int* val, cudaStream_t s)
{
    SegBase sb;
    for (int c = 0; c < 8; c++) sb.base[c] = c < 7 ? (long long)seg_host[c] : 0;
    if (n_seg > 0) k_fill_keys<<<(unsigned)((n_seg + 255) / 256), 256, 0, s>>>(n_seg, key, val);
    if (n_pairs > 0)
        k_sig_scatter<<<(unsigned)((n_pairs + 255) / 256), 256, 0, s>>>(n_pairs, pclass, Q, qmax_bits, tau, sb, cursor,
                                                                       key, val);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// For bra b of class X: kets of class Y (sorted by Q descending) with Q_b Q_k >= tau form a
// prefix; when X == Y only kets k <= b are unique.  The prefix splits into an FP64 head
// (Q_b Q_k >= cutoff) and an FP32 tail.  The list lengths are read on the device (entries
// b >= n_bra get zero counts), so the schedule needs no host round trip.
__global__ void k_ket_counts_dev(int cap, const unsigned* __restrict__ n_bra_p, const double* __restrict__ qb,
                                 const unsigned* __restrict__ n_ket_p, const double* __restrict__ qk, int same,
                                 double tau, double cutoff, long long* __restrict__ c64, long long* __restrict__ c32,
                                 int* __restrict__ kstart32)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= cap) return;
    const int n_bra = (int)*n_bra_p, n_ket = (int)*n_ket_p;
    if (b >= n_bra || n_ket == 0) {
        c64[b] = 0;
        c32[b] = 0;
        kstart32[b] = 0;
        return;
    }
    const double Qb = qb[b];
    int n = n_ket;
    if (tau > 0.0) {
        int lo = 0, hi = n_ket;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Qb * qk[mid] >= tau)
                lo = mid + 1;
            else
                hi = mid;
        }
        n = lo;
    }
    if (same && n > b + 1) n = b + 1;
    int n64 = n;
    if (cutoff > 0.0) {
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Qb * qk[mid] >= cutoff)
                lo = mid + 1;
            else
                hi = mid;
        }
        n64 = lo;
    }
    c64[b] = n64;
    c32[b] = n - n64;
    kstart32[b] = n64;
}

int launch_ket_counts_dev(int cap, const unsigned* n_bra, const double* qb, const unsigned* n_ket, const double* qk,
                          int same, double tau, double cutoff, long long* c64, long long* c32, int* kstart32,
                          cudaStream_t s)
{
    if (cap > 0)
        k_ket_counts_dev<<<(cap + 255) / 256, 256, 0, s>>>(cap, n_bra, qb, n_ket, qk, same, tau, cutoff, c64, c32,
                                                            kstart32);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_shell_coef(int n_sh, const int* l, const int* nprim, const int* prim0, const double* exps,
                      const double* coefs, double* cn, cudaStream_t s)
{
    if (n_sh > 0) k_shell_coef<<<(n_sh + 255) / 256, 256, 0, s>>>(n_sh, l, nprim, prim0, exps, coefs, cn);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_comp_norm(int n_sh, const int* l, const int* bf0, double* out, cudaStream_t s)
{
    if (n_sh > 0) k_comp_norm<<<(n_sh + 255) / 256, 256, 0, s>>>(n_sh, l, bf0, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_build_pairs(long long n_pairs, int maxpp, const int* l, const int* atom, const int* bf0, const int* nprim,
                       const int* prim0, const double* exps, const double* cn, const double* xyz, PairHdr* pairs,
                       void* p64, void* p32, int* pclass, cudaStream_t s)
{
    if (n_pairs == 0) return 0;
    k_build_pairs<<<(unsigned)((n_pairs + 127) / 128), 128, 0, s>>>(n_pairs, maxpp, l, atom, bf0, nprim, prim0, exps, cn,
                                                                  xyz, pairs, (PrimPair<double>*)p64,
                                                                  (PrimPair<float>*)p32, pclass);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_class_count(long long n, const int* pclass, unsigned long long* cnt, cudaStream_t s)
{
    if (n > 0) k_class_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, pclass, cnt);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_class_scatter_all(long long n, const int* pclass, int X, unsigned* cursor, int* ids, cudaStream_t s)
{
    if (n > 0) k_class_scatter_all<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, pclass, X, cursor, ids);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_copy_q(long long n, const double* Q, PairHdr* pairs, unsigned long long* qmax_bits, cudaStream_t s)
{
    if (n > 0) {
        k_copy_q<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, Q, pairs);
        k_max_q<<<256, 256, 0, s>>>(n, Q, qmax_bits);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_class_scatter_sig(long long n, const int* pclass, const double* Q, int X, double qmax, double tau,
                             unsigned* cursor, double* key, int* val, cudaStream_t s)
{
    if (n > 0)
        k_class_scatter_sig<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, pclass, Q, X, qmax, tau, cursor, key, val);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_scan(int n, const long long* in, long long* out, cudaStream_t s)
{
    k_scan<<<1, 1024, 0, s>>>(n, in, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Bra lookup table of one class and precision: entry c = bra of quartet min(c << kChunkShift, n - 1),
// c = 0 .. ((n - 1) >> kChunkShift) + 1, so that quartet q's bra lies in [t[q >> S], t[(q >> S) + 1]].
__global__ void k_chunk_bra(int n_bra, const long long* __restrict__ off, long long n, long long n_entries,
                            int* __restrict__ out)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_entries) return;
    const long long q = min(c << kChunkShift, n - 1);
    out[c] = find_bra(off, n_bra, q);
}

long long chunk_entries(long long n) { return n > 0 ? ((n - 1) >> kChunkShift) + 2 : 0; }

int launch_chunk_bra(int n_bra, const long long* off, long long n, int* out, cudaStream_t s)
{
    const long long e = chunk_entries(n);
    if (e > 0) k_chunk_bra<<<(unsigned)((e + 255) / 256), 256, 0, s>>>(n_bra, off, n, e, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hf

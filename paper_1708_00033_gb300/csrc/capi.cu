// C-ABI entry points (include/hf.h): argument checks, device memory, and the
// order of the setup and Fock-build kernels on the context's stream.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "eri_common.cuh"
#include "hf_internal.h"
#include "setup.cuh"

namespace hf {

static thread_local std::string g_err;

void set_error(int code, const std::string& msg)
{
    (void)code;
    g_err = msg;
}

int cuda_status(cudaError_t e, const char* what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return HF_E_CUDA;
}

int DevBuf::alloc(size_t n)
{
    release();
    owned = true;
    if (n == 0) n = 16;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        g_err = "device allocation of " + std::to_string(n) + " bytes failed";
        return HF_E_NOMEM;
    }
    bytes = n;
    return HF_OK;
}

void DevBuf::release()
{
    if (p && owned) cudaFree(p);
    p = nullptr;
    bytes = 0;
    owned = true;
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

#define TRY(x)                       \
    do {                             \
        int rc_ = (x);               \
        if (rc_ != HF_OK) return rc_; \
    } while (0)

#define KCHK(x)                                                                  \
    do {                                                                         \
        if ((x) != 0) return cuda_status(cudaGetLastError(), "kernel launch " #x); \
    } while (0)

size_t next_pow2(size_t n)
{
    size_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

int class_index(int X, int Y)
{
    for (int c = 0; c < kNumClasses; c++)
        if (kEriClasses[c].X == X && kEriClasses[c].Y == Y) return c;
    return -1;
}

}  // namespace

}  // namespace hf

using namespace hf;

extern "C" {

const char* hf_strerror(int status)
{
    switch (status) {
        case HF_OK: return "success";
        case HF_E_INVALID: return "invalid argument";
        case HF_E_UNSUPPORTED: return "unsupported input or device";
        case HF_E_NOMEM: return "out of memory";
        case HF_E_CUDA: return "CUDA runtime error";
        case HF_E_TIMEOUT: return "device wait timed out";
        case HF_E_NOCONV: return "SCF did not converge";
        default: return "unknown status";
    }
}

const char* hf_last_error(void) { return g_err.c_str(); }

int hf_create(hf_ctx** out, int device, void* cuda_stream)
{
    if (!out) return fail(HF_E_INVALID, "hf_create: ctx pointer is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(HF_E_UNSUPPORTED, "hf_create: no CUDA device");
    }
    if (device < 0 || device >= ndev) return fail(HF_E_INVALID, "hf_create: device index out of range");
    cudaDeviceProp prop;
    HF_CUDA(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(HF_E_UNSUPPORTED, "hf_create: library is built for sm_103a (GB300); device is sm_" +
                                          std::to_string(prop.major) + std::to_string(prop.minor));
    DeviceGuard g(device);
    hf_ctx* c = new hf_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->num_sms = prop.multiProcessorCount;
    int rc = c->boys64.alloc(sizeof(double) * kBoysRows64 * kBoysStride64);
    if (rc == HF_OK) rc = c->boys32.alloc(sizeof(float) * kBoysRows32 * kBoysStride32);
    if (rc == HF_OK && build_boys_tables(c->boys64.as<double>(), c->boys32.as<float>(), c->stream) != 0)
        rc = cuda_status(cudaGetLastError(), "boys table kernel");
    if (rc == HF_OK) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = cuda_status(e, "hf_create sync");
    }
    if (rc == HF_OK) {
        // Reserve per-thread local memory for the largest ERI kernel once, so that launches of the
        // spilling high-angular-momentum kernels do not grow and shrink the reservation each time.
        size_t need = 0;
        for (int ci = 0; ci < kNumClasses; ci++) {
            need = std::max(need, kEriClasses[ci].local_bytes());
            if (kEriClasses[ci].local_bytes_rys) need = std::max(need, kEriClasses[ci].local_bytes_rys());
        }
        size_t cur = 0;
        if (cudaDeviceGetLimit(&cur, cudaLimitStackSize) == cudaSuccess && need > cur)
            if (cudaDeviceSetLimit(cudaLimitStackSize, need) != cudaSuccess)
                rc = cuda_status(cudaGetLastError(), "hf_create: local memory reservation");
        cudaGetLastError();
    }
    // the allocation-free build's fixed scratch: looking its address up loads its module now, so that
    // the driver reserves that memory here and not inside an hf_fock_build_noalloc call
    if (rc == HF_OK) rc = noalloc_scratch_address(&c->noalloc_scratch);
    if (rc == HF_OK) {
        for (auto& ev : c->ev) {
            if (cudaEventCreate(&ev) != cudaSuccess) {
                rc = cuda_status(cudaGetLastError(), "cudaEventCreate");
                break;
            }
        }
        c->events_ready = (rc == HF_OK);
    }
    if (rc != HF_OK) {
        delete c;
        return rc;
    }
    *out = c;
    return HF_OK;
}

static void ctx_release(hf_ctx* c)
{
    DeviceGuard g(c->device);
    if (c->events_ready)
        for (auto& ev : c->ev)
            if (ev) cudaEventDestroy(ev);
    delete c;
}

void hf_destroy(hf_ctx* c)
{
    if (!c) return;
    if (c->n_systems > 0) {  // released together with its last system
        c->destroy_pending = true;
        return;
    }
    ctx_release(c);
}

}  // extern "C"

// Carves 256-byte-aligned views out of one allocation.
struct Arena {
    size_t used = 0;
    std::vector<std::pair<DevBuf*, size_t>> items;
    void add(DevBuf& b, size_t bytes)
    {
        items.push_back({&b, used});
        b.bytes = bytes;
        used += (bytes + 255) & ~(size_t)255;
    }
    int commit(DevBuf& owner)
    {
        TRY(owner.alloc(used ? used : 256));
        for (auto& it : items) {
            const size_t n = it.first->bytes;
            it.first->view((char*)owner.p + it.second, n);
        }
        return HF_OK;
    }
};

static int system_setup(hf_system* S, const hf_geometry* geom, const hf_basis* basis)
{
    hf_ctx* ctx = S->ctx;
    cudaStream_t st = ctx->stream;
    hf_system& X = *S;
    const int na = geom->n_atoms, ns = basis->n_shells;
    // host bookkeeping of the basis layout (offsets only)
    std::vector<int> bf0(ns), prim0(ns);
    int nbf = 0, npr = 0, maxnp = 0;
    for (int s = 0; s < ns; s++) {
        bf0[s] = nbf;
        prim0[s] = npr;
        nbf += (basis->l[s] + 1) * (basis->l[s] + 2) / 2;
        npr += basis->nprim[s];
        maxnp = std::max(maxnp, (int)basis->nprim[s]);
    }
    std::vector<double> Zd(na);
    int nel = 0;
    for (int a = 0; a < na; a++) {
        Zd[a] = geom->Z[a];
        nel += geom->Z[a];
    }
    S->Z_h.assign(geom->Z, geom->Z + na);
    S->atom_bf0_h.assign(na, -1);
    S->atom_nbf_h.assign(na, 0);
    {
        int last = -1;
        for (int s = 0; s < ns; s++) {
            const int a = basis->atom[s];
            if (S->atom_bf0_h[a] < 0) S->atom_bf0_h[a] = bf0[s];
            else if (last != a) S->atom_nbf_h[a] = -1000000;  // shells of this atom are not contiguous
            S->atom_nbf_h[a] += (basis->l[s] + 1) * (basis->l[s] + 2) / 2;
            last = a;
        }
        for (int a = 0; a < na; a++)
            if (S->atom_nbf_h[a] < 0) S->atom_bf0_h[a] = -1;
    }
    S->n_atoms = na;
    S->n_shells = ns;
    S->n_bf = nbf;
    S->n_electrons = nel;
    X.maxpp = maxnp * maxnp;
    const long long npairs = (long long)ns * (ns + 1) / 2;
    if (npairs * (long long)X.maxpp >= (1ll << 31)) return fail(HF_E_UNSUPPORTED, "too many primitive pairs");
    S->n_pairs_all = (int)npairs;
    const size_t NN = (size_t)nbf * nbf;

    // ---------------------------------------------- inputs, matrices, pairs
    DevBuf coef_in;
    Arena a1;
    a1.add(S->sh_l, sizeof(int) * ns);
    a1.add(S->sh_atom, sizeof(int) * ns);
    a1.add(S->sh_bf0, sizeof(int) * ns);
    a1.add(S->sh_nprim, sizeof(int) * ns);
    a1.add(S->sh_prim0, sizeof(int) * ns);
    a1.add(S->sh_exp, sizeof(double) * npr);
    a1.add(coef_in, sizeof(double) * npr);
    a1.add(S->atom_xyz, sizeof(double) * 3 * na);
    a1.add(S->atom_Z, sizeof(double) * na);
    a1.add(S->sh_coef, sizeof(double) * npr);
    a1.add(S->comp_norm, sizeof(double) * nbf);
    a1.add(S->Ebuf, sizeof(double) * 320);
    a1.add(S->pairs, sizeof(PairHdr) * npairs);
    a1.add(S->prims64, sizeof(PrimPair<double>) * npairs * X.maxpp);
    a1.add(S->prims32, sizeof(PrimPair<float>) * npairs * X.maxpp);
    a1.add(S->pair_class, sizeof(int) * npairs);
    a1.add(X.counts, sizeof(unsigned long long) * 16);
    a1.add(X.Qall, sizeof(double) * npairs);
    a1.add(X.Bprim, sizeof(double) * npairs * X.maxpp);
    TRY(a1.commit(X.arena_in));
    Arena a2;
    a2.add(S->S, NN * sizeof(double));
    a2.add(S->H, NN * sizeof(double));
    a2.add(S->P64, NN * sizeof(double));
    if (S->th.fp32_cutoff > 0.0) a2.add(S->P32, NN * sizeof(float));
    a2.add(S->Jt, NN * sizeof(double));
    a2.add(S->Kt, NN * sizeof(double));
    a2.add(S->F, NN * sizeof(double));
    a2.add(X.staging_P, NN * sizeof(double));
    a2.add(X.staging_out, 2 * NN * sizeof(double));
    a2.add(X.bad, sizeof(int));
    a2.add(X.prim_count, sizeof(unsigned long long) * 2 * kNumClasses);
    TRY(a2.commit(X.arena_mat));
    HF_CUDA(cudaMemcpyAsync(S->sh_l.p, basis->l, sizeof(int) * ns, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemcpyAsync(S->sh_atom.p, basis->atom, sizeof(int) * ns, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemcpyAsync(S->sh_bf0.p, bf0.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemcpyAsync(S->sh_nprim.p, basis->nprim, sizeof(int) * ns, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemcpyAsync(S->sh_prim0.p, prim0.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemcpyAsync(S->sh_exp.p, basis->exps, sizeof(double) * npr, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemcpyAsync(coef_in.p, basis->coefs, sizeof(double) * npr, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemcpyAsync(S->atom_xyz.p, geom->xyz, sizeof(double) * 3 * na, cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaMemcpyAsync(S->atom_Z.p, Zd.data(), sizeof(double) * na, cudaMemcpyHostToDevice, st));
    KCHK(launch_shell_coef(ns, S->sh_l.as<int>(), S->sh_nprim.as<int>(), S->sh_prim0.as<int>(), S->sh_exp.as<double>(),
                           coef_in.as<double>(), S->sh_coef.as<double>(), st));
    KCHK(launch_comp_norm(ns, S->sh_l.as<int>(), S->sh_bf0.as<int>(), S->comp_norm.as<double>(), st));
    KCHK(launch_one_electron(ns, na, nbf, S->sh_l.as<int>(), S->sh_atom.as<int>(), S->sh_bf0.as<int>(),
                             S->sh_nprim.as<int>(), S->sh_prim0.as<int>(), S->sh_exp.as<double>(),
                             S->sh_coef.as<double>(), S->atom_xyz.as<double>(), S->atom_Z.as<double>(),
                             S->comp_norm.as<double>(), ctx->boys64.as<double>(), S->S.as<double>(),
                             S->H.as<double>(), st));
    KCHK(launch_nuclear_repulsion(na, S->atom_xyz.as<double>(), S->atom_Z.as<double>(), S->Ebuf.as<double>() + 300,
                                  st));
    KCHK(launch_build_pairs(npairs, X.maxpp, S->sh_l.as<int>(), S->sh_atom.as<int>(), S->sh_bf0.as<int>(),
                            S->sh_nprim.as<int>(), S->sh_prim0.as<int>(), S->sh_exp.as<double>(),
                            S->sh_coef.as<double>(), S->atom_xyz.as<double>(), S->pairs.as<PairHdr>(),
                            S->prims64.p, S->prims32.p, S->pair_class.as<int>(), st));
    unsigned long long* cnt_dev = X.counts.as<unsigned long long>();  // [0..5] class counts, [8..15] cursors
    HF_CUDA(cudaMemsetAsync(cnt_dev, 0, sizeof(unsigned long long) * 16, st));
    KCHK(launch_class_count(npairs, S->pair_class.as<int>(), cnt_dev, st));
    unsigned long long cnt_all[kNumPairClasses];
    HF_CUDA(cudaMemcpyAsync(cnt_all, cnt_dev, sizeof(cnt_all), cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));  // host sync 1 of 2: class sizes

    // ------------------------------------------------------ schedule arena
    size_t npad[kNumPairClasses], seg[kNumPairClasses + 1], base_all[kNumPairClasses + 1];
    seg[0] = base_all[0] = 0;
    for (int c = 0; c < kNumPairClasses; c++) {
        npad[c] = cnt_all[c] ? next_pow2(cnt_all[c]) : 0;
        seg[c + 1] = seg[c] + npad[c];
        base_all[c + 1] = base_all[c] + cnt_all[c];
    }
    DevBuf ids_all, key, val, rb;
    DevBuf c64[kNumClasses], c32[kNumClasses];
    Arena a3;
    a3.add(ids_all, sizeof(int) * (npairs ? npairs : 1));
    a3.add(key, sizeof(double) * (seg[kNumPairClasses] ? seg[kNumPairClasses] : 1));
    a3.add(val, sizeof(int) * (seg[kNumPairClasses] ? seg[kNumPairClasses] : 1));
    a3.add(rb, 512);  // readback block: unsigned nsig[8] | long long totals[2*21] | double E_nn
    for (int ci = 0; ci < kNumClasses; ci++) {
        const size_t cap = cnt_all[kEriClasses[ci].X];
        auto& pl = S->plan[ci];
        a3.add(c64[ci], sizeof(long long) * (cap ? cap : 1));
        a3.add(c32[ci], sizeof(long long) * (cap ? cap : 1));
        a3.add(pl.kstart32, sizeof(int) * (cap ? cap : 1));
        a3.add(pl.offsets64, sizeof(long long) * (cap + 1));
        a3.add(pl.offsets32, sizeof(long long) * (cap + 1));
    }
    TRY(a3.commit(X.arena_sched));
    unsigned* nsig_dev = rb.as<unsigned>();
    long long* totals_dev = (long long*)(rb.as<char>() + 32);
    double* enn_dev = (double*)(rb.as<char>() + 32 + 8 * 2 * kNumClasses);
    HF_CUDA(cudaMemsetAsync(rb.p, 0, 512, st));

    // --------------------------------------------------- Schwarz bounds
    HF_CUDA(cudaMemsetAsync(X.Qall.p, 0, sizeof(double) * npairs, st));
    HF_CUDA(cudaMemsetAsync(X.Bprim.p, 0, sizeof(double) * npairs * X.maxpp, st));
    for (int c = 0; c < kNumPairClasses; c++) {
        if (!cnt_all[c]) continue;
        int* ids = ids_all.as<int>() + base_all[c];
        KCHK(launch_class_scatter_all(npairs, S->pair_class.as<int>(), c, (unsigned*)(cnt_dev + 8 + c), ids, st));
        SchwarzArgs sa;
        sa.pairs = S->pairs.as<PairHdr>();
        sa.prims64 = S->prims64.p;
        sa.ids = ids;
        sa.n = (int)cnt_all[c];
        sa.Q = X.Qall.as<double>();
        sa.boys64 = ctx->boys64.as<double>();
        sa.Bprim = X.Bprim.as<double>();
        sa.items = X.maxpp + 1;
        kEriClasses[class_index(c, c)].launch_schwarz(sa, kEriThreads, st);
        HF_CUDA(cudaGetLastError());
    }
    KCHK(launch_sort_prims(npairs, S->pairs.as<PairHdr>(), X.Bprim.as<double>(), S->prims64.p, S->prims32.p, st));
    unsigned long long* qbits_dev = cnt_dev + 7;
    HF_CUDA(cudaMemsetAsync(qbits_dev, 0, sizeof(unsigned long long), st));
    KCHK(launch_copy_q(npairs, X.Qall.as<double>(), S->pairs.as<PairHdr>(), qbits_dev, st));

    // ------------------------------------- significant pairs, sorted by Q
    const double tau = S->th.schwarz_tau;
    KCHK(launch_sig_scatter(npairs, (long long)seg[kNumPairClasses], S->pair_class.as<int>(), X.Qall.as<double>(),
                            qbits_dev, tau, seg, nsig_dev, key.as<double>(), val.as<int>(), st));
    for (int c = 0; c < kNumPairClasses; c++) {
        if (!npad[c]) continue;
        KCHK(bitonic_sort_desc(key.as<double>() + seg[c], val.as<int>() + seg[c], (int)npad[c], (int)npad[c], st));
        S->class_ids[c].view(val.as<int>() + seg[c], sizeof(int) * npad[c]);
        X.class_q[c].view(key.as<double>() + seg[c], sizeof(double) * npad[c]);
    }

    // ------------------------------------------------- quartet schedule
    S->quartets_total = 0;
    for (int ci = 0; ci < kNumClasses; ci++) {
        const int Xc = kEriClasses[ci].X, Yc = kEriClasses[ci].Y;
        auto& pl = S->plan[ci];
        pl.n_unscreened = (Xc == Yc) ? (long long)cnt_all[Xc] * (cnt_all[Xc] + 1) / 2
                                     : (long long)cnt_all[Xc] * (long long)cnt_all[Yc];
        S->quartets_total += pl.n_unscreened;
        const int cap = (int)cnt_all[Xc];
        if (!cap || !cnt_all[Yc]) continue;
        KCHK(launch_ket_counts_dev(cap, nsig_dev + Xc, X.class_q[Xc].as<double>(), nsig_dev + Yc,
                                   X.class_q[Yc].as<double>(), Xc == Yc, tau, S->th.fp32_cutoff, c64[ci].as<long long>(),
                                   c32[ci].as<long long>(), pl.kstart32.as<int>(), st));
        KCHK(launch_scan(cap, c64[ci].as<long long>(), pl.offsets64.as<long long>(), st));
        KCHK(launch_scan(cap, c32[ci].as<long long>(), pl.offsets32.as<long long>(), st));
        HF_CUDA(cudaMemcpyAsync(totals_dev + 2 * ci, pl.offsets64.as<long long>() + cap, sizeof(long long),
                                cudaMemcpyDeviceToDevice, st));
        HF_CUDA(cudaMemcpyAsync(totals_dev + 2 * ci + 1, pl.offsets32.as<long long>() + cap, sizeof(long long),
                                cudaMemcpyDeviceToDevice, st));
    }
    HF_CUDA(cudaMemcpyAsync(enn_dev, S->Ebuf.as<double>() + 300, sizeof(double), cudaMemcpyDeviceToDevice, st));
    HF_CUDA(cudaMemcpyAsync(enn_dev + 1, qbits_dev, sizeof(double), cudaMemcpyDeviceToDevice, st));
    unsigned char rbh[512];
    HF_CUDA(cudaMemcpyAsync(rbh, rb.p, 512, cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));  // host sync 2 of 2: significant counts, quartet totals, E_nn
    const unsigned* nsig_h = (const unsigned*)rbh;
    const long long* totals_h = (const long long*)(rbh + 32);
    memcpy(&S->E_nn, rbh + 32 + 8 * 2 * kNumClasses, sizeof(double));
    memcpy(&S->Qmax, rbh + 32 + 8 * 2 * kNumClasses + 8, sizeof(double));
    for (int c = 0; c < kNumPairClasses; c++) S->class_count[c] = (int)nsig_h[c];
    for (int ci = 0; ci < kNumClasses; ci++) {
        S->plan[ci].n64 = totals_h[2 * ci];
        S->plan[ci].n32 = totals_h[2 * ci + 1];
    }
    // ket tables (field-major copies of each class's records in class-list order)
    for (int c = 0; c < kNumPairClasses; c++) {
        const int n = S->class_count[c];
        if (n <= 0) continue;
        const long long stride = ((long long)n + 31) / 32 * 32;
        S->ket_stride[c] = stride;
        const size_t rows = (size_t)X.maxpp;
        TRY(S->ket_tab[c].alloc(rows * stride * (9 * sizeof(double) + 9 * sizeof(float) + sizeof(float))));
        double* t64 = S->ket_tab[c].as<double>();
        float* t32 = (float*)(t64 + 9 * rows * stride);
        float* tB = t32 + 9 * rows * stride;
        KCHK(launch_ket_table(n, X.maxpp, stride, S->class_ids[c].as<int>(), S->pairs.as<PairHdr>(), S->prims64.p,
                              S->prims32.p, t64, t32, tB, st));
        TRY(S->class_hdr[c].alloc(sizeof(PairHdr) * (size_t)n));
        KCHK(launch_gather_headers(n, S->class_ids[c].as<int>(), S->pairs.as<PairHdr>(), S->class_hdr[c].as<PairHdr>(),
                                   st));
    }
    // bra lookup tables (their sizes follow from the quartet totals)
    for (int ci = 0; ci < kNumClasses; ci++) {
        auto& pl = S->plan[ci];
        const int nb = S->class_count[kEriClasses[ci].X];
        if (pl.n64 > 0) {
            TRY(pl.chunk64.alloc(sizeof(int) * chunk_entries(pl.n64)));
            KCHK(launch_chunk_bra(nb, pl.offsets64.as<long long>(), pl.n64, pl.chunk64.as<int>(), st));
        }
        if (pl.n32 > 0) {
            TRY(pl.chunk32.alloc(sizeof(int) * chunk_entries(pl.n32)));
            KCHK(launch_chunk_bra(nb, pl.offsets32.as<long long>(), pl.n32, pl.chunk32.as<int>(), st));
        }
    }
    HF_CUDA(cudaGetLastError());
    return HF_OK;
}

static int check_geometry_basis(const hf_geometry* g, const hf_basis* b, const hf_thresholds* th)
{
    if (!g || !b) return fail(HF_E_INVALID, "geometry or basis is NULL");
    if (g->n_atoms < 1 || !g->Z || !g->xyz) return fail(HF_E_INVALID, "geometry: empty or NULL arrays");
    if (b->n_shells < 1 || !b->atom || !b->l || !b->nprim || !b->exps || !b->coefs)
        return fail(HF_E_INVALID, "basis: empty or NULL arrays");
    for (int a = 0; a < g->n_atoms; a++) {
        if (g->Z[a] < 0) return fail(HF_E_INVALID, "geometry: negative nuclear charge");
        for (int x = 0; x < 3; x++)
            if (!isfinite(g->xyz[3 * a + x])) return fail(HF_E_INVALID, "geometry: non-finite coordinate");
    }
    long long np = 0;
    for (int s = 0; s < b->n_shells; s++) {
        if (b->atom[s] < 0 || b->atom[s] >= g->n_atoms) return fail(HF_E_INVALID, "basis: atom index out of range");
        if (b->l[s] == HF_SP_SHELL && !b->coefs_p)
            return fail(HF_E_INVALID, "basis: sp shell without p coefficients (coefs_p is NULL)");
        if (b->l[s] < 0 && b->l[s] != HF_SP_SHELL) return fail(HF_E_INVALID, "basis: negative angular momentum");
        if (b->l[s] > kMaxL) return fail(HF_E_UNSUPPORTED, "basis: l > 2 is not supported");
        if (b->nprim[s] < 1) return fail(HF_E_INVALID, "basis: shell without primitives");
        if (b->nprim[s] > kMaxPrim) return fail(HF_E_UNSUPPORTED, "basis: more than 8 primitives in a shell");
        np += b->nprim[s];
    }
    for (long long k = 0; k < np; k++) {
        if (!(b->exps[k] > 0.0) || !isfinite(b->exps[k])) return fail(HF_E_INVALID, "basis: exponent not positive");
        if (!isfinite(b->coefs[k])) return fail(HF_E_INVALID, "basis: non-finite coefficient");
    }
    if (b->coefs_p) {
        long long o = 0;
        for (int s = 0; s < b->n_shells; s++) {
            if (b->l[s] == HF_SP_SHELL)
                for (int k = 0; k < b->nprim[s]; k++)
                    if (!isfinite(b->coefs_p[o + k])) return fail(HF_E_INVALID, "basis: non-finite p coefficient");
            o += b->nprim[s];
        }
    }
    if (th) {
        if (!(th->schwarz_tau >= 0.0) || !(th->fp32_cutoff >= 0.0)) return fail(HF_E_INVALID, "thresholds: negative");
        if (!(th->prim_tau >= 0.0)) return fail(HF_E_INVALID, "thresholds: negative prim_tau");
    }
    return HF_OK;
}

// A basis with sp shells written as separate shells: each sp shell becomes an s shell (coefficients
// coefs) followed by a p shell (coefficients coefs_p) with the same exponents on the same atom, which
// keeps the basis-function order s, x, y, z of the sp shell.
struct ExpandedBasis {
    std::vector<int32_t> atom, l, nprim;
    std::vector<double> exps, coefs;
    hf_basis view{};
};

static const hf_basis* expand_sp_shells(const hf_basis* b, ExpandedBasis& e)
{
    bool any = false;
    for (int s = 0; s < b->n_shells; s++) any |= b->l[s] == HF_SP_SHELL;
    if (!any) return b;
    long long o = 0;
    for (int s = 0; s < b->n_shells; s++) {
        const int n = b->nprim[s];
        const int parts = b->l[s] == HF_SP_SHELL ? 2 : 1;
        for (int part = 0; part < parts; part++) {
            e.atom.push_back(b->atom[s]);
            e.l.push_back(b->l[s] == HF_SP_SHELL ? part : b->l[s]);
            e.nprim.push_back(n);
            const double* c = part == 1 ? b->coefs_p : b->coefs;
            for (int k = 0; k < n; k++) {
                e.exps.push_back(b->exps[o + k]);
                e.coefs.push_back(c[o + k]);
            }
        }
        o += n;
    }
    e.view.n_shells = (int32_t)e.l.size();
    e.view.atom = e.atom.data();
    e.view.l = e.l.data();
    e.view.nprim = e.nprim.data();
    e.view.exps = e.exps.data();
    e.view.coefs = e.coefs.data();
    e.view.coefs_p = nullptr;
    return &e.view;
}

extern "C" {

int hf_system_create(hf_ctx* ctx, const hf_geometry* geom, const hf_basis* basis_in, const hf_thresholds* th,
                     hf_system** out)
{
    if (!ctx || !out) return fail(HF_E_INVALID, "hf_system_create: NULL ctx or output pointer");
    *out = nullptr;
    TRY(check_geometry_basis(geom, basis_in, th));
    ExpandedBasis eb;
    const hf_basis* basis = expand_sp_shells(basis_in, eb);
    DeviceGuard g(ctx->device);
    hf_system* S = new hf_system();
    S->ctx = ctx;
    S->device = ctx->device;
    S->stream = ctx->stream;
    if (th) S->th = *th;
    int rc = system_setup(S, geom, basis);
    if (rc != HF_OK) {
        cudaStreamSynchronize(ctx->stream);
        delete S;
        return rc;
    }
    ctx->n_systems++;
    *out = S;
    return HF_OK;
}

void hf_system_destroy(hf_system* S)
{
    if (!S) return;
    hf_ctx* ctx = S->ctx;
    {
        DeviceGuard g(S->device);
        cudaStreamSynchronize(S->stream);
        delete S;
    }
    if (ctx && --ctx->n_systems == 0 && ctx->destroy_pending) ctx_release(ctx);
}

int hf_system_get_info(const hf_system* S, hf_system_info* info)
{
    if (!S || !info) return fail(HF_E_INVALID, "hf_system_get_info: NULL argument");
    memset(info, 0, sizeof(*info));
    info->n_atoms = S->n_atoms;
    info->n_shells = S->n_shells;
    info->n_bf = S->n_bf;
    info->n_electrons = S->n_electrons;
    info->n_pairs = S->n_pairs_all;
    for (int c = 0; c < kNumPairClasses; c++) info->n_significant_pairs += S->class_count[c];
    info->quartets_unscreened = S->quartets_total;
    for (int c = 0; c < kNumClasses; c++) {
        info->quartets_fp64 += S->plan[c].n64;
        info->quartets_fp32 += S->plan[c].n32;
    }
    info->E_nn = S->E_nn;
    info->Q_max = S->Qmax;
    long long bytes = 0;
    const DevBuf* bufs[] = {&S->sh_l, &S->sh_atom, &S->sh_bf0, &S->sh_nprim, &S->sh_prim0, &S->sh_exp, &S->sh_coef,
                            &S->atom_xyz, &S->atom_Z, &S->comp_norm, &S->pairs, &S->prims64, &S->prims32,
                            &S->pair_class, &S->S, &S->H, &S->P64, &S->P32, &S->Jt, &S->Kt, &S->F, &S->Ebuf,
                            &S->Qall, &S->staging_P, &S->staging_out};
    for (auto* b : bufs) bytes += b->bytes;
    for (int c = 0; c < kNumPairClasses; c++)
        bytes += S->class_ids[c].bytes + S->class_q[c].bytes + S->ket_tab[c].bytes + S->class_hdr[c].bytes;
    for (int c = 0; c < kNumClasses; c++)
        bytes += S->plan[c].offsets64.bytes + S->plan[c].offsets32.bytes + S->plan[c].kstart32.bytes +
                 S->plan[c].chunk64.bytes + S->plan[c].chunk32.bytes;
    info->device_bytes = bytes;
    return HF_OK;
}

int hf_one_electron(hf_system* S, double* Sout, double* Hout, int flags)
{
    if (!S) return fail(HF_E_INVALID, "hf_one_electron: NULL system");
    DeviceGuard g(S->ctx->device);
    const size_t bytes = (size_t)S->n_bf * S->n_bf * sizeof(double);
    const cudaMemcpyKind kind = (flags & HF_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaStream_t st = S->ctx->stream;
    if (Sout) HF_CUDA(cudaMemcpyAsync(Sout, S->S.p, bytes, kind, st));
    if (Hout) HF_CUDA(cudaMemcpyAsync(Hout, S->H.p, bytes, kind, st));
    HF_CUDA(cudaStreamSynchronize(st));
    return HF_OK;
}

// Accumulators of one build: the system's Jt / Kt (one copy shared by every block, updated with FP64
// atomics), or fock_copies zeroed copies of each, block b writing copy b % fock_copies, summed into
// Jt / Kt after the ERI launches (the GPU analogue of the paper's private Fock matrices).
static int begin_accumulate(hf_system& X, EriArgs& a, cudaStream_t st)
{
    const size_t NN = (size_t)X.n_bf * X.n_bf;
    if (X.fock_copies > 1) {
        HF_CUDA(cudaMemsetAsync(X.copies.p, 0, 2 * (size_t)X.fock_copies * NN * sizeof(double), st));
        a.Jt = X.copies.as<double>();
        a.Kt = a.Jt + (size_t)X.fock_copies * NN;
        a.n_copies = X.fock_copies;
        a.copy_stride = (long long)NN;
    } else {
        HF_CUDA(cudaMemsetAsync(X.Jt.p, 0, NN * sizeof(double), st));
        HF_CUDA(cudaMemsetAsync(X.Kt.p, 0, NN * sizeof(double), st));
        a.Jt = X.Jt.as<double>();
        a.Kt = X.Kt.as<double>();
        a.n_copies = 1;
        a.copy_stride = 0;
    }
    return HF_OK;
}

static int end_accumulate(hf_system& X, cudaStream_t st)
{
    if (X.fock_copies <= 1) return HF_OK;
    const long long NN = (long long)X.n_bf * X.n_bf;
    const double* c = X.copies.as<double>();
    KCHK(launch_sum_copies(X.fock_copies, NN, c, X.Jt.as<double>(), X.ctx->num_sms, st));
    KCHK(launch_sum_copies(X.fock_copies, NN, c + (size_t)X.fock_copies * NN, X.Kt.as<double>(), X.ctx->num_sms, st));
    return HF_OK;
}

int hf_system_set_fock_copies(hf_system* S, int32_t copies)
{
    if (!S) return fail(HF_E_INVALID, "hf_system_set_fock_copies: NULL system");
    if (copies < 1 || copies > 4096) return fail(HF_E_INVALID, "hf_system_set_fock_copies: copies must be 1..4096");
    DeviceGuard g(S->ctx->device);
    HF_CUDA(cudaStreamSynchronize(S->ctx->stream));
    if (copies == 1) {
        S->copies.release();
        S->fock_copies = 1;
        return HF_OK;
    }
    const size_t NN = (size_t)S->n_bf * S->n_bf;
    S->copies.release();
    S->fock_copies = 1;
    if (S->copies.alloc(2 * (size_t)copies * NN * sizeof(double)) != HF_OK) {
        cudaGetLastError();
        return fail(HF_E_NOMEM, "hf_system_set_fock_copies: cannot allocate the accumulator copies");
    }
    S->fock_copies = copies;
    return HF_OK;
}

}  // extern "C"

// Whether a launch of class ci runs the Rys-quadrature kernel: an FP64 launch of a class whose Rys variant
// the flags select (class_uses_rys), with the ket tables in use.
static bool uses_rys(int ci, int flags, int use_f32, const EriArgs& a)
{
    return !use_f32 && class_uses_rys(ci, flags) && a.kt;
}
// (the ket tables always exist for a class with significant pairs, so a.kt is set for every launch)

// The per-class ERI launches shared by hf_fock_build, hf_fock_build_partial and hf_fock_build_noalloc.
int hf::launch_eri_classes(hf_system* S, EriArgs a, int shard, int n_shards, int flags, cudaEvent_t* ev,
                           unsigned long long* prim_count)
{
    hf_ctx* ctx = S->ctx;
    cudaStream_t st = ctx->stream;
    hf_system& X = *S;
    a.pairs = S->pairs.as<PairHdr>();
    a.prims64 = S->prims64.p;
    a.prims32 = S->prims32.p;
    a.N = S->n_bf;
    a.boys64 = ctx->boys64.as<double>();
    a.boys32 = ctx->boys32.as<float>();
    a.prim_tau = S->th.prim_tau;
    for (int ci = 0; ci < kNumClasses; ci++) {
        const auto& pl = S->plan[ci];
        const int Xc = kEriClasses[ci].X, Yc = kEriClasses[ci].Y;
        a.bra = S->class_ids[Xc].as<int>();
        a.ket = S->class_ids[Yc].as<int>();
        a.bhdr = S->class_hdr[Xc].as<PairHdr>();
        a.khdr = S->class_hdr[Yc].as<PairHdr>();
        a.n_bra = S->class_count[Xc];
        a.same = Xc == Yc;
        for (int prec = 0; prec < 2; prec++) {
            const long long n = prec ? pl.n32 : pl.n64;
            const long long q0 = n * shard / n_shards, q1 = n * (shard + 1) / n_shards;
            if (ev) HF_CUDA(cudaEventRecord(ev[4 * ci + 2 * prec], st));
            a.prim_count = prim_count ? prim_count + 2 * ci + prec : nullptr;
            if (q1 > q0) {
                a.offsets = prec ? pl.offsets32.as<long long>() : pl.offsets64.as<long long>();
                a.kstart = prec ? pl.kstart32.as<int>() : nullptr;
                a.chunk = prec ? pl.chunk32.as<int>() : pl.chunk64.as<int>();
                a.q_begin = q0;
                a.n_quartets = q1;
                const int use_f32 = prec && !(flags & HF_FP64_ONLY);
                a.kt = nullptr;
                a.ktB = nullptr;
                a.kstride = 0;
                if (X.ket_tab[Yc].p) {
                    const long long st_ = X.ket_stride[Yc];
                    const double* t64 = X.ket_tab[Yc].as<double>();
                    const float* t32 = (const float*)(t64 + 9 * (size_t)X.maxpp * st_);
                    a.kt = use_f32 ? (const void*)t32 : (const void*)t64;
                    a.ktB = t32 + 9 * (size_t)X.maxpp * st_;
                    a.kstride = st_;
                }
                // a class too small to fill the GPU with one thread per quartet shares each quartet's
                // primitive work among a lane group instead (shorter latency, same result)
                const int lanes = (!use_f32 && q1 - q0 < (long long)ctx->num_sms * 256) ? kEriClasses[ci].lanes : 1;
                const long long blocks = ((q1 - q0) * lanes + kEriThreads - 1) / kEriThreads;
                const int grid = (int)std::min<long long>(blocks, (long long)ctx->num_sms * 16);
                // FP64 launches run each warp's window of quartets sorted by staircase length (64 waters:
                // 2% faster); the FP32 kernels, bound by latency rather than a pipe, ran 10% slower with it
                // and are compiled without it
                a.sort_work = use_f32 ? 0 : 1;
                if (uses_rys(ci, flags, use_f32, a))
                    kEriClasses[ci].launch_rys(a, 0, grid, kEriThreads, st, lanes);
                else
                    kEriClasses[ci].launch(a, use_f32, grid, kEriThreads, st, lanes);
                HF_CUDA(cudaGetLastError());
            }
            if (ev) HF_CUDA(cudaEventRecord(ev[4 * ci + 2 * prec + 1], st));
        }
    }
    return HF_OK;
}

extern "C" {

int hf_fock_build(hf_system* S, const double* P, double* F, double* J, double* K, double* E_elec, hf_stats* stats,
                  int flags)
{
    if (!S || !P) return fail(HF_E_INVALID, "hf_fock_build: NULL system or density");
    DeviceGuard g(S->ctx->device);
    hf_ctx* ctx = S->ctx;
    hf_system& X = *S;
    cudaStream_t st = ctx->stream;
    const int N = S->n_bf;
    const size_t NN = (size_t)N * N;
    const bool dev = (flags & HF_PTR_DEVICE) != 0;
    const bool timing = (flags & HF_TIMING) != 0 && stats;
    // 1. density in, check, raw-normalised copies.  The check's flag stays on the device: the ERI,
    // assembly and energy kernels do nothing when it is set, and the host reads it once, at the end.
    const double* dP = P;
    if (!dev) {
        HF_CUDA(cudaMemcpyAsync(X.staging_P.p, P, NN * sizeof(double), cudaMemcpyHostToDevice, st));
        dP = X.staging_P.as<double>();
    }
    if (timing) HF_CUDA(cudaEventRecord(ctx->ev[4 * kNumClasses], st));
    HF_CUDA(cudaMemsetAsync(X.bad.p, 0, sizeof(int), st));
    KCHK(launch_scale_density(N, dP, S->comp_norm.as<double>(), S->P64.as<double>(),
                              S->P32.p ? S->P32.as<float>() : nullptr, X.bad.as<int>(), st));
    // 2. ERI + digestion, one launch per class and precision
    EriArgs a;
    memset(&a, 0, sizeof(a));
    TRY(begin_accumulate(X, a, st));
    if (timing) HF_CUDA(cudaEventRecord(ctx->ev[4 * kNumClasses + 1], st));
    a.P64 = S->P64.as<double>();
    a.P32 = S->P32.p ? S->P32.as<float>() : nullptr;
    a.bad = X.bad.as<int>();
    if (stats) HF_CUDA(cudaMemsetAsync(X.prim_count.p, 0, sizeof(unsigned long long) * 2 * kNumClasses, st));
    TRY(launch_eri_classes(S, a, 0, 1, flags, timing ? ctx->ev : nullptr,
                           stats ? X.prim_count.as<unsigned long long>() : nullptr));
    TRY(end_accumulate(X, st));
    if (timing) HF_CUDA(cudaEventRecord(ctx->ev[4 * kNumClasses + 2], st));
    // 3. symmetrise and assemble (skipped on the device when the density was rejected)
    double* dF = dev && F ? F : S->F.as<double>();
    double* dJ = dev ? J : (J ? X.staging_out.as<double>() : nullptr);
    double* dK = dev ? K : (K ? X.staging_out.as<double>() + NN : nullptr);
    KCHK(launch_assemble(N, S->Jt.as<double>(), S->Kt.as<double>(), S->comp_norm.as<double>(), S->H.as<double>(), dJ,
                         dK, dF, X.bad.as<int>(), st));
    if (E_elec) KCHK(launch_energy(N, dP, S->H.as<double>(), dF, S->Ebuf.as<double>(), S->Ebuf.as<double>() + 256, st));
    if (timing) HF_CUDA(cudaEventRecord(ctx->ev[4 * kNumClasses + 3], st));
    int bad = 0;
    double e_host = 0.0;
    HF_CUDA(cudaMemcpyAsync(&bad, X.bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (E_elec) HF_CUDA(cudaMemcpyAsync(&e_host, S->Ebuf.as<double>() + 256, sizeof(double), cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    HF_CUDA(cudaGetLastError());
    if (bad) return fail(HF_E_INVALID, "hf_fock_build: density is not finite or not symmetric");
    if (!dev) {  // host outputs are written only once the density is known to be valid
        if (F) HF_CUDA(cudaMemcpyAsync(F, dF, NN * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (J) HF_CUDA(cudaMemcpyAsync(J, dJ, NN * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (K) HF_CUDA(cudaMemcpyAsync(K, dK, NN * sizeof(double), cudaMemcpyDeviceToHost, st));
        HF_CUDA(cudaStreamSynchronize(st));
    }
    if (E_elec) *E_elec = e_host;
    if (stats) {
        unsigned long long pc[2 * kNumClasses];
        HF_CUDA(cudaMemcpy(pc, X.prim_count.p, sizeof(pc), cudaMemcpyDeviceToHost));
        memset(stats, 0, sizeof(*stats));
        stats->quartets_unscreened = S->quartets_total;
        for (int ci = 0; ci < kNumClasses; ci++) {
            const auto& pl = S->plan[ci];
            stats->class_quartets_fp64[ci] = pl.n64;
            stats->class_quartets_fp32[ci] = pl.n32;
            stats->quartets_fp64 += pl.n64;
            stats->quartets_fp32 += pl.n32;
            stats->prim_quartets_fp64 += (int64_t)pc[2 * ci];
            stats->prim_quartets_fp32 += (int64_t)pc[2 * ci + 1];
            const double pf = kEriClasses[ci].prim_flops, cf = kEriClasses[ci].cont_flops;
            const bool rys = class_uses_rys(ci, flags);
            const double pf64 = rys ? kEriClasses[ci].prim_flops_rys : pf;
            const double pf32 = (rys && (flags & HF_FP64_ONLY)) ? pf64 : pf;  // FP32 launches stay Obara-Saika
            stats->class_flops_fp64[ci] = pf64 * (double)pc[2 * ci] + cf * (double)pl.n64;
            stats->class_flops_fp32[ci] = pf32 * (double)pc[2 * ci + 1] + cf * (double)pl.n32;
            stats->flops_fp64 += stats->class_flops_fp64[ci];
            stats->flops_fp32 += stats->class_flops_fp32[ci];
            stats->kernels_launched += (pl.n64 > 0) + (pl.n32 > 0);
            if (timing) {
                cudaEventElapsedTime(&stats->ms_class_fp64[ci], ctx->ev[4 * ci], ctx->ev[4 * ci + 1]);
                cudaEventElapsedTime(&stats->ms_class_fp32[ci], ctx->ev[4 * ci + 2], ctx->ev[4 * ci + 3]);
            }
        }
        stats->kernels_launched += 2 + (E_elec ? 2 : 0) + (X.fock_copies > 1 ? 2 : 0);  // density scaling,
                                                                                    // assembly, energy, copy sums
        if (timing) {
            cudaEventElapsedTime(&stats->ms_eri, ctx->ev[4 * kNumClasses + 1], ctx->ev[4 * kNumClasses + 2]);
            cudaEventElapsedTime(&stats->ms_total, ctx->ev[4 * kNumClasses], ctx->ev[4 * kNumClasses + 3]);
        }
    }
    return HF_OK;
}


// One shard of the Fock build: the quartets [n s / S, n (s+1) / S) of every class launch.
int hf_fock_build_partial(hf_system* S, const double* P, int shard, int n_shards, double* J, double* K, int flags)
{
    if (!S || !P || !J || !K) return fail(HF_E_INVALID, "hf_fock_build_partial: NULL argument");
    if (n_shards < 1 || shard < 0 || shard >= n_shards) return fail(HF_E_INVALID, "hf_fock_build_partial: bad shard");
    DeviceGuard g(S->ctx->device);
    hf_ctx* ctx = S->ctx;
    hf_system& X = *S;
    cudaStream_t st = ctx->stream;
    const int N = S->n_bf;
    const size_t NN = (size_t)N * N;
    const bool dev = (flags & HF_PTR_DEVICE) != 0;
    const double* dP = P;
    if (!dev) {
        HF_CUDA(cudaMemcpyAsync(X.staging_P.p, P, NN * sizeof(double), cudaMemcpyHostToDevice, st));
        dP = X.staging_P.as<double>();
    }
    HF_CUDA(cudaMemsetAsync(X.bad.p, 0, sizeof(int), st));
    KCHK(launch_scale_density(N, dP, S->comp_norm.as<double>(), S->P64.as<double>(),
                              S->P32.p ? S->P32.as<float>() : nullptr, X.bad.as<int>(), st));
    EriArgs a;
    memset(&a, 0, sizeof(a));
    TRY(begin_accumulate(X, a, st));
    a.P64 = S->P64.as<double>();
    a.P32 = S->P32.p ? S->P32.as<float>() : nullptr;
    a.bad = X.bad.as<int>();
    if ((flags & HF_DENSITY_SCREEN) && S->th.schwarz_tau > 0.0) {
        if (!X.dsh.p) TRY(X.dsh.alloc(sizeof(float) * (size_t)S->n_shells * S->n_shells));
        KCHK(launch_shell_block_max(S->n_shells, N, S->sh_l.as<int>(), S->sh_bf0.as<int>(), dP, X.dsh.as<float>(),
                                    st));
        a.dsh = X.dsh.as<float>();
        a.n_sh = S->n_shells;
        a.dtau = (float)S->th.schwarz_tau;
    }
    TRY(launch_eri_classes(S, a, shard, n_shards, flags, nullptr, nullptr));
    TRY(end_accumulate(X, st));
    // J and K of this shard (no H): the assembly kernel's F output is only scratch here
    double* dJ = dev ? J : X.staging_out.as<double>();
    double* dK = dev ? K : X.staging_out.as<double>() + NN;
    KCHK(launch_assemble(N, S->Jt.as<double>(), S->Kt.as<double>(), S->comp_norm.as<double>(), S->H.as<double>(), dJ,
                         dK, S->F.as<double>(), X.bad.as<int>(), st));
    int bad = 0;
    HF_CUDA(cudaMemcpyAsync(&bad, X.bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    if (bad) return fail(HF_E_INVALID, "hf_fock_build_partial: density is not finite or not symmetric");
    if (!dev) {
        HF_CUDA(cudaMemcpyAsync(J, dJ, NN * sizeof(double), cudaMemcpyDeviceToHost, st));
        HF_CUDA(cudaMemcpyAsync(K, dK, NN * sizeof(double), cudaMemcpyDeviceToHost, st));
        HF_CUDA(cudaStreamSynchronize(st));
    }
    return HF_OK;
}

// F = H + J - K/2 (and E_elec) from J and K summed over the shards of a sharded build.
int hf_fock_assemble(hf_system* S, const double* P, const double* J, const double* K, double* F, double* E_elec,
                     int flags)
{
    if (!S || !J || !K || !F) return fail(HF_E_INVALID, "hf_fock_assemble: NULL system, J, K or F");
    if (E_elec && !P) return fail(HF_E_INVALID, "hf_fock_assemble: the energy needs the density P");
    DeviceGuard g(S->ctx->device);
    hf_system& X = *S;
    cudaStream_t st = S->ctx->stream;
    const int N = S->n_bf;
    const size_t NN = (size_t)N * N;
    const bool dev = (flags & HF_PTR_DEVICE) != 0;
    const double *dJ = J, *dK = K, *dP = P;
    double* dF = dev ? F : S->F.as<double>();
    if (!dev) {  // staging: J and K in staging_out, P in staging_P
        HF_CUDA(cudaMemcpyAsync(X.staging_out.p, J, NN * sizeof(double), cudaMemcpyHostToDevice, st));
        HF_CUDA(cudaMemcpyAsync(X.staging_out.as<double>() + NN, K, NN * sizeof(double), cudaMemcpyHostToDevice, st));
        dJ = X.staging_out.as<double>();
        dK = dJ + NN;
        if (P) {
            HF_CUDA(cudaMemcpyAsync(X.staging_P.p, P, NN * sizeof(double), cudaMemcpyHostToDevice, st));
            dP = X.staging_P.as<double>();
        }
    }
    HF_CUDA(cudaMemsetAsync(X.bad.p, 0, sizeof(int), st));
    KCHK(launch_fock_from_jk((long long)NN, S->H.as<double>(), dJ, dK, dF, X.bad.as<int>(), st));
    if (E_elec) KCHK(launch_energy(N, dP, S->H.as<double>(), dF, S->Ebuf.as<double>(), S->Ebuf.as<double>() + 256, st));
    int bad = 0;
    double e_host = 0.0;
    HF_CUDA(cudaMemcpyAsync(&bad, X.bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (E_elec) HF_CUDA(cudaMemcpyAsync(&e_host, S->Ebuf.as<double>() + 256, sizeof(double), cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    if (bad) return fail(HF_E_INVALID, "hf_fock_assemble: J or K is not finite");
    if (!dev) {
        HF_CUDA(cudaMemcpyAsync(F, dF, NN * sizeof(double), cudaMemcpyDeviceToHost, st));
        HF_CUDA(cudaStreamSynchronize(st));
    }
    if (E_elec) *E_elec = e_host;
    return HF_OK;
}
}  // extern "C"

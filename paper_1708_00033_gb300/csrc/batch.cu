// Batched Fock builds for many independent molecules (one SCF iteration of a
// batch): one persistent kernel per angular class covers every molecule's
// quartets through a device work queue, the class kernels run concurrently on
// forked streams, and the whole step (density scaling, accumulator clearing,
// 21 class kernels, assembly, energies) is captured once in a CUDA graph and
// replayed per build.  A project-written autotuner picks each class kernel's
// block size, work-queue chunk and blocks per SM by timing candidates.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "eri_common.cuh"
#include "hf_internal.h"
#include "setup.cuh"

namespace hf {
namespace {

struct MolMat {
    int N;
    int pad;
    long long off;  // offset of the molecule's N x N block in the packed arrays
    const double* comp_norm;
    double* P64;
    double* Jt;
    double* Kt;
    const double* H;
};

__device__ __forceinline__ int find_mol(const long long* __restrict__ off, int n, long long e)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= e)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// P' = n P n into each molecule's raw-normalised density, accumulators cleared
__global__ void k_batch_scale(long long len, int n_mol, const long long* __restrict__ eoff,
                              const MolMat* __restrict__ mm, const double* __restrict__ P, int* __restrict__ bad)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    const int m = find_mol(eoff, n_mol, e);
    const MolMat d = mm[m];
    const long long t = e - d.off;
    const int i = (int)(t / d.N), j = (int)(t % d.N);
    const double v = P[e], w = P[d.off + (long long)j * d.N + i];
    if (!isfinite(v) || fabs(v - w) > 1e-12 * fmax(1.0, fabs(v))) atomicOr(bad, 1);
    d.P64[t] = d.comp_norm[i] * d.comp_norm[j] * v;
    d.Jt[t] = 0.0;
    d.Kt[t] = 0.0;
}

__global__ void k_batch_assemble(long long len, int n_mol, const long long* __restrict__ eoff,
                                 const MolMat* __restrict__ mm, double* __restrict__ F)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    const int m = find_mol(eoff, n_mol, e);
    const MolMat d = mm[m];
    const long long t = e - d.off;
    const int i = (int)(t / d.N), j = (int)(t % d.N);
    const long long tt = (long long)j * d.N + i;
    const double s = 0.5 * d.comp_norm[i] * d.comp_norm[j];
    F[e] = d.H[t] + s * (d.Jt[t] + d.Jt[tt]) - 0.5 * s * (d.Kt[t] + d.Kt[tt]);
}

// E_m = 1/2 sum P (H + F), one block per molecule
__global__ void k_batch_energy(const MolMat* __restrict__ mm, const double* __restrict__ P,
                               const double* __restrict__ F, double* __restrict__ E)
{
    __shared__ double sm[256];
    const MolMat d = mm[blockIdx.x];
    const long long n = (long long)d.N * d.N;
    double acc = 0.0;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) acc += P[d.off + t] * (d.H[t] + F[d.off + t]);
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) E[blockIdx.x] = 0.5 * sm[0];
}

int bfail(int code, const std::string& msg)
{
    set_error(code, msg);
    return code;
}

#define B_TRY(x)                       \
    do {                               \
        int rc_ = (x);                 \
        if (rc_ != HF_OK) return rc_;  \
    } while (0)

struct BatchDevice {
    int prev = -1;
    explicit BatchDevice(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~BatchDevice()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace hf

using namespace hf;

struct hf_batch {
    hf_ctx* ctx = nullptr;
    int device = 0;
    int n_mol = 0;
    std::vector<hf_system*> sys;
    std::vector<long long> eoff_h;  // [n_mol + 1]
    long long len = 0;
    DevBuf eoff, mm, Pin, Fout, E, bad;
    DevBuf mols[kNumClasses], moloff[kNumClasses], counters;
    long long n_total[kNumClasses] = {};
    int block[kNumClasses], chunk[kNumClasses], bps[kNumClasses];
    cudaStream_t st = nullptr;
    cudaStream_t cst[kNumClasses] = {};
    cudaEvent_t fork = nullptr, join[kNumClasses] = {}, t0 = nullptr, t1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int num_sms = 0;
    ~hf_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (int c = 0; c < kNumClasses; c++) {
            if (cst[c]) cudaStreamDestroy(cst[c]);
            if (join[c]) cudaEventDestroy(join[c]);
        }
        if (fork) cudaEventDestroy(fork);
        if (t0) cudaEventDestroy(t0);
        if (t1) cudaEventDestroy(t1);
        if (st) cudaStreamDestroy(st);
        for (auto* s : sys) hf_system_destroy(s);
    }
};

static BatchArgs batch_args(hf_batch* B, int c, long long limit)
{
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.mols = B->mols[c].as<MolClass>();
    a.mol_off = B->moloff[c].as<long long>();
    a.n_mol = B->n_mol;
    a.chunk = B->chunk[c];
    a.n_total = limit >= 0 ? std::min(limit, B->n_total[c]) : B->n_total[c];
    a.counter = B->counters.as<unsigned long long>() + c;
    a.prim_tau = B->sys[0]->th.prim_tau;
    a.boys64 = B->ctx->boys64.as<double>();
    return a;
}

static int capture_graph(hf_batch* B)
{
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    if (B->graph) {
        cudaGraphDestroy(B->graph);
        B->graph = nullptr;
    }
    cudaStream_t st = B->st;
    HF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(B->counters.p, 0, sizeof(unsigned long long) * kNumClasses, st);
    cudaMemsetAsync(B->bad.p, 0, sizeof(int), st);
    k_batch_scale<<<(unsigned)((B->len + 255) / 256), 256, 0, st>>>(B->len, B->n_mol, B->eoff.as<long long>(),
                                                                     B->mm.as<MolMat>(), B->Pin.as<double>(),
                                                                     B->bad.as<int>());
    cudaEventRecord(B->fork, st);
    for (int c = 0; c < kNumClasses; c++) {
        if (B->n_total[c] <= 0) continue;
        cudaStreamWaitEvent(B->cst[c], B->fork, 0);
        const BatchArgs a = batch_args(B, c, -1);
        kEriClasses[c].launch_batch(a, B->num_sms * B->bps[c], B->block[c], B->cst[c]);
        cudaEventRecord(B->join[c], B->cst[c]);
        cudaStreamWaitEvent(st, B->join[c], 0);
    }
    k_batch_assemble<<<(unsigned)((B->len + 255) / 256), 256, 0, st>>>(B->len, B->n_mol, B->eoff.as<long long>(),
                                                                        B->mm.as<MolMat>(), B->Fout.as<double>());
    k_batch_energy<<<B->n_mol, 256, 0, st>>>(B->mm.as<MolMat>(), B->Pin.as<double>(), B->Fout.as<double>(),
                                             B->E.as<double>());
    cudaError_t e = cudaStreamEndCapture(st, &B->graph);
    if (e != cudaSuccess) return cuda_status(e, "hf_batch: graph capture");
    HF_CUDA(cudaGraphInstantiate(&B->exec, B->graph, 0));
    return HF_OK;
}

extern "C" {

int hf_batch_create(hf_ctx* ctx, int n_mol, const hf_geometry* geoms, const hf_basis* bases, const hf_thresholds* th,
                    hf_batch** out)
{
    if (!ctx || !out || n_mol <= 0 || !geoms || !bases) return bfail(HF_E_INVALID, "hf_batch_create: bad arguments");
    *out = nullptr;
    BatchDevice g(ctx->device);
    hf_batch* B = new hf_batch();
    B->ctx = ctx;
    B->device = ctx->device;
    B->n_mol = n_mol;
    B->num_sms = ctx->num_sms;
    auto cleanup = [&](int rc) {
        delete B;
        return rc;
    };
    hf_thresholds t{};
    if (th) t = *th;
    t.fp32_cutoff = 0.0;  // the batched path is FP64 throughout
    for (int m = 0; m < n_mol; m++) {
        hf_system* s = nullptr;
        int rc = hf_system_create(ctx, &geoms[m], &bases[m], &t, &s);
        if (rc != HF_OK) return cleanup(rc);
        B->sys.push_back(s);
    }
    // packed layout
    B->eoff_h.resize(n_mol + 1);
    B->eoff_h[0] = 0;
    for (int m = 0; m < n_mol; m++) B->eoff_h[m + 1] = B->eoff_h[m] + (long long)B->sys[m]->n_bf * B->sys[m]->n_bf;
    B->len = B->eoff_h[n_mol];
    std::vector<MolMat> mm(n_mol);
    for (int m = 0; m < n_mol; m++) {
        hf_system* s = B->sys[m];
        mm[m].N = s->n_bf;
        mm[m].pad = 0;
        mm[m].off = B->eoff_h[m];
        mm[m].comp_norm = s->comp_norm.as<double>();
        mm[m].P64 = s->P64.as<double>();
        mm[m].Jt = s->Jt.as<double>();
        mm[m].Kt = s->Kt.as<double>();
        mm[m].H = s->H.as<double>();
    }
    int rc = HF_OK;
    if ((rc = B->eoff.alloc(sizeof(long long) * (n_mol + 1))) != HF_OK) return cleanup(rc);
    if ((rc = B->mm.alloc(sizeof(MolMat) * n_mol)) != HF_OK) return cleanup(rc);
    if ((rc = B->Pin.alloc(sizeof(double) * B->len)) != HF_OK) return cleanup(rc);
    if ((rc = B->Fout.alloc(sizeof(double) * B->len)) != HF_OK) return cleanup(rc);
    if ((rc = B->E.alloc(sizeof(double) * n_mol)) != HF_OK) return cleanup(rc);
    if ((rc = B->bad.alloc(sizeof(int))) != HF_OK) return cleanup(rc);
    if ((rc = B->counters.alloc(sizeof(unsigned long long) * kNumClasses)) != HF_OK) return cleanup(rc);
    if (cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(cuda_status(cudaGetLastError(), "hf_batch: stream"));
    cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    cudaEventCreate(&B->t0);
    cudaEventCreate(&B->t1);
    cudaMemcpyAsync(B->eoff.p, B->eoff_h.data(), sizeof(long long) * (n_mol + 1), cudaMemcpyHostToDevice, B->st);
    cudaMemcpyAsync(B->mm.p, mm.data(), sizeof(MolMat) * n_mol, cudaMemcpyHostToDevice, B->st);
    for (int c = 0; c < kNumClasses; c++) {
        const int Xc = kEriClasses[c].X, Yc = kEriClasses[c].Y;
        std::vector<MolClass> mc(n_mol);
        std::vector<long long> off(n_mol + 1, 0);
        for (int m = 0; m < n_mol; m++) {
            hf_system* s = B->sys[m];
            MolClass& d = mc[m];
            memset(&d, 0, sizeof(d));
            d.pairs = s->pairs.as<PairHdr>();
            d.prims64 = s->prims64.p;
            d.bra = s->class_ids[Xc].as<int>();
            d.ket = s->class_ids[Yc].as<int>();
            d.offsets = s->plan[c].offsets64.as<long long>();
            d.n_bra = s->class_count[Xc];
            d.same = Xc == Yc;
            d.N = s->n_bf;
            d.P64 = s->P64.as<double>();
            d.Jt = s->Jt.as<double>();
            d.Kt = s->Kt.as<double>();
            off[m + 1] = off[m] + s->plan[c].n64;
        }
        B->n_total[c] = off[n_mol];
        if ((rc = B->mols[c].alloc(sizeof(MolClass) * n_mol)) != HF_OK) return cleanup(rc);
        if ((rc = B->moloff[c].alloc(sizeof(long long) * (n_mol + 1))) != HF_OK) return cleanup(rc);
        cudaMemcpyAsync(B->mols[c].p, mc.data(), sizeof(MolClass) * n_mol, cudaMemcpyHostToDevice, B->st);
        cudaMemcpyAsync(B->moloff[c].p, off.data(), sizeof(long long) * (n_mol + 1), cudaMemcpyHostToDevice, B->st);
        cudaStreamSynchronize(B->st);  // the host vectors go out of scope
        if (cudaStreamCreateWithFlags(&B->cst[c], cudaStreamNonBlocking) != cudaSuccess)
            return cleanup(cuda_status(cudaGetLastError(), "hf_batch: class stream"));
        cudaEventCreateWithFlags(&B->join[c], cudaEventDisableTiming);
        B->block[c] = 128;
        B->chunk[c] = 128;
        B->bps[c] = 4;
    }
    if (cudaStreamSynchronize(B->st) != cudaSuccess) return cleanup(cuda_status(cudaGetLastError(), "hf_batch: setup"));
    if ((rc = capture_graph(B)) != HF_OK) return cleanup(rc);
    *out = B;
    return HF_OK;
}

void hf_batch_destroy(hf_batch* B)
{
    if (!B) return;
    BatchDevice g(B->device);
    cudaStreamSynchronize(B->st);
    delete B;
}

int hf_batch_get_info(const hf_batch* B, hf_batch_info* info)
{
    if (!B || !info) return bfail(HF_E_INVALID, "hf_batch_get_info: NULL argument");
    memset(info, 0, sizeof(*info));
    info->n_mol = B->n_mol;
    info->packed_len = B->len;
    for (int c = 0; c < kNumClasses; c++) {
        info->class_quartets[c] = B->n_total[c];
        info->quartets += B->n_total[c];
        info->block[c] = B->block[c];
        info->chunk[c] = B->chunk[c];
        info->blocks_per_sm[c] = B->bps[c];
    }
    for (int m = 0; m < B->n_mol; m++) info->n_bf_total += B->sys[m]->n_bf;
    return HF_OK;
}

int hf_batch_offsets(const hf_batch* B, int64_t* off)
{
    if (!B || !off) return bfail(HF_E_INVALID, "hf_batch_offsets: NULL argument");
    for (int m = 0; m <= B->n_mol; m++) off[m] = B->eoff_h[m];
    return HF_OK;
}

int hf_fock_build_batch(hf_batch* B, const double* P, double* F, double* E_elec, float* ms, int flags)
{
    if (!B || !P || !F) return bfail(HF_E_INVALID, "hf_fock_build_batch: NULL argument");
    BatchDevice g(B->device);
    cudaStream_t st = B->st;
    const bool dev = (flags & HF_PTR_DEVICE) != 0;
    const size_t bytes = sizeof(double) * B->len;
    if (flags & HF_BATCH_SEQUENTIAL) {
        // one hf_fock_build per molecule on the context stream (the unbatched reference)
        hf_ctx* ctx = B->ctx;
        HF_CUDA(cudaEventRecord(B->t0, ctx->stream));
        for (int m = 0; m < B->n_mol; m++) {
            double e = 0.0;
            const int rc = hf_fock_build(B->sys[m], P + B->eoff_h[m], F + B->eoff_h[m], nullptr, nullptr,
                                         E_elec ? &e : nullptr, nullptr, dev ? HF_PTR_DEVICE : HF_PTR_HOST);
            if (rc != HF_OK) return rc;
            if (E_elec) E_elec[m] = e;
        }
        HF_CUDA(cudaEventRecord(B->t1, ctx->stream));
        HF_CUDA(cudaEventSynchronize(B->t1));
        if (ms) cudaEventElapsedTime(ms, B->t0, B->t1);
        return HF_OK;
    }
    HF_CUDA(cudaMemcpyAsync(B->Pin.p, P, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    HF_CUDA(cudaEventRecord(B->t0, st));
    HF_CUDA(cudaGraphLaunch(B->exec, st));
    HF_CUDA(cudaEventRecord(B->t1, st));
    int bad = 0;
    HF_CUDA(cudaMemcpyAsync(&bad, B->bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    if (bad) return bfail(HF_E_INVALID, "hf_fock_build_batch: a density is not finite or not symmetric");
    HF_CUDA(cudaMemcpyAsync(F, B->Fout.p, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (E_elec) HF_CUDA(cudaMemcpyAsync(E_elec, B->E.p, sizeof(double) * B->n_mol, cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    if (ms) cudaEventElapsedTime(ms, B->t0, B->t1);
    return HF_OK;
}

int hf_batch_tune(hf_batch* B, const char* cache_path, int64_t sample_quartets)
{
    if (!B) return bfail(HF_E_INVALID, "hf_batch_tune: NULL batch");
    BatchDevice g(B->device);
    cudaStream_t st = B->st;
    // cached choices
    bool have[kNumClasses] = {};
    if (cache_path) {
        FILE* f = fopen(cache_path, "r");
        if (f) {
            char name[32];
            int bl, ch, bp;
            while (fscanf(f, "%31s %d %d %d", name, &bl, &ch, &bp) == 4)
                for (int c = 0; c < kNumClasses; c++)
                    if (!strcmp(name, kEriClasses[c].name) && bl > 0 && bl <= 256 && ch > 0 && bp > 0 && bp <= 16) {
                        B->block[c] = bl;
                        B->chunk[c] = ch;
                        B->bps[c] = bp;
                        have[c] = true;
                    }
            fclose(f);
        }
    }
    const int blocks[] = {64, 128, 256};
    const int chunks[] = {32, 128, 512};
    const int bpss[] = {2, 4, 8};
    for (int c = 0; c < kNumClasses; c++) {
        if (have[c] || B->n_total[c] <= 0) continue;
        // sample about 2e10 algorithmic operations per candidate launch (a few ms), at most sample_quartets
        const double per_quartet = 81.0 * kEriClasses[c].prim_flops + kEriClasses[c].cont_flops;
        long long limit = (long long)(2e10 / per_quartet);
        limit = std::max(2048LL, std::min(limit, sample_quartets > 0 ? (long long)sample_quartets : 2000000LL));
        float best = 1e30f;
        int best_bl = B->block[c], best_ch = B->chunk[c], best_bp = B->bps[c];
        for (int bl : blocks)
            for (int ch : chunks)
                for (int bp : bpss) {
                    BatchArgs a = batch_args(B, c, limit);
                    a.chunk = ch;
                    HF_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st));
                    kEriClasses[c].launch_batch(a, B->num_sms * bp, bl, st);  // warm-up
                    HF_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st));
                    HF_CUDA(cudaEventRecord(B->t0, st));
                    kEriClasses[c].launch_batch(a, B->num_sms * bp, bl, st);
                    HF_CUDA(cudaEventRecord(B->t1, st));
                    HF_CUDA(cudaEventSynchronize(B->t1));
                    HF_CUDA(cudaGetLastError());
                    float t = 0.f;
                    cudaEventElapsedTime(&t, B->t0, B->t1);
                    if (t < best) {
                        best = t;
                        best_bl = bl;
                        best_ch = ch;
                        best_bp = bp;
                    }
                }
        B->block[c] = best_bl;
        B->chunk[c] = best_ch;
        B->bps[c] = best_bp;
    }
    if (cache_path) {
        FILE* f = fopen(cache_path, "w");
        if (f) {
            for (int c = 0; c < kNumClasses; c++)
                fprintf(f, "%s %d %d %d\n", kEriClasses[c].name, B->block[c], B->chunk[c], B->bps[c]);
            fclose(f);
        }
    }
    return capture_graph(B);
}

}  // extern "C"

// hf_fock_build_noalloc: the Fock build of hf_fock_build for callers that
// cannot allocate device memory at call time (for example code running under
// a memory pool that forbids cudaMalloc, or a caller that has reserved all
// device memory up front).  Its scratch (the raw-normalised density, the
// unsymmetrised J and K accumulators and a status flag) lives in one
// file-scope __device__ array of fixed size instead of per-system buffers, so
// the call itself allocates nothing: no cudaMalloc, no cudaFree, no
// allocating library routine.
//
// Limits and sharing:
//   - systems with at most HF_NOALLOC_MAX_BF (512) basis functions;
//   - the array is one per device for the life of the process and every call
//     on that device uses it; the accumulators are cleared at the start of
//     each call, so a call does not see the previous call's results, but two
//     calls whose device work overlaps (different streams, or different
//     threads on one stream without ordering) race on the array;
//   - the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) and caches it; make that first call before any
//     stream capture.
#include <string.h>

#include <mutex>
#include <string>

#include "eri_common.cuh"
#include "hf_internal.h"
#include "setup.cuh"

namespace hf {
namespace {

constexpr size_t kNoAllocN2 = (size_t)HF_NOALLOC_MAX_BF * HF_NOALLOC_MAX_BF;

struct NoAllocScratch {
    double P64[kNoAllocN2];
    double Jt[kNoAllocN2];
    double Kt[kNoAllocN2];
    float P32[kNoAllocN2];
    int bad;
};

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

int noalloc_fail(int code, const std::string& msg)
{
    set_error(code, msg);
    return code;
}

struct NoAllocDeviceGuard {
    int prev = -1;
    explicit NoAllocDeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~NoAllocDeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Device address of the scratch on the current device (looked up once).
int scratch_address(int dev, NoAllocScratch** out)
{
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(HF_E_UNSUPPORTED, "hf_fock_build_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_status(e, "hf_fock_build_noalloc: cudaGetSymbolAddress");
        g_noalloc_addr[dev] = p;
    }
    *out = (NoAllocScratch*)g_noalloc_addr[dev];
    return HF_OK;
}

}  // namespace
}  // namespace hf

using namespace hf;

extern "C" int hf_fock_build_noalloc(hf_system* S, const double* P, double* F, double* J, double* K)
{
    if (!S || !P || !F) return noalloc_fail(HF_E_INVALID, "hf_fock_build_noalloc: NULL system, density or F");
    if (S->n_bf > HF_NOALLOC_MAX_BF)
        return noalloc_fail(HF_E_INVALID, "hf_fock_build_noalloc: system has " + std::to_string(S->n_bf) +
                                              " basis functions; the fixed scratch holds at most " +
                                              std::to_string(HF_NOALLOC_MAX_BF));
    hf_ctx* ctx = S->ctx;
    NoAllocDeviceGuard g(ctx->device);
    NoAllocScratch* sc = nullptr;
    int rc = scratch_address(ctx->device, &sc);
    if (rc != HF_OK) return rc;
    cudaStream_t st = ctx->stream;
    const int N = S->n_bf;
    const size_t NN = (size_t)N * N;
    // density check and raw-normalised copies (into the fixed scratch)
    HF_CUDA(cudaMemsetAsync(&sc->bad, 0, sizeof(int), st));
    if (launch_scale_density(N, P, S->comp_norm.as<double>(), sc->P64, S->th.fp32_cutoff > 0.0 ? sc->P32 : nullptr,
                             &sc->bad, st) != 0)
        return cuda_status(cudaGetLastError(), "hf_fock_build_noalloc: density kernel");
    int bad = 0;
    HF_CUDA(cudaMemcpyAsync(&bad, &sc->bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    if (bad) return noalloc_fail(HF_E_INVALID, "hf_fock_build_noalloc: density is not finite or not symmetric");
    // the accumulators must start at zero on every call
    HF_CUDA(cudaMemsetAsync(sc->Jt, 0, NN * sizeof(double), st));
    HF_CUDA(cudaMemsetAsync(sc->Kt, 0, NN * sizeof(double), st));
    EriArgs a;
    memset(&a, 0, sizeof(a));
    a.pairs = S->pairs.as<PairHdr>();
    a.prims64 = S->prims64.p;
    a.prims32 = S->prims32.p;
    a.N = N;
    a.P64 = sc->P64;
    a.P32 = S->th.fp32_cutoff > 0.0 ? sc->P32 : nullptr;
    a.Jt = sc->Jt;
    a.Kt = sc->Kt;
    a.boys64 = ctx->boys64.as<double>();
    a.boys32 = ctx->boys32.as<float>();
    a.prim_tau = S->th.prim_tau;
    for (int ci = 0; ci < kNumClasses; ci++) {
        const auto& pl = S->plan[ci];
        const int Xc = kEriClasses[ci].X, Yc = kEriClasses[ci].Y;
        a.bra = S->class_ids[Xc].as<int>();
        a.ket = S->class_ids[Yc].as<int>();
        a.n_bra = S->class_count[Xc];
        a.same = Xc == Yc;
        for (int prec = 0; prec < 2; prec++) {
            const long long n = prec ? pl.n32 : pl.n64;
            if (n <= 0) continue;
            a.offsets = prec ? pl.offsets32.as<long long>() : pl.offsets64.as<long long>();
            a.kstart = prec ? pl.kstart32.as<int>() : nullptr;
            a.n_quartets = n;
            const int lanes = (!prec && n < (long long)ctx->num_sms * 256) ? kEriClasses[ci].lanes : 1;
            const long long blocks = (n * lanes + kEriThreads - 1) / kEriThreads;
            const int grid = (int)(blocks < (long long)ctx->num_sms * 16 ? blocks : (long long)ctx->num_sms * 16);
            kEriClasses[ci].launch(a, prec, grid, kEriThreads, st, lanes);
            HF_CUDA(cudaGetLastError());
        }
    }
    if (launch_assemble(N, sc->Jt, sc->Kt, S->comp_norm.as<double>(), S->H.as<double>(), J, K, F, st) != 0)
        return cuda_status(cudaGetLastError(), "hf_fock_build_noalloc: assembly kernel");
    HF_CUDA(cudaStreamSynchronize(st));
    HF_CUDA(cudaGetLastError());
    return HF_OK;
}

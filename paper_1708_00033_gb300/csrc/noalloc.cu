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
//   - the array's device address is looked up when a context is created
//     (hf_create calls noalloc_scratch_address with the context's device
//     current).  That lookup loads this file's module, which is when the
//     driver reserves the array's memory; later calls only use the address
//     the context holds.  A context created after a device reset looks it up
//     again.
#include <string.h>

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

}  // namespace

// Called by hf_create with the context's device current.
int noalloc_scratch_address(void** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_status(e, "hf_create: address of the allocation-free build's scratch");
    *out = p;
    return HF_OK;
}

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
    if (!ctx->noalloc_scratch) return noalloc_fail(HF_E_CUDA, "hf_fock_build_noalloc: the context has no scratch address");
    NoAllocDeviceGuard g(ctx->device);
    NoAllocScratch* sc = (NoAllocScratch*)ctx->noalloc_scratch;
    cudaStream_t st = ctx->stream;
    const int N = S->n_bf;
    const size_t NN = (size_t)N * N;
    const bool mixed = S->th.fp32_cutoff > 0.0;
    // density check and raw-normalised copies (into the fixed scratch); the flag stays on the device,
    // where the ERI and assembly kernels skip their work when it is set
    HF_CUDA(cudaMemsetAsync(&sc->bad, 0, sizeof(int), st));
    if (launch_scale_density(N, P, S->comp_norm.as<double>(), sc->P64, mixed ? sc->P32 : nullptr, &sc->bad, st) != 0)
        return cuda_status(cudaGetLastError(), "hf_fock_build_noalloc: density kernel");
    // the accumulators must start at zero on every call
    HF_CUDA(cudaMemsetAsync(sc->Jt, 0, NN * sizeof(double), st));
    HF_CUDA(cudaMemsetAsync(sc->Kt, 0, NN * sizeof(double), st));
    EriArgs a;
    memset(&a, 0, sizeof(a));
    a.P64 = sc->P64;
    a.P32 = mixed ? sc->P32 : nullptr;
    a.Jt = sc->Jt;
    a.Kt = sc->Kt;
    a.n_copies = 1;
    a.bad = &sc->bad;
    int rc = launch_eri_classes(S, a, 0, 1, 0, nullptr, nullptr);
    if (rc != HF_OK) return rc;
    if (launch_assemble(N, sc->Jt, sc->Kt, S->comp_norm.as<double>(), S->H.as<double>(), J, K, F, &sc->bad, st) != 0)
        return cuda_status(cudaGetLastError(), "hf_fock_build_noalloc: assembly kernel");
    int bad = 0;
    HF_CUDA(cudaMemcpyAsync(&bad, &sc->bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    HF_CUDA(cudaStreamSynchronize(st));
    HF_CUDA(cudaGetLastError());
    if (bad) return noalloc_fail(HF_E_INVALID, "hf_fock_build_noalloc: density is not finite or not symmetric");
    return HF_OK;
}

// Device microbenchmarks that give the denominators of the ERI and digestion
// rooflines: FP64 and FP32 FMA throughput (the ERI kernels are bound by the
// FP64 FMA pipe, their FP32 variants by the FP32 pipe) and FP64 atomic-add
// throughput (the digestion of Eq. 1a-1f), each timed with CUDA events.
#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>
#include <string>

#include "hf_internal.h"

namespace hf {

// CH independent FMA chains per thread; the result is stored only under a
// condition that never holds, so the chains are not removed
template <typename T, int CH>
__global__ void k_fma_chains(T* out, int iters, T a, T b)
{
    T x[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++) x[c] = x[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s += x[c];
    if (s == (T)-1.2345) out[0] = s;
}

// iters FP64 atomic adds per thread at hash-scattered addresses of buf[0..mask]
__global__ void k_red_random(double* buf, unsigned mask, int iters)
{
    unsigned h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u;
    for (int i = 0; i < iters; i++) {
        h = h * 1664525u + 1013904223u;
        atomicAdd(&buf[(h >> 8) & mask], 1.0);
    }
}

// the same count with consecutive threads on consecutive addresses
__global__ void k_red_coalesced(double* buf, unsigned mask, int iters)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = 0; i < iters; i++) atomicAdd(&buf[(t + (unsigned)i * 4096u) & mask], 1.0);
}

namespace {

int peaks_fail(int code, const std::string& msg)
{
    set_error(code, msg);
    return code;
}

struct PeaksDeviceGuard {
    int prev = -1;
    explicit PeaksDeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~PeaksDeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace hf

using namespace hf;

extern "C" int hf_measure_peaks(hf_ctx* ctx, hf_peaks* out)
{
    if (!ctx || !out) return peaks_fail(HF_E_INVALID, "hf_measure_peaks: NULL argument");
    PeaksDeviceGuard g(ctx->device);
    cudaStream_t st = ctx->stream;
    const int nsm = ctx->num_sms;
    constexpr unsigned kAtomicDoubles = 1u << 20;  // 8 MB target: resident in L2, like the Fock accumulators
    DevBuf sink, buf;
    if (sink.alloc(64) != HF_OK || buf.alloc(kAtomicDoubles * sizeof(double)) != HF_OK)
        return peaks_fail(HF_E_NOMEM, "hf_measure_peaks: cannot allocate the benchmark buffers");
    HF_CUDA(cudaMemsetAsync(buf.p, 0, kAtomicDoubles * sizeof(double), st));
    cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[1];
    float ms = 0.0f;
    memset(out, 0, sizeof(*out));
    // best of three timed launches after one warm-up
    auto best = [&](auto&& launch, double work) -> double {
        launch();
        double r = 0.0;
        for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(e0, st);
            launch();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
            cudaEventElapsedTime(&ms, e0, e1);
            r = std::max(r, work / (ms * 1e-3));
        }
        return r;
    };
    const int threads = 512, blocks = 2 * nsm;
    {
        const int iters = 4096;
        const double flops = 2.0 * 8 * iters * (double)threads * blocks;
        out->fp64_fma_gflops =
            best([&] { k_fma_chains<double, 8><<<blocks, threads, 0, st>>>(sink.as<double>(), iters, 1.0000001, 1e-9); },
                 flops) * 1e-9;
    }
    {
        const int iters = 65536;
        const double flops = 2.0 * 8 * iters * (double)threads * blocks;
        out->fp32_fma_gflops =
            best([&] { k_fma_chains<float, 8><<<blocks, threads, 0, st>>>(sink.as<float>(), iters, 1.0000001f, 1e-9f); },
                 flops) * 1e-9;
    }
    {
        const int iters = 1024, ab = nsm * 8, at = 256;
        const double ops = (double)iters * ab * at;
        out->red_add_f64_random_gops =
            best([&] { k_red_random<<<ab, at, 0, st>>>(buf.as<double>(), kAtomicDoubles - 1, iters); }, ops) * 1e-9;
        out->red_add_f64_coalesced_gops =
            best([&] { k_red_coalesced<<<ab, at, 0, st>>>(buf.as<double>(), kAtomicDoubles - 1, iters); }, ops) * 1e-9;
    }
    HF_CUDA(cudaGetLastError());
    HF_CUDA(cudaStreamSynchronize(st));
    if (out->fp64_fma_gflops < 0 || out->fp32_fma_gflops < 0 || out->red_add_f64_random_gops < 0)
        return peaks_fail(HF_E_CUDA, "hf_measure_peaks: timing failed");
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, ctx->device);
    out->sm_max_mhz = clk / 1000.0;
    out->num_sms = nsm;
    return HF_OK;
}

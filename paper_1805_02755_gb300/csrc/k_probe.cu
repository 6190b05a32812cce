// FP32 pipe probe: the measured side of the FP32-bound rooflines.  Each
// work-item runs eight independent chains x <- x * m + c (with m, c near 1
// and 0 the chains contract toward c / (1 - m), never overflow and never go
// subnormal) for 16 x iters steps each and writes their sum, so every FFMA
// stays in the program.  With eight chains per thread and every CTA slot of
// the SM filled, the FFMA latency is covered and the run time is set by the
// FP32 pipe: FFMAs per second = 128 x iters x work-items / time.
#include <cuda_runtime.h>

#include "ecl_internal.h"
#include "sched.cuh"

namespace ecl {
namespace {

constexpr int kBlock = 256;
constexpr int kChains = 8;
constexpr int kSteps = 16;  // steps per chain and loop iteration

struct ProbeParams {
    float *out;
    int32_t iters;
    float m, c;
    uint32_t lws;
};

struct ProbeBody {
    using Params = ProbeParams;
    Params p;

    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const uint64_t wi = (off + t) * p.lws + threadIdx.x;
        float x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = 1.0f + (float)(wi & 255u) * 1e-3f + (float)k * 1e-4f;
        for (int32_t i = 0; i < p.iters; ++i) {
#pragma unroll
            for (int u = 0; u < kSteps; ++u) {
#pragma unroll
                for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], p.m, p.c);
            }
        }
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += x[k];
        p.out[wi] = s;
    }
};

__global__ void __launch_bounds__(kBlock) k_fp32_probe(ProbeParams prm, SchedArgs s)
{
    ProbeBody b;
    b.p = prm;
    drive(s, b);
}

// out float[gws], iters, m, c
ecl_status validate(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    if (lws != kBlock) {
        err = "lws must be 256";
        return ECL_ERR_SIZE;
    }
    if (a.i32(1) < 1) {
        err = "iters must be >= 1";
        return ECL_ERR_ARG;
    }
    if (a.bytes[0] < gws * sizeof(float)) {
        err = "out holds fewer than gws floats";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

uint64_t grain(const KArgs &, uint64_t, uint32_t) { return 1; }

uint32_t nchunks(const KArgs &, uint64_t, uint32_t, uint64_t, uint64_t len) { return (uint32_t)len; }

int ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fp32_probe, kBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ecl_status launch(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    ProbeParams p;
    p.out = a.buf<float>(0);
    p.iters = a.i32(1);
    p.m = a.f32(2);
    p.c = a.f32(3);
    p.lws = c.lws;
    k_fp32_probe<<<c.grid, kBlock, 0, c.stream>>>(p, s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

}  // namespace

extern const KernelDesc kFp32Probe = {
    "fp32_probe", 4,
    {{"out", A_BUF_OUT}, {"iters", A_I32}, {"m", A_F32}, {"c", A_F32}},
    1, 1, kBlock, 0, validate, grain, nchunks, ctas_per_sm, launch,
};

}  // namespace ecl

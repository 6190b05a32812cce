// Binomial option pricing (Listing 1 workload: one work-group per option
// lattice, out pattern 1:lws) for a batch of European calls of uneven depth
// N = 1..2048 on a Cox-Ross-Rubinstein lattice, FP32.
//
// One warp (the work-group, lws 32) prices one option.  Level t of the
// lattice holds nodes j = 0..t; node j lives in lane j / R, register slot
// j % R, with R in {64, 32, ..., 1}.  A backward step needs node j+1: in the
// same lane except for the last slot, which one shuffle per level brings
// from the next lane.  When the live nodes fit in half the registers the
// warp repacks to R/2 (one shuffle per slot), so at least half of every
// lane's slots stay live.
//
// Arithmetic (exact in real numbers, arranged for FP32):
//   p = 1/2 + q,  q = (expm1(r dt) - 2 sinh^2(a/2)) / (2 sinh a),  a = sigma sqrt(dt)
// is the CRR probability (e^{r dt} - d)/(u - d) written so that the large
// part 1/2 is exact and only the small q carries rounding.  The lattice is
// stored scaled by 2 per level, B = 2^(N-t) V / disc^(N-t), so one node
// update is  B_j <- (B_{j+1} + B_j) + 2q (B_{j+1} - B_j)  (add, sub, FMA);
// every 32 levels all nodes are multiplied by 2^-32 (exact) and the power
// is removed at the end together with disc^N = e^{-rT}.
// In-the-money calls (S > K) are priced through the put on the same lattice
// and put-call parity, which holds exactly on a CRR lattice:
//   C = P + S - K e^{-rT},  dC/dS = dP/dS + 1,  dC/dsigma = dP/dsigma.
// The put lattice of a deep in-the-money call holds small values, while the
// call lattice would carry two large vega terms (leaf and dq/dsigma parts)
// that cancel, losing several digits in FP32.
// Greeks are the exact derivatives of this discrete price (forward mode):
//   delta tree: same recursion, leaves u^j d^(N-j) for in-the-money leaves;
//   vega tree:  dB_j <- (dB_{j+1} + dB_j) + 2q (dB_{j+1} - dB_j) + 2q' (B_{j+1} - B_j),
//               q' = dq/dsigma = sqrt(dt) (-1/2 - q coth a),
//               leaves S_T (2j - N) sqrt(dt) for in-the-money leaves.
#include <cuda_runtime.h>

#include "ecl_internal.h"
#include "sched.cuh"

namespace ecl {
namespace {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

struct BinoParams {
    const float *S, *K, *T, *sigma;
    const int *steps;
    float r;
    int64_t n;
    float *price;
    float2 *greeks;  // (delta, vega) or nullptr
};

struct Lat {
    float q2;      // 2q
    float q2p;     // 2 dq/dsigma
    int active;    // live nodes at the current level
    int rescale;   // levels since the last rescale
    int shift;     // power of two still to remove from the result
};

template <int R, bool G>
__device__ __forceinline__ void level(float (&B)[R], float (&D)[R], float (&V)[R], Lat &L)
{
    const float bn = __shfl_down_sync(kFull, B[0], 1);
    float dn = 0.f, vn = 0.f;
    if (G) {
        dn = __shfl_down_sync(kFull, D[0], 1);
        vn = __shfl_down_sync(kFull, V[0], 1);
    }
#pragma unroll
    for (int s = 0; s < R; ++s) {
        const float up = (s + 1 < R) ? B[s + 1] : bn;
        const float diff = up - B[s];
        if (G) {
            const float dup = (s + 1 < R) ? D[s + 1] : dn;
            const float vup = (s + 1 < R) ? V[s + 1] : vn;
            V[s] = fmaf(L.q2p, diff, fmaf(L.q2, vup - V[s], vup + V[s]));
            D[s] = fmaf(L.q2, dup - D[s], dup + D[s]);
        }
        B[s] = fmaf(L.q2, diff, up + B[s]);
    }
    L.active -= 1;
    if (++L.rescale == 32) {
        L.rescale = 0;
        L.shift -= 32;
#pragma unroll
        for (int s = 0; s < R; ++s) {
            B[s] *= 0x1p-32f;
            if (G) {
                D[s] *= 0x1p-32f;
                V[s] *= 0x1p-32f;
            }
        }
    }
}

// Runs levels with R slots per lane until the live nodes fit in R/2, then
// repacks and continues with R/2.
template <int R, bool G>
__device__ __forceinline__ void phase(float (&B)[R], float (&D)[R], float (&V)[R], Lat &L)
{
    const int lane = threadIdx.x & 31;
    const int limit = (R > 1) ? kWarp * (R / 2) : 1;
    while (L.active > limit) level<R, G>(B, D, V, L);
    if constexpr (R > 1) {
        constexpr int H = R / 2;
        float b2[H], d2[H], v2[H];
        const int src = lane >> 1;
        const bool odd = lane & 1;
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const float lo = __shfl_sync(kFull, B[s], src), hi = __shfl_sync(kFull, B[H + s], src);
            b2[s] = odd ? hi : lo;
            if (G) {
                const float dl = __shfl_sync(kFull, D[s], src), dh = __shfl_sync(kFull, D[H + s], src);
                const float vl = __shfl_sync(kFull, V[s], src), vh = __shfl_sync(kFull, V[H + s], src);
                d2[s] = odd ? dh : dl;
                v2[s] = odd ? vh : vl;
            }
        }
        phase<H, G>(b2, d2, v2, L);
        if (lane == 0) {
            B[0] = b2[0];
            if (G) {
                D[0] = d2[0];
                V[0] = v2[0];
            }
        }
    }
}

// Leaves and the first backward level for R slots per lane, then the rest.
template <int R, bool G>
__device__ __forceinline__ void price_option(const BinoParams &p, int64_t o)
{
    const int lane = threadIdx.x & 31;
    const float S = __ldg(p.S + o), K = __ldg(p.K + o), T = __ldg(p.T + o), sig = __ldg(p.sigma + o);
    const int N = __ldg(p.steps + o);
    const float dt = T / (float)N;
    const float sdt = sqrtf(dt);
    const float a = sig * sdt;
    const float sh = sinhf(0.5f * a);
    const float num = expm1f(p.r * dt) - 2.0f * sh * sh;
    const float s1 = sinhf(a);
    const float q = num / (2.0f * s1);
    Lat L;
    L.q2 = 2.0f * q;
    L.q2p = 2.0f * sdt * (-0.5f - q * (coshf(a) / s1));
    L.active = N;  // nodes of level N-1
    L.rescale = 0;
    L.shift = N;
    const bool put = S > K;  // price the out-of-the-money side, then parity
    float B[R], D[R], V[R];
    // level N-1 directly from the leaves j and j+1
    float lb = 0.f, ld = 0.f, lv = 0.f;  // leaf j of the previous slot (j+1 of this one)
#pragma unroll
    for (int s = R; s >= 0; --s) {
        const int j = lane * R + s;
        float b = 0.f, d = 0.f, v = 0.f;
        if (j <= N) {
            const float m = (float)(2 * j - N);
            const float g = expf(a * m);
            const float ST = S * g;
            if (put ? (ST < K) : (ST > K)) {
                b = put ? K - ST : ST - K;
                if (G) {
                    d = put ? -g : g;
                    v = put ? -(ST * m * sdt) : ST * m * sdt;
                }
            }
        }
        if (s < R) {
            const float diff = lb - b;
            B[s] = fmaf(L.q2, diff, lb + b);
            if (G) {
                D[s] = fmaf(L.q2, ld - d, ld + d);
                V[s] = fmaf(L.q2p, diff, fmaf(L.q2, lv - v, lv + v));
            }
        }
        lb = b;
        ld = d;
        lv = v;
    }
    L.rescale = 1;
    phase<R, G>(B, D, V, L);
    if (lane == 0) {
        // remove the remaining 2^shift (exact), then discount
        const float disc = expf(-p.r * T);
        const float scale = ldexpf(disc, -L.shift);
        float price = B[0] * scale, delta = D[0] * scale;
        if (put) {
            price += S - K * disc;
            delta += 1.0f;
        }
        p.price[o] = price;
        if (G) p.greeks[o] = make_float2(delta, V[0] * scale);
    }
}

template <bool G>
__device__ void dispatch(const BinoParams &p, int64_t o)
{
    const int N = __ldg(p.steps + o);
    if (N < 1 || N > 2048) {  // outside the supported depths: NaN results
        if ((threadIdx.x & 31) == 0) {
            p.price[o] = __int_as_float(0x7fc00000);
            if (G) p.greeks[o] = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
        }
        return;
    }
    if (N > 1024) price_option<64, G>(p, o);
    else if (N > 512) price_option<32, G>(p, o);
    else if (N > 256) price_option<16, G>(p, o);
    else if (N > 128) price_option<8, G>(p, o);
    else if (N > 64) price_option<4, G>(p, o);
    else if (N > 32) price_option<2, G>(p, o);
    else price_option<1, G>(p, o);
}

template <bool G>
struct BinoBody {
    using Params = BinoParams;
    Params p;

    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const int64_t o = (int64_t)(off + t);
        if (o < p.n) dispatch<G>(p, o);
    }
};

template <bool G>
__global__ void __launch_bounds__(kWarp) k_binomial(BinoParams prm, SchedArgs s)
{
    BinoBody<G> b;
    b.p = prm;
    drive(s, b);
}

int occ(const void *fn)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kWarp, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ecl_status validate(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    const int64_t n = a.i32(6);
    if (n <= 0) {
        err = "options must be positive";
        return ECL_ERR_ARG;
    }
    if (lws != kWarp) {
        err = "lws must be 32 (one warp prices one option)";
        return ECL_ERR_SIZE;
    }
    if (gws < (uint64_t)n * kWarp) {
        err = "the NDRange (32 work-items per option) does not cover the options";
        return ECL_ERR_SIZE;
    }
    for (int i = 0; i < 5; ++i)
        if (a.bytes[i] < (uint64_t)n * 4) {
            err = "input buffers must hold n values";
            return ECL_ERR_BUFFER;
        }
    if (a.bytes[7] < (uint64_t)n * 4) {
        err = "price buffer must hold n floats";
        return ECL_ERR_BUFFER;
    }
    if (a.ptr[8] && (a.bytes[8] < (uint64_t)n * 8 || (uintptr_t)a.ptr[8] % 8)) {
        err = "greeks buffer must be an aligned float2[n]";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

uint64_t grain(const KArgs &, uint64_t, uint32_t) { return 1; }

uint32_t nchunks(const KArgs &, uint64_t, uint32_t, uint64_t, uint64_t len) { return (uint32_t)len; }

int ctas_per_sm() { return occ((const void *)k_binomial<true>); }

ecl_status launch(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    BinoParams p;
    p.S = a.buf<const float>(0);
    p.K = a.buf<const float>(1);
    p.T = a.buf<const float>(2);
    p.sigma = a.buf<const float>(3);
    p.steps = a.buf<const int>(4);
    p.r = a.f32(5);
    p.n = a.i32(6);
    p.price = a.buf<float>(7);
    p.greeks = a.buf<float2>(8);
    if (p.greeks)
        k_binomial<true><<<c.grid, kWarp, 0, c.stream>>>(p, s);
    else
        k_binomial<false><<<c.grid, kWarp, 0, c.stream>>>(p, s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

}  // namespace

extern const KernelDesc kBinomial = {
    "binomial", 9,
    {{"S", A_BUF_IN}, {"K", A_BUF_IN}, {"T", A_BUF_IN}, {"sigma", A_BUF_IN}, {"steps", A_BUF_IN},
     {"r", A_F32}, {"n", A_I32}, {"price", A_BUF_OUT}, {"greeks", A_BUF_OUT_OPT}},
    1, 0, kWarp, 0, validate, grain, nchunks, ctas_per_sm, launch,
};

}  // namespace ecl

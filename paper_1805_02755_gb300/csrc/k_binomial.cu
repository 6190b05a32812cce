// Binomial option pricing (Listing 1 workload: one work-group per option
// lattice, out pattern 1:lws) for a batch of European calls of uneven depth
// N = 1..2048 on a Cox-Ross-Rubinstein lattice, FP32.
//
// One warp (the work-group, lws 32) prices one option.  Level t of the
// lattice holds nodes j = 0..t; node j lives in lane j / R, register slot
// j % R, where the width R steps down 64, 56, 48, ..., 2, 1 as the lattice
// shrinks; a lattice starts at the narrowest width that holds its leaves
// (each width's code exists once and is entered by index).  A backward step needs node j+1: in the same lane except for the
// last slot, which one shuffle per level brings from the next lane.  When
// the live nodes fit in the next width the warp repacks its registers
// through a padded shared buffer, so ~90% of the computed slots stay live.
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
// Greeks are the exact derivatives of this discrete price.  Forward mode
// through one level gives
//   delta tree: the same recursion, leaves u^j d^(N-j) for in-the-money leaves;
//   vega tree:  dB_j <- (dB_{j+1} + dB_j) + 2q (dB_{j+1} - dB_j) + 2q' (B_{j+1} - B_j),
//               q' = dq/dsigma = sqrt(dt) (-1/2 - q coth a),
//               leaves S_T (2j - N) sqrt(dt) for in-the-money leaves.
// The level operator L = (1 + 2q) shift + (1 - 2q) identity and the
// difference operator (shift - identity) are both shift-invariant, so they
// commute, and the N coefficient terms of the vega tree add up to
//   N 2q' (B_1 - B_0)   (B_1, B_0: the two nodes of level 1, same scaling).
// So delta, the leaf part of vega and the price are three independent
// lattices of the same recursion: the warp runs the price code three times
// with different leaves, keeps B_1 - B_0 from the price pass, and
//   vega = root(vega leaves) + N 2q' (B_1 - B_0).
// This is the same derivative; in FP32 emulation its error matches the
// level-by-level form (~1e-6 relative).
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
    int active;    // live nodes at the current level
    int rescale;   // levels since the last rescale
    int shift;     // power of two still to remove from the result
};

// Lane widths (nodes per lane) the warp steps through as the lattice shrinks.
// Going from width R to the next width R' happens when the live nodes fit in
// 32 R'.  Every width is a fully unrolled level loop plus a repack, so the
// list trades computed-but-dead slots against code size: measured on the
// 2^20-option batch (price + greeks), finer lists (33 widths: ~96% live
// slots) ran up to 2x slower on instruction fetch, and this 14-width list
// (~88% live) was the fastest of eight candidates.
constexpr int kWidths[] = {64, 56, 48, 40, 32, 28, 24, 20, 16, 12, 8, 4, 2, 1};
constexpr int kNWidths = sizeof(kWidths) / sizeof(kWidths[0]);
__host__ __device__ constexpr int width_at(int i) { return i < kNWidths ? kWidths[i] : 0; }
constexpr int kMaxR = 64;
constexpr int kMaxSteps = kWarp * kMaxR;               // deepest lattice: 2048 steps
constexpr int kShNodes = kMaxSteps + 1 + kMaxSteps / 32 + 32;  // leaves 0..N with padding

__device__ __forceinline__ int shidx(int j) { return j + (j >> 5); }  // avoids bank conflicts

// One backward level on the first R slots of B.
template <int R>
__device__ __forceinline__ void level(float (&B)[kMaxR], Lat &L)
{
    const float bn = __shfl_down_sync(kFull, B[0], 1);
#pragma unroll
    for (int s = 0; s < R; ++s) {
        const float up = (s + 1 < R) ? B[s + 1] : bn;
        B[s] = fmaf(L.q2, up - B[s], up + B[s]);
    }
    L.active -= 1;
    if (++L.rescale == 32) {
        L.rescale = 0;
        L.shift -= 32;
#pragma unroll
        for (int s = 0; s < R; ++s) B[s] *= 0x1p-32f;
    }
}

// B[0..R) <- shared nodes lane*R .. lane*R + R - 1 at width R = width_at(WI).
template <int WI>
__device__ __forceinline__ void load_width(float (&B)[kMaxR], const float *sh, int lane)
{
    constexpr int R = width_at(WI);
#pragma unroll
    for (int s = 0; s < R; ++s) B[s] = sh[shidx(lane * R + s)];
}

// Width width_at(WI): levels until the live nodes fit the next width, then
// the repack through the warp's shared buffer.  At the last width (1) the
// levels run down to the root, keeping lane 0's level-1 difference
// d1 = B_1 - B_0 at the root's scaling.
template <int WI>
__device__ __forceinline__ void width_step(float (&B)[kMaxR], Lat &L, float *sh, int lane, float &d1)
{
    constexpr int R = width_at(WI);
    constexpr int R2 = width_at(WI + 1);
    if constexpr (R2 > 0) {
        while (L.active > kWarp * R2) level<R>(B, L);
        __syncwarp();
#pragma unroll
        for (int s = 0; s < R; ++s) sh[shidx(lane * R + s)] = B[s];
        __syncwarp();
        load_width<WI + 1>(B, sh, lane);
    } else {
        while (L.active > 2) level<1>(B, L);
        if (L.active == 2) {
            d1 = __shfl_down_sync(kFull, B[0], 1) - B[0];
            level<1>(B, L);
            if (L.rescale == 0) d1 *= 0x1p-32f;
        }
    }
}

// Runtime width index -> the width's code (each width's code exists once).
template <int WI>
__device__ __forceinline__ void width_step_at(int wi, float (&B)[kMaxR], Lat &L, float *sh, int lane, float &d1)
{
    if constexpr (WI < kNWidths) {
        if (wi == WI) width_step<WI>(B, L, sh, lane, d1);
        else width_step_at<WI + 1>(wi, B, L, sh, lane, d1);
    }
}

template <int WI>
__device__ __forceinline__ void load_width_at(int wi, float (&B)[kMaxR], const float *sh, int lane)
{
    if constexpr (WI < kNWidths) {
        if (wi == WI) load_width<WI>(B, sh, lane);
        else load_width_at<WI + 1>(wi, B, sh, lane);
    }
}

// The narrowest width index whose 32 lanes hold n nodes.
template <int WI>
__device__ __forceinline__ int width_for(int n)
{
    if constexpr (WI + 1 < kNWidths) {
        if (kWarp * width_at(WI + 1) >= n) return width_for<WI + 1>(n);
    }
    return WI;
}

// Per-option constants of the lattice.
struct Opt {
    float S, K, sdt, a, q2;
    int N;
    bool put;
};

// The leaves 0..N of the priced side (zero where out of the money and
// beyond N) into shared buffer 0 (price), and with greeks also into buffers
// 1 (delta: dS_T/dS) and 2 (vega leaf part: dS_T/dsigma), one exp per leaf.
__device__ __forceinline__ void leaves(const Opt &o, float *sh, int lane, bool greeks)
{
    __syncwarp();
    for (int j = lane; j <= kMaxSteps; j += kWarp) {
        float b = 0.f, dl = 0.f, vg = 0.f;
        if (j <= o.N) {
            const float m = (float)(2 * j - o.N);
            const float g = expf(o.a * m);
            const float ST = o.S * g;
            if (o.put ? (ST < o.K) : (ST > o.K)) {
                b = o.put ? o.K - ST : ST - o.K;
                dl = o.put ? -g : g;
                vg = o.put ? -(ST * m * o.sdt) : ST * m * o.sdt;
            }
        }
        sh[shidx(j)] = b;
        if (greeks) {
            sh[kShNodes + shidx(j)] = dl;
            sh[2 * kShNodes + shidx(j)] = vg;
        }
    }
    __syncwarp();
}

// One backward induction from the leaves in `sh` (which it then uses as the
// repack buffer).  Returns the root on lane 0 (scaled by 2^shift) and, on
// lane 0, d1 = B_1 - B_0 of level 1 at the root's scaling.
__device__ __forceinline__ float lattice(const Opt &o, float *sh, int lane, int &shift, float &d1)
{
    Lat L;
    L.q2 = o.q2;
    L.shift = o.N;
    float B[kMaxR];
    int wi;
    if (o.N + 1 <= kMaxSteps) {
        // the N + 1 leaves as level N, at the narrowest width that holds them
        wi = width_for<0>(o.N + 1);
        load_width_at<0>(wi, B, sh, lane);
        L.active = o.N + 1;
        L.rescale = 0;
    } else {
        // N = 2048: 2049 leaves do not fit 32 x 64 slots; level N-1 from the leaves
        wi = 0;
#pragma unroll
        for (int s = 0; s < kMaxR; ++s) {
            const int j = lane * kMaxR + s;
            const float lb = sh[shidx(j + 1)], b = sh[shidx(j)];
            B[s] = fmaf(L.q2, lb - b, lb + b);
        }
        L.active = o.N;
        L.rescale = 1;
    }
    for (;; ++wi) {
        width_step_at<0>(wi, B, L, sh, lane, d1);
        if (wi == kNWidths - 1) break;
    }
    shift = L.shift;
    return B[0];
}

template <bool G>
__device__ __forceinline__ void price_option(const BinoParams &p, int64_t o, float *sh)
{
    const int lane = threadIdx.x & 31;
    const float S = __ldg(p.S + o), K = __ldg(p.K + o), T = __ldg(p.T + o), sig = __ldg(p.sigma + o);
    const int N = __ldg(p.steps + o);
    if (N < 1 || N > kMaxSteps) {  // outside the supported depths: NaN results
        if (lane == 0) {
            p.price[o] = __int_as_float(0x7fc00000);
            if (G && p.greeks) p.greeks[o] = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
        }
        return;
    }
    const float dt = T / (float)N;
    const float sdt = sqrtf(dt);
    const float a = sig * sdt;
    const float sh2 = sinhf(0.5f * a);
    const float num = expm1f(p.r * dt) - 2.0f * sh2 * sh2;
    const float s1 = sinhf(a);
    const float q = num / (2.0f * s1);
    Opt op;
    op.S = S;
    op.K = K;
    op.sdt = sdt;
    op.a = a;
    op.q2 = 2.0f * q;
    op.N = N;
    op.put = S > K;  // price the out-of-the-money side, then parity
    // price, then (greeks) delta and the vega leaf part; one copy of the
    // unrolled level code serves the three passes
    int shift = 0;
    float d1 = 0.f, root[3] = {0.f, 0.f, 0.f};
    const int passes = (G && p.greeks) ? 3 : 1;
    leaves(op, sh, lane, passes == 3);
#pragma unroll 1
    for (int k = 0; k < passes; ++k) {
        float dk;
        const float r = lattice(op, sh + k * kShNodes, lane, shift, dk);
        if (k == 0) {
            root[0] = r;
            d1 = dk;
        } else if (k == 1) {
            root[1] = r;
        } else {
            root[2] = r;
        }
    }
    const float b = root[0];
    float delta = root[1], vega = root[2];
    if (passes == 3) {
        const float q2p = 2.0f * sdt * (-0.5f - q * (coshf(a) / s1));  // 2 dq/dsigma
        vega = fmaf((float)N * q2p, d1, vega);
    }
    if (lane == 0) {
        // remove the remaining 2^shift (exact), then discount
        const float disc = expf(-p.r * T);
        const float scale = ldexpf(disc, -shift);
        float price = b * scale;
        delta *= scale;
        if (op.put) {
            price += S - K * disc;
            delta += 1.0f;
        }
        p.price[o] = price;
        if (G && p.greeks) p.greeks[o] = make_float2(delta, vega * scale);
    }
}

template <bool G>
struct BinoBody {
    using Params = BinoParams;
    Params p;
    float *sh;

    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const int64_t o = (int64_t)(off + t);
        if (o < p.n) price_option<G>(p, o, sh);
    }
};

template <bool G>
__global__ void __launch_bounds__(kWarp) k_binomial(BinoParams prm, SchedArgs s)
{
    __shared__ float sh[(G ? 3 : 1) * kShNodes];
    BinoBody<G> b;
    b.p = prm;
    b.sh = sh;
    drive(s, b);
}

// ---------------------------------------------------------------- batches
// Many option batches of uneven size as one NDRange: instance i owns global
// options [first_i, first_i + n_i); a work-group (option) finds its instance
// by binary search over `first` (ascending, first_0 = 0).  Mirrors
// ecl_binomial_instance in include/ecl.h.
struct BinoInstance {
    const float *S, *K, *T, *sigma;
    const int *steps;
    float *price;
    float2 *greeks;  // may be NULL
    int64_t first;
    int64_t n;
    float r;
    int32_t pad;
};
static_assert(sizeof(BinoInstance) == 80, "ecl_binomial_instance layout");

struct BinoBatchParams {
    const BinoInstance *inst;
    int32_t count;
    int64_t total;
};

template <bool G>
struct BinoBatchBody {
    using Params = BinoBatchParams;
    Params p;
    float *sh;

    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const int64_t o = (int64_t)(off + t);
        if (o >= p.total) return;
        int lo = 0, hi = p.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&p.inst[mid].first) <= o) lo = mid;
            else hi = mid - 1;
        }
        const BinoInstance &in = p.inst[lo];
        const int64_t local = o - in.first;
        if (local < 0 || local >= in.n) return;
        BinoParams bp;
        bp.S = in.S;
        bp.K = in.K;
        bp.T = in.T;
        bp.sigma = in.sigma;
        bp.steps = in.steps;
        bp.r = in.r;
        bp.n = in.n;
        bp.price = in.price;
        bp.greeks = G ? in.greeks : nullptr;
        price_option<G>(bp, local, sh);
    }
};

template <bool G>
__global__ void __launch_bounds__(kWarp) k_binomial_batch(BinoBatchParams prm, SchedArgs s)
{
    __shared__ float sh[(G ? 3 : 1) * kShNodes];
    BinoBatchBody<G> b;
    b.p = prm;
    b.sh = sh;
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

// ---- binomial_batch: table of instances, count, total options, with_greeks
ecl_status v_batch(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    const int64_t count = a.i32(1), total = a.i64(2);
    if (count <= 0 || total <= 0) {
        err = "count and total must be positive";
        return ECL_ERR_ARG;
    }
    if (a.bytes[0] < (uint64_t)count * sizeof(BinoInstance) || (uintptr_t)a.ptr[0] % 16) {
        err = "the instance table must hold count 16-byte aligned entries of 80 bytes";
        return ECL_ERR_BUFFER;
    }
    if (lws != kWarp) {
        err = "lws must be 32 (one warp prices one option)";
        return ECL_ERR_SIZE;
    }
    if (gws < (uint64_t)total * kWarp) {
        err = "the NDRange (32 work-items per option) does not cover the options";
        return ECL_ERR_SIZE;
    }
    return ECL_OK;
}

int batch_ctas_per_sm() { return occ((const void *)k_binomial_batch<true>); }

ecl_status l_batch(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    BinoBatchParams p;
    p.inst = a.buf<const BinoInstance>(0);
    p.count = a.i32(1);
    p.total = a.i64(2);
    if (a.i32(3))
        k_binomial_batch<true><<<c.grid, kWarp, 0, c.stream>>>(p, s);
    else
        k_binomial_batch<false><<<c.grid, kWarp, 0, c.stream>>>(p, s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

}  // namespace

extern const KernelDesc kBinomialBatch = {
    "binomial_batch", 4,
    {{"instances", A_BUF_IN}, {"count", A_I32}, {"total", A_I64}, {"with_greeks", A_I32}},
    1, 0, kWarp, 0, v_batch, grain, nchunks, batch_ctas_per_sm, l_batch,
};

extern const KernelDesc kBinomial = {
    "binomial", 9,
    {{"S", A_BUF_IN}, {"K", A_BUF_IN}, {"T", A_BUF_IN}, {"sigma", A_BUF_IN}, {"steps", A_BUF_IN},
     {"r", A_F32}, {"n", A_I32}, {"price", A_BUF_OUT}, {"greeks", A_BUF_OUT_OPT}},
    1, 0, kWarp, 0, validate, grain, nchunks, ctas_per_sm, launch,
};

}  // namespace ecl

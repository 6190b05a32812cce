// All-pairs NBody (Listing 2: float4 positions (x, y, z, m), softening passed
// squared, lws 64, out pattern 1:1) and the potential-energy family built on
// the same pair loop:
//   nbody          one explicit step: in pos/vel -> out pos/vel
//   nbody_acc      a_i = sum_j m_j d_ij / (|d_ij|^2 + eps2)^(3/2)
//   nbody_adjoint  dL/dE * (dE/dr_i, dE/dm_i), dE/dr_i = -m_i a_i,
//                  dE/dm_i = -sum_{j!=i} m_j / sqrt(|d_ij|^2 + eps2)
//   nbody_energy   E = -sum_{i<j} m_i m_j / sqrt(|d_ij|^2 + eps2)
//   nbody_fd       central differences of E in sampled coordinates
//
// The CTA has 256 threads.  Force kernels: a work-group of lws bodies (lws
// 32..256, a power of two) is cut into S j-segments (whole 512-body tiles),
// one chunk each, so that a run has enough chunks to balance the persistent
// CTAs; each chunk writes its per-body partial sums to the workspace and the
// last chunk of the work-group (a counter per work-group) adds the S
// partials in segment order and writes the result.  Within a chunk, thread
// t owns two bodies of the work-group (t % (lws/2) and that + lws/2,
// computed together in packed FP32x2 arithmetic) and the j-slice
// t / (lws/2).  Energy: thread t owns body t % lws and the j-slice t / lws.
// j-bodies are staged in shared memory 512 (force) or 256 (energy) at a time,
// tiles on an absolute grid.  Each thread sums the pair terms of one tile in
// FP32, then adds the tile sum to its running FP32 total (two-level
// summation); the slices of a body are added in slice order.
// The energy and finite-difference sums are FP32 pair terms accumulated in
// FP64, reduced in a fixed order, so results do not depend on scheduling.
#include <cuda_runtime.h>

#include <mutex>

#include "ecl_internal.h"
#include "f32x2.cuh"
#include "sched.cuh"

namespace ecl {
namespace {

constexpr int kBlock = 256;   // energy and finite-difference CTAs
constexpr int kTile = 256;
constexpr int kFBlock = 256;  // force CTA: 8 compute warps (+ the scheduler warp), 3 per SM
// j-bodies per staged force tile: a thread's j-slice of a tile is 2 lws/2
// bodies, so that the persistent form's per-tile call (see pair_tile_call)
// is paid once per 64 pairs at lws 64.  Measured at 65536 bodies against
// 256-body tiles: force 1.862 -> 1.812 ms, adjoint 1.975 -> 1.900 ms (1024:
// 1.790 / 1.965 ms).
constexpr int kFTile = 512;
constexpr int kFStage = kFTile / kFBlock;  // j-bodies each thread stages per tile
// Force shared memory: two duplicated tiles (x,x,y,y) and (z,z,m,m), double
// buffered (the slice partials reuse the first half after the tile loop),
// then each thread's running totals (a_x, a_y, a_z, potential) of its two
// bodies, [4][kFBlock] packed pairs.  The totals change once per tile; kept
// here rather than in registers they leave the pair loop its registers: with
// them in registers, the claim-loop form of the kernel (72 registers at 3 CTAs
// per SM) spent six register moves per pair iteration.
constexpr size_t kFSmem = 2 * 2 * kFTile * sizeof(float4) + 4 * kFBlock * sizeof(unsigned long long);

enum NMode : uint32_t { NB_STEP = 0, NB_ACC = 1, NB_ADJ = 2 };

struct NBodyParams {
    const float4 *pos;
    const float4 *vel;
    int64_t n;
    float dt, eps2;
    float4 *out_pos, *out_vel;  // NB_STEP
    float4 *out_acc;            // NB_ACC
    const float *grad_E;        // NB_ADJ: device scalar dL/dE
    float4 *out_grad;           // NB_ADJ
    float4 *part;               // [G][seg][lws] partial sums (seg > 1)
    unsigned *wgcnt;            // [G] segments finished per work-group
    uint32_t seg;               // j-segments (chunks) per work-group
    uint32_t lws;
};

// j-segments per work-group of the force kernels: enough chunks (about 8192,
// ~18 per resident CTA) that the last chunks, which set the end of the run,
// are short; at most 16 and at most one per staged tile.
__host__ __device__ inline uint32_t force_segments(uint64_t G, int64_t n)
{
    const int64_t ntiles = (n + kFTile - 1) / kFTile;
    uint64_t s = (8192 + G - 1) / (G ? G : 1);
    if (s > 16) s = 16;
    if ((int64_t)s > ntiles) s = (uint64_t)ntiles;
    return s < 1 ? 1u : (uint32_t)s;
}

// Stage j-tile `tile` (zero-mass padding beyond n).
__device__ __forceinline__ void stage_tile(float4 *sh, const float4 *pos, int64_t n, int64_t tile)
{
    const int64_t j = tile * kTile + threadIdx.x;
    sh[threadIdx.x] = (j < n) ? __ldg(pos + j) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// j-body `tile * kFTile + h * kFBlock + threadIdx.x` (zero-mass padding beyond n).
__device__ __forceinline__ float4 tile_body(const float4 *pos, int64_t n, int64_t tile, int h)
{
    const int64_t j = tile * kFTile + h * kFBlock + threadIdx.x;
    return (j < n) ? __ldg(pos + j) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Store one j-body duplicated for packed use: (x,x,y,y) and (z,z,m,m).
__device__ __forceinline__ void put_dup(float4 *shxy, float4 *shzm, const float4 &q, int h)
{
    shxy[h * kFBlock + threadIdx.x] = make_float4(q.x, q.x, q.y, q.y);
    shzm[h * kFBlock + threadIdx.x] = make_float4(q.z, q.z, q.w, q.w);
}

// The pair loop over one tile's j-slice for a thread's two bodies: sums of
// s d (and, for the adjoint, of m_j inv) over the slice, each body's sequence
//   d = r_j - r_i, r2 = dx dx + (dy dy + (dz dz + eps2)), inv = rsqrt(r2),
//   s = (m_j inv)(inv inv), sum += s d.
struct TileSums {
    f2 x, y, z, p;
};

template <uint32_t MODE, uint32_t SPAN>
__device__ __forceinline__ TileSums pair_tile(const ulonglong2 *qxy, const ulonglong2 *qzm, f2 X, f2 Y, f2 Z, f2 EPS)
{
    f2 TX = 0, TY = 0, TZ = 0, TP = 0;
#pragma unroll
    for (uint32_t k = 0; k < SPAN; ++k) {
        const ulonglong2 xy = qxy[k], zm = qzm[k];
        const f2 dx = sub2(xy.x, X), dy = sub2(xy.y, Y), dz = sub2(zm.x, Z);
        const f2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, EPS)));
        float r0, r1;
        upk(r2, r0, r1);
        const f2 inv = pk(rsqrtf(r0), rsqrtf(r1));
        const f2 mi = mul2(zm.y, inv);
        if (MODE == NB_ADJ) TP = add2(TP, mi);
        const f2 sc = mul2(mi, mul2(inv, inv));
        TX = fma2(sc, dx, TX);
        TY = fma2(sc, dy, TY);
        TZ = fma2(sc, dz, TZ);
    }
    return TileSums{TX, TY, TZ, TP};
}

// The same as a call, for the persistent form: a function of its own gets its
// own register allocation.  Inlined into the claim loop (72 registers at 3
// CTAs per SM, the driver's loop state live around it) the pair loop spent
// about four register moves per pair; called once per tile it spends none,
// while the caller saves a few values around each call.  The monolithic form
// keeps the inlined loop, its faster form.
template <uint32_t MODE, uint32_t SPAN>
__device__ __noinline__ TileSums pair_tile_call(const ulonglong2 *qxy, const ulonglong2 *qzm, f2 X, f2 Y, f2 Z,
                                                f2 EPS)
{
    return pair_tile<MODE, SPAN>(qxy, qzm, X, Y, Z, EPS);
}

// Force loop: thread t owns bodies (b, b + lws/2) of the work-group, b =
// t % (lws/2), and the j-slice t / (lws/2); both bodies advance together in
// packed FP32x2 arithmetic, each exactly as the scalar sequence
//   d = r_j - r_i, r2 = dx dx + (dy dy + (dz dz + eps2)), inv = rsqrt(r2),
//   s = (m_j inv)(inv inv), a += s d.
template <uint32_t MODE, bool CALL>
struct ForceBody {
    static constexpr uint32_t kThreads = kFBlock;
    using Params = NBodyParams;
    Params p;
    float4 *shxy, *shzm;  // [2][kFTile] duplicated j-bodies, double-buffered
    float4 *red;          // [2 * kFBlock] slice partials (aliases shxy)
    f2 *acc;              // [4][kFBlock] running totals of this thread's bodies
    uint32_t *flag;       // shared: this chunk completes its work-group

    static __host__ __device__ uint32_t nchunks(const Params &q, uint64_t, uint64_t len)
    {
        return (uint32_t)(len * q.seg);
    }

    // The body's output from its total a = (a_x, a_y, a_z, potential sum).
    __device__ __forceinline__ void finish(int64_t i, const float4 &pi, const float4 &a)
    {
        if (MODE == NB_ACC) {
            p.out_acc[i] = make_float4(a.x, a.y, a.z, 0.f);
        } else if (MODE == NB_STEP) {
            const float4 v = __ldg(p.vel + i);
            const float h = 0.5f * p.dt * p.dt;
            p.out_pos[i] = make_float4(pi.x + v.x * p.dt + a.x * h, pi.y + v.y * p.dt + a.y * h,
                                       pi.z + v.z * p.dt + a.z * h, pi.w);
            p.out_vel[i] = make_float4(v.x + a.x * p.dt, v.y + a.y * p.dt, v.z + a.z * p.dt, v.w);
        } else {
            // the self term j == i added m_i / sqrt(eps2) to the potential sum
            const float self = pi.w * rsqrtf(p.eps2);
            const float g = __ldg(p.grad_E);
            p.out_grad[i] = make_float4(-g * pi.w * a.x, -g * pi.w * a.y, -g * pi.w * a.z, -g * (a.w - self));
        }
    }

    // Tiles [ta, tb) of the j-bodies for this thread's two bodies (X, Y, Z)
    // and j-slice s of SPAN bodies per tile.  Tiles are double-buffered: the
    // next tile's loads are in flight while the current one is computed, one
    // barrier per tile.
    template <uint32_t SPAN>
    __device__ __forceinline__ void tiles(int64_t ta, int64_t tb, uint32_t s, f2 X, f2 Y, f2 Z, f2 EPS)
    {
        f2 *A = acc + threadIdx.x;
        A[0] = 0;
        A[kFBlock] = 0;
        A[2 * kFBlock] = 0;
        if (MODE == NB_ADJ) A[3 * kFBlock] = 0;
        body_sync(kFBlock);  // the previous chunk is done with both buffers
        if (ta < tb) {
#pragma unroll
            for (int h = 0; h < kFStage; ++h) put_dup(shxy, shzm, tile_body(p.pos, p.n, ta, h), h);
        }
        body_sync(kFBlock);
        for (int64_t tile = ta; tile < tb; ++tile) {
            const uint32_t cur = (uint32_t)(tile - ta) & 1u;
            const bool more = tile + 1 < tb;
            float4 nxt[kFStage];
#pragma unroll
            for (int h = 0; h < kFStage; ++h)
                nxt[h] = more ? tile_body(p.pos, p.n, tile + 1, h) : make_float4(0.f, 0.f, 0.f, 0.f);
            const ulonglong2 *qxy = reinterpret_cast<const ulonglong2 *>(shxy + cur * kFTile + s * SPAN);
            const ulonglong2 *qzm = reinterpret_cast<const ulonglong2 *>(shzm + cur * kFTile + s * SPAN);
            const TileSums T = CALL ? pair_tile_call<MODE, SPAN>(qxy, qzm, X, Y, Z, EPS)
                                    : pair_tile<MODE, SPAN>(qxy, qzm, X, Y, Z, EPS);
            const f2 TX = T.x, TY = T.y, TZ = T.z, TP = T.p;
            A[0] = add2(A[0], TX);
            A[kFBlock] = add2(A[kFBlock], TY);
            A[2 * kFBlock] = add2(A[2 * kFBlock], TZ);
            if (MODE == NB_ADJ) A[3 * kFBlock] = add2(A[3 * kFBlock], TP);
            // the other buffer was last read before the previous barrier
            if (more) {
#pragma unroll
                for (int h = 0; h < kFStage; ++h)
                    put_dup(shxy + (cur ^ 1u) * kFTile, shzm + (cur ^ 1u) * kFTile, nxt[h], h);
            }
            body_sync(kFBlock);
        }
    }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const uint32_t half = p.lws / 2;
        const uint32_t S = kFBlock / half;            // j-slices
        const uint32_t b = threadIdx.x % half, s = threadIdx.x / half;
        const uint64_t wg = off + t / p.seg;
        const uint32_t sg = t % p.seg;
        const int64_t i0 = (int64_t)wg * p.lws + b, i1 = i0 + half;
        const bool v0 = i0 < p.n, v1 = i1 < p.n;
        const float4 p0 = v0 ? __ldg(p.pos + i0) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 p1 = v1 ? __ldg(p.pos + i1) : make_float4(0.f, 0.f, 0.f, 0.f);
        const f2 X = pk(p0.x, p1.x), Y = pk(p0.y, p1.y), Z = pk(p0.z, p1.z);
        const f2 EPS = pk(p.eps2, p.eps2);
        const int64_t ntiles = (p.n + kFTile - 1) / kFTile;
        const int64_t ta = ntiles * sg / p.seg, tb = ntiles * (sg + 1) / p.seg;
        // the j-slice length kFTile / S equals kFStage * half: one instance
        // of the tile loop per lws, so that the pair loop's trip count is a
        // constant
        switch (half) {
        case 16: tiles<16 * kFStage>(ta, tb, s, X, Y, Z, EPS); break;
        case 32: tiles<32 * kFStage>(ta, tb, s, X, Y, Z, EPS); break;
        case 64: tiles<64 * kFStage>(ta, tb, s, X, Y, Z, EPS); break;
        default: tiles<128 * kFStage>(ta, tb, s, X, Y, Z, EPS); break;
        }
        // combine the slices of each body in slice order
        float ax0, ax1, ay0, ay1, az0, az1, pt0 = 0.f, pt1 = 0.f;
        const f2 *A = acc + threadIdx.x;
        upk(A[0], ax0, ax1);
        upk(A[kFBlock], ay0, ay1);
        upk(A[2 * kFBlock], az0, az1);
        if (MODE == NB_ADJ) upk(A[3 * kFBlock], pt0, pt1);
        body_sync(kFBlock);
        red[threadIdx.x] = make_float4(ax0, ay0, az0, pt0);
        red[kFBlock + threadIdx.x] = make_float4(ax1, ay1, az1, pt1);
        body_sync(kFBlock);
        // slice-0 thread handles body b, slice-1 thread body b + half
        const bool mine = s < 2 && (s == 0 ? v0 : v1);
        const uint32_t lb = s == 0 ? b : b + half;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mine) {
            const float4 *r = red + (s == 0 ? 0 : kFBlock);
            a = r[b];
            for (uint32_t q = 1; q < S; ++q) {
                const float4 e = r[q * half + b];
                a.x += e.x;
                a.y += e.y;
                a.z += e.z;
                a.w += e.w;
            }
        }
        if (p.seg == 1) {
            if (mine) finish(s == 0 ? i0 : i1, s == 0 ? p0 : p1, a);
            return;
        }
        // segment partial to the workspace; the work-group's last segment sums them
        float4 *wpart = p.part + (size_t)wg * p.seg * p.lws;
        if (mine) wpart[(size_t)sg * p.lws + lb] = a;
        __threadfence();
        body_sync(kFBlock);
        if (threadIdx.x == 0) *flag = (atomicAdd(p.wgcnt + wg, 1u) + 1 == p.seg) ? 1u : 0u;
        body_sync(kFBlock);
        if (*flag) {
            __threadfence();
            if (mine) {
                float4 tot = __ldcg(wpart + lb);
                for (uint32_t q = 1; q < p.seg; ++q) {
                    const float4 e = __ldcg(wpart + (size_t)q * p.lws + lb);
                    tot.x += e.x;
                    tot.y += e.y;
                    tot.z += e.z;
                    tot.w += e.w;
                }
                finish(s == 0 ? i0 : i1, s == 0 ? p0 : p1, tot);
            }
            if (threadIdx.x == 0) p.wgcnt[wg] = 0u;  // ready for the next run
        }
    }
};

// ---------------------------------------------------------------- energy
constexpr uint32_t kESeg = 8;  // chunks (j-segments) per work-group of the energy

struct EnergyParams {
    const float4 *pos;
    int64_t n;
    float eps2;
    double *out_E;
    double *partial;     // one per (work-group, segment)
    unsigned *counter;   // chunks finished in this run (reset by the last)
    uint64_t G;
    uint32_t lws;
};

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

struct EnergyBody {
    static constexpr uint32_t kThreads = kBlock;
    using Params = EnergyParams;
    Params p;
    float4 *sh;
    double *dsh;  // [kBlock / 32] warp sums, then [1] flag

    // Rows i < j make early work-groups far costlier than late ones; each
    // work-group's j-range is cut into kESeg tile-aligned segments so that no
    // single chunk dominates the run.
    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len)
    {
        return (uint32_t)(len * kESeg);
    }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const uint32_t lws = p.lws;
        const uint32_t S = kBlock / lws;
        const uint32_t b = threadIdx.x % lws, s = threadIdx.x / lws;
        const uint64_t wg = off + t / kESeg;
        const uint32_t seg = t % kESeg;
        const int64_t i0 = (int64_t)wg * lws;
        const int64_t i = i0 + b;
        const bool valid = i < p.n;
        const float4 pi = valid ? __ldg(p.pos + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t span = kTile / S;
        double e = 0.0;
        const int64_t ntiles = (p.n + kTile - 1) / kTile;
        // rows i < j only: tiles from the one holding this work-group onwards, this segment's share
        const int64_t tfirst = i0 / kTile, nt = ntiles - tfirst;
        const int64_t ta = tfirst + nt * seg / kESeg, tb = tfirst + nt * (seg + 1) / kESeg;
        for (int64_t tile = ta; tile < tb; ++tile) {
            body_sync(kBlock);
            stage_tile(sh, p.pos, p.n, tile);
            body_sync(kBlock);
            float tp = 0.f;
            const int64_t j0 = tile * kTile + s * span;
            const float4 *q = sh + s * span;
            if (j0 + (int64_t)span - 1 <= i) {
                // whole slice at or before i: contributes nothing
            } else if (j0 > i) {
#pragma unroll 8
                for (uint32_t k = 0; k < span; ++k) {
                    const float4 pj = q[k];
                    const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, p.eps2)));
                    tp = fmaf(pj.w, rsqrtf(r2), tp);
                }
            } else {
                for (uint32_t k = 0; k < span; ++k) {
                    const float4 pj = q[k];
                    const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, p.eps2)));
                    const float m = (j0 + (int64_t)k > i) ? pj.w : 0.f;
                    tp = fmaf(m, rsqrtf(r2), tp);
                }
            }
            e += (double)tp;
        }
        // this thread's share of -m_i sum_{j>i} m_j phi_ij, reduced in a fixed order
        double v = valid ? -(double)pi.w * e : 0.0;
        v = warp_sum_d(v);
        body_sync(kBlock);
        if ((threadIdx.x & 31) == 0) dsh[threadIdx.x / 32] = v;
        body_sync(kBlock);
        if (threadIdx.x == 0) {
            double w = 0.0;
            for (int q = 0; q < kBlock / 32; ++q) w += dsh[q];
            p.partial[wg * kESeg + seg] = w;
            __threadfence();
            const unsigned before = atomicAdd(p.counter, 1u);
            dsh[0] = (before + 1 == (unsigned)(p.G * kESeg)) ? 1.0 : 0.0;
        }
        body_sync(kBlock);
        if (dsh[0] != 0.0) {  // last chunk of the run: sum the partials in order
            __threadfence();
            double acc = 0.0;
            const uint64_t np = p.G * kESeg;
            const uint64_t per = (np + kBlock - 1) / kBlock;
            const uint64_t a = threadIdx.x * per;
            const uint64_t z = min(np, a + per);
            for (uint64_t w = a; w < z; ++w) acc += *((volatile double *)p.partial + w);
            body_sync(kBlock);
            __shared__ double tree[kBlock];
            tree[threadIdx.x] = acc;
            body_sync(kBlock);
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int q = 0; q < kBlock; ++q) tot += tree[q];
                *p.out_E = tot;
                *p.counter = 0u;
            }
        }
        body_sync(kBlock);
    }
};

// ---------------------------------------------------------------- finite differences
// j-segments per finite-difference sample: enough chunks (about 4096) that
// the samples spread over every SM, each segment at least one 256-body span.
constexpr uint32_t kFDSegMax = 16;

__host__ __device__ inline uint32_t fd_segments(int64_t count, int64_t n)
{
    uint64_t s = (4096 + (uint64_t)count - 1) / (uint64_t)(count > 0 ? count : 1);
    if (s > kFDSegMax) s = kFDSegMax;
    const int64_t spans = (n + kBlock - 1) / kBlock;
    if ((int64_t)s > spans) s = (uint64_t)spans;
    return s < 1 ? 1u : (uint32_t)s;
}

struct FDParams {
    const float4 *pos;
    int64_t n;
    float eps2, h;
    const int *body, *comp;
    int64_t count;
    double *out;
    double *part;   // [count][seg] FP64 partial sums (seg > 1)
    unsigned *cnt;  // [count] segments finished per sample
    uint32_t seg;
};

struct FDBody {
    static constexpr uint32_t kThreads = kBlock;
    using Params = FDParams;
    Params p;
    double *dsh;  // [kBlock / 32]

    static __host__ __device__ uint32_t nchunks(const Params &q, uint64_t, uint64_t len)
    {
        return (uint32_t)(len * q.seg);
    }

    // chunk = segment sg of one sample: -m_i * (row(q+) - row(q-)) / (x+ - x-),
    // row(q) = sum_{j != i} m_j / sqrt(|q - r_j|^2 + eps2), summed as the FP64
    // sum of the FP32 term differences m_j phi(q+) - m_j phi(q-) (the two
    // terms are within a factor 2 of each other, so each difference is exact
    // in FP32); the segments' sums are added in segment order by the last.
    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const int64_t smp = (int64_t)(off + t / p.seg);
        const uint32_t sg = t % p.seg;
        if (smp >= p.count) return;
        const int64_t i = p.body[smp];
        const int c = p.comp[smp];
        if (i < 0 || i >= p.n || c < 0 || c > 2) {  // invalid sample: NaN, no access
            if (threadIdx.x == 0 && sg == 0) p.out[smp] = __longlong_as_double(0x7ff8000000000000ll);
            return;
        }
        const float4 pi = __ldg(p.pos + i);
        const float xc = c == 0 ? pi.x : (c == 1 ? pi.y : pi.z);
        const float xp = xc + p.h, xm = xc - p.h;
        float4 qp = pi, qm = pi;
        if (c == 0) { qp.x = xp; qm.x = xm; }
        else if (c == 1) { qp.y = xp; qm.y = xm; }
        else { qp.z = xp; qm.z = xm; }
        const int64_t j0 = p.n * (int64_t)sg / p.seg, j1 = p.n * (int64_t)(sg + 1) / p.seg;
        double acc = 0.0;
        for (int64_t j = j0 + threadIdx.x; j < j1; j += kBlock) {
            if (j == i) continue;
            const float4 pj = __ldg(p.pos + j);
            float dx = qp.x - pj.x, dy = qp.y - pj.y, dz = qp.z - pj.z;
            const float fp = pj.w * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, p.eps2))));
            dx = qm.x - pj.x;
            dy = qm.y - pj.y;
            dz = qm.z - pj.z;
            const float fm = pj.w * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, p.eps2))));
            acc += (double)(fp - fm);
        }
        acc = warp_sum_d(acc);
        body_sync(kBlock);
        if ((threadIdx.x & 31) == 0) dsh[threadIdx.x / 32] = acc;
        body_sync(kBlock);
        if (threadIdx.x == 0) {
            double w = 0.0;
            for (int q = 0; q < kBlock / 32; ++q) w += dsh[q];
            const double scale = -(double)pi.w / ((double)xp - (double)xm);
            if (p.seg == 1) {
                p.out[smp] = scale * w;
            } else {
                double *part = p.part + (size_t)smp * p.seg;
                part[sg] = w;
                __threadfence();
                if (atomicAdd(p.cnt + smp, 1u) + 1 == p.seg) {
                    __threadfence();
                    double tot = 0.0;
                    for (uint32_t q = 0; q < p.seg; ++q) tot += *((volatile double *)part + q);
                    p.out[smp] = scale * tot;
                    p.cnt[smp] = 0u;  // ready for the next run
                }
            }
        }
        body_sync(kBlock);
    }
};

// ---------------------------------------------------------------- kernels
// One instance per launch form (FORM: DRIVE_MONO or DRIVE_QUEUE), each with
// a single copy of the force body.
template <uint32_t MODE, int FORM>
__global__ void __launch_bounds__(kFBlock + 32, 3) k_nbody_force(NBodyParams prm, SchedArgs s)
{
    extern __shared__ __align__(16) float4 fsm[];
    __shared__ uint32_t flag;
    ForceBody<MODE, FORM == DRIVE_QUEUE> b;
    b.p = prm;
    b.shxy = fsm;
    b.shzm = fsm + 2 * kFTile;
    b.red = fsm;
    b.acc = reinterpret_cast<f2 *>(fsm + 4 * kFTile);
    b.flag = &flag;
    drive_ws<ForceBody<MODE, FORM == DRIVE_QUEUE>, FORM>(s, b);
}

// One instance per launch form (DRIVE_MONO, DRIVE_QUEUE), each with a single
// inlined copy of the body.
template <int FORM>
__global__ void __launch_bounds__(kBlock + 32) k_nbody_energy(EnergyParams prm, SchedArgs s)
{
    __shared__ float4 sh[kTile];
    __shared__ double dsh[kBlock / 32];
    EnergyBody b;
    b.p = prm;
    b.sh = sh;
    b.dsh = dsh;
    drive_ws<EnergyBody, FORM>(s, b);
}

__global__ void __launch_bounds__(kBlock + 32) k_nbody_fd(FDParams prm, SchedArgs s)
{
    __shared__ double dsh[kBlock / 32];
    FDBody b;
    b.p = prm;
    b.dsh = dsh;
    drive_ws(s, b);
}

int occ(const void *fn, int block = kBlock + 32, size_t smem = 0)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// Force kernels take kFSmem bytes of dynamic shared memory, above the default
// limit: the opt-in is a per-function attribute of the current device, set
// before every occupancy query and launch (a cheap driver call).
template <uint32_t MODE>
bool force_smem_ok()
{
    static std::atomic<unsigned long long> queue_done{0}, mono_done{0};
    return smem_limit_once((const void *)k_nbody_force<MODE, DRIVE_QUEUE>, (int)kFSmem, queue_done) &&
           smem_limit_once((const void *)k_nbody_force<MODE, DRIVE_MONO>, (int)kFSmem, mono_done);
}

template <uint32_t MODE>
int occ_force()
{
    if (!force_smem_ok<MODE>()) {
        cudaGetLastError();
        return 0;
    }
    return occ((const void *)k_nbody_force<MODE, DRIVE_QUEUE>, kFBlock + 32, kFSmem);
}

template <uint32_t MODE>
ecl_status launch_force(const NBodyParams &p, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    if (!force_smem_ok<MODE>()) {
        err = "cannot enable the force kernel's shared memory";
        cudaGetLastError();
        return ECL_ERR_CUDA;
    }
    if (s.mode == MODE_MONO)
        k_nbody_force<MODE, DRIVE_MONO><<<c.grid, kFBlock + 32, kFSmem, c.stream>>>(p, s);
    else
        k_nbody_force<MODE, DRIVE_QUEUE><<<c.grid, kFBlock + 32, kFSmem, c.stream>>>(p, s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

ecl_status launched(std::string &err)
{
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

bool lws_ok(uint32_t lws) { return lws == 32 || lws == 64 || lws == 128 || lws == 256; }

ecl_status check_bodies(const KArgs &a, int pos_arg, int n_arg, uint64_t gws, uint32_t lws, std::string &err)
{
    const int64_t n = a.i32(n_arg);
    if (n <= 0) {
        err = "bodies must be positive";
        return ECL_ERR_ARG;
    }
    if (!lws_ok(lws)) {
        err = "lws must be 32, 64, 128 or 256";
        return ECL_ERR_SIZE;
    }
    if (gws < (uint64_t)n) {
        err = "the NDRange (one body per work-item) does not cover the bodies";
        return ECL_ERR_SIZE;
    }
    if (a.bytes[pos_arg] < (uint64_t)n * 16 || (uintptr_t)a.ptr[pos_arg] % 16) {
        err = "positions must be 16-byte aligned float4[n]";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

bool out4_ok(const KArgs &a, int i, int64_t n) { return a.bytes[i] >= (uint64_t)n * 16 && (uintptr_t)a.ptr[i] % 16 == 0; }

uint64_t grain1(const KArgs &, uint64_t, uint32_t) { return 1; }

// Force kernels: S chunks per work-group (bodies at argument n_arg).
template <int n_arg>
uint32_t nchunks_force(const KArgs &a, uint64_t gws, uint32_t lws, uint64_t, uint64_t len)
{
    return (uint32_t)(len * force_segments(gws / lws, a.i32(n_arg)));
}

// Segment count and workspace (per-segment partials + per-work-group
// counters) of a force launch.
bool force_ws(NBodyParams &p, const LaunchCtx &c, const void *owner, std::string &err)
{
    const uint64_t G = c.gws / c.lws;
    p.seg = force_segments(G, p.n);
    p.part = nullptr;
    p.wgcnt = nullptr;
    if (p.seg == 1) return true;
    const size_t cnt_bytes = (G * sizeof(unsigned) + 255) / 256 * 256;
    char *ws = (char *)workspace_get(c.ws, cnt_bytes + (size_t)G * p.seg * c.lws * sizeof(float4), err, owner,
                                     c.stream);
    if (!ws) return false;
    p.wgcnt = (unsigned *)ws;
    p.part = (float4 *)(ws + cnt_bytes);
    return true;
}

uint32_t nchunks_energy(const KArgs &, uint64_t, uint32_t, uint64_t, uint64_t len) { return (uint32_t)(len * kESeg); }

// ---- nbody (Listing 2 order): in_pos, in_vel, bodies, del_t, esp_sqr, out_pos, out_vel
ecl_status v_step(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    ecl_status st = check_bodies(a, 0, 2, gws, lws, err);
    if (st != ECL_OK) return st;
    const int64_t n = a.i32(2);
    if (!out4_ok(a, 1, n) || !out4_ok(a, 5, n) || !out4_ok(a, 6, n)) {
        err = "velocity and output buffers must be 16-byte aligned float4[n]";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

ecl_status l_step(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    NBodyParams p{};
    p.pos = a.buf<const float4>(0);
    p.vel = a.buf<const float4>(1);
    p.n = a.i32(2);
    p.dt = a.f32(3);
    p.eps2 = a.f32(4);
    p.out_pos = a.buf<float4>(5);
    p.out_vel = a.buf<float4>(6);
    p.lws = c.lws;
    if (!force_ws(p, c, (const void *)k_nbody_force<NB_STEP, DRIVE_QUEUE>, err)) return ECL_ERR_CUDA;
    return launch_force<NB_STEP>(p, s, c, err);
}

int o_step() { return occ_force<NB_STEP>(); }

// ---- nbody_acc: in_pos, bodies, esp_sqr, out_acc
ecl_status v_acc(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    ecl_status st = check_bodies(a, 0, 1, gws, lws, err);
    if (st != ECL_OK) return st;
    if (!out4_ok(a, 3, a.i32(1))) {
        err = "out_acc must be a 16-byte aligned float4[n]";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

ecl_status l_acc(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    NBodyParams p{};
    p.pos = a.buf<const float4>(0);
    p.n = a.i32(1);
    p.eps2 = a.f32(2);
    p.out_acc = a.buf<float4>(3);
    p.lws = c.lws;
    if (!force_ws(p, c, (const void *)k_nbody_force<NB_ACC, DRIVE_QUEUE>, err)) return ECL_ERR_CUDA;
    return launch_force<NB_ACC>(p, s, c, err);
}

int o_acc() { return occ_force<NB_ACC>(); }

// ---- nbody_adjoint: in_pos, bodies, esp_sqr, grad_E, out_grad
ecl_status v_adj(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    ecl_status st = check_bodies(a, 0, 1, gws, lws, err);
    if (st != ECL_OK) return st;
    if (a.bytes[3] < 4) {
        err = "grad_E must hold one float";
        return ECL_ERR_BUFFER;
    }
    if (!out4_ok(a, 4, a.i32(1))) {
        err = "out_grad must be a 16-byte aligned float4[n]";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

ecl_status l_adj(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    NBodyParams p{};
    p.pos = a.buf<const float4>(0);
    p.n = a.i32(1);
    p.eps2 = a.f32(2);
    p.grad_E = a.buf<const float>(3);
    p.out_grad = a.buf<float4>(4);
    p.lws = c.lws;
    if (!force_ws(p, c, (const void *)k_nbody_force<NB_ADJ, DRIVE_QUEUE>, err)) return ECL_ERR_CUDA;
    return launch_force<NB_ADJ>(p, s, c, err);
}

int o_adj() { return occ_force<NB_ADJ>(); }

// ---- nbody_energy: in_pos, bodies, esp_sqr, out_energy (double[1]); workspace: G partials + counter
ecl_status v_energy(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    ecl_status st = check_bodies(a, 0, 1, gws, lws, err);
    if (st != ECL_OK) return st;
    if (a.bytes[3] < 8 || (uintptr_t)a.ptr[3] % 8) {
        err = "out_energy must be an aligned double[1]";
        return ECL_ERR_BUFFER;
    }
    if (gws / lws > 0xffffffffull / kESeg) {
        err = "too many work-groups";
        return ECL_ERR_SIZE;
    }
    return ECL_OK;
}

ecl_status l_energy(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    const uint64_t G = c.gws / c.lws;
    char *ws = (char *)workspace_get(c.ws, 256 + G * kESeg * sizeof(double), err, (const void *)k_nbody_energy<DRIVE_QUEUE>, c.stream);
    if (!ws) return ECL_ERR_CUDA;
    EnergyParams p{};
    p.pos = a.buf<const float4>(0);
    p.n = a.i32(1);
    p.eps2 = a.f32(2);
    p.out_E = a.buf<double>(3);
    p.counter = (unsigned *)ws;
    p.partial = (double *)(ws + 256);
    p.G = G;
    p.lws = c.lws;
    if (s.mode == MODE_MONO)
        k_nbody_energy<DRIVE_MONO><<<c.grid, kBlock + 32, 0, c.stream>>>(p, s);
    else
        k_nbody_energy<DRIVE_QUEUE><<<c.grid, kBlock + 32, 0, c.stream>>>(p, s);
    return launched(err);
}

int o_energy() { return occ((const void *)k_nbody_energy<DRIVE_QUEUE>); }

// ---- nbody_fd: in_pos, bodies, esp_sqr, h, body[], comp[], count, out[] (double)
ecl_status v_fd(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    const int64_t n = a.i32(1), cnt = a.i32(6);
    if (n <= 0 || cnt <= 0) {
        err = "bodies and sample count must be positive";
        return ECL_ERR_ARG;
    }
    if (lws != 1 || gws < (uint64_t)cnt) {
        err = "one work-group (lws 1) per sample";
        return ECL_ERR_SIZE;
    }
    if (a.bytes[0] < (uint64_t)n * 16 || (uintptr_t)a.ptr[0] % 16) {
        err = "positions must be 16-byte aligned float4[n]";
        return ECL_ERR_BUFFER;
    }
    if (a.bytes[4] < (uint64_t)cnt * 4 || a.bytes[5] < (uint64_t)cnt * 4 || a.bytes[7] < (uint64_t)cnt * 8) {
        err = "sample buffers smaller than the sample count";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

ecl_status l_fd(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    FDParams p{};
    p.pos = a.buf<const float4>(0);
    p.n = a.i32(1);
    p.eps2 = a.f32(2);
    p.h = a.f32(3);
    p.body = a.buf<const int>(4);
    p.comp = a.buf<const int>(5);
    p.count = a.i32(6);
    p.out = a.buf<double>(7);
    p.seg = fd_segments(p.count, p.n);
    if (p.seg > 1) {
        const size_t cnt_bytes = ((size_t)p.count * sizeof(unsigned) + 255) / 256 * 256;
        char *ws = (char *)workspace_get(c.ws, cnt_bytes + (size_t)p.count * p.seg * sizeof(double), err,
                                         (const void *)k_nbody_fd, c.stream);
        if (!ws) return ECL_ERR_CUDA;
        p.cnt = (unsigned *)ws;
        p.part = (double *)(ws + cnt_bytes);
    }
    k_nbody_fd<<<c.grid, kBlock + 32, 0, c.stream>>>(p, s);
    return launched(err);
}

uint32_t nchunks_fd(const KArgs &a, uint64_t, uint32_t, uint64_t, uint64_t len)
{
    return (uint32_t)(len * fd_segments(a.i32(6), a.i32(1)));
}

int o_fd() { return occ((const void *)k_nbody_fd); }

}  // namespace

extern const KernelDesc kNBody = {
    "nbody", 7,
    {{"in_pos", A_BUF_IN}, {"in_vel", A_BUF_IN}, {"bodies", A_I32}, {"del_t", A_F32}, {"esp_sqr", A_F32},
     {"out_pos", A_BUF_OUT}, {"out_vel", A_BUF_OUT}},
    1, 1, kFBlock + 32, 0, v_step, grain1, nchunks_force<2>, o_step, l_step,
};

extern const KernelDesc kNBodyAcc = {
    "nbody_acc", 4,
    {{"in_pos", A_BUF_IN}, {"bodies", A_I32}, {"esp_sqr", A_F32}, {"out_acc", A_BUF_OUT}},
    1, 1, kFBlock + 32, 0, v_acc, grain1, nchunks_force<1>, o_acc, l_acc,
};

extern const KernelDesc kNBodyAdjoint = {
    "nbody_adjoint", 5,
    {{"in_pos", A_BUF_IN}, {"bodies", A_I32}, {"esp_sqr", A_F32}, {"grad_E", A_BUF_IN},
     {"out_grad", A_BUF_OUT}},
    1, 1, kFBlock + 32, 0, v_adj, grain1, nchunks_force<1>, o_adj, l_adj,
};

extern const KernelDesc kNBodyEnergy = {
    "nbody_energy", 4,
    {{"in_pos", A_BUF_IN}, {"bodies", A_I32}, {"esp_sqr", A_F32}, {"out_energy", A_BUF_OUT}},
    1, 0, kBlock + 32, 0, v_energy, grain1, nchunks_energy, o_energy, l_energy,
};

extern const KernelDesc kNBodyFD = {
    "nbody_fd", 8,
    {{"in_pos", A_BUF_IN}, {"bodies", A_I32}, {"esp_sqr", A_F32}, {"h", A_F32}, {"body", A_BUF_IN},
     {"comp", A_BUF_IN}, {"count", A_I32}, {"out", A_BUF_OUT}},
    1, 1, kBlock + 32, 0, v_fd, grain1, nchunks_fd, o_fd, l_fd,
};

// ---------------------------------------------------------------- energy without allocation
// Scratch of ecl_nbody_energy_noalloc: a 256-byte header (the chunk counter)
// followed by one FP64 partial per (work-group, segment).  It lives in every
// GPU that loads this library, for the life of the process.
namespace {
constexpr uint64_t kNoAllocPartials = 1u << 16;  // 512 KiB of FP64 partials
constexpr uint32_t kNoAllocLws = 64;
constexpr int kNoAllocMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_energy_scratch[256 + kNoAllocPartials * sizeof(double)];

namespace {
std::mutex g_scratch_mu;
void *g_scratch_ptr[kNoAllocMaxDevices];
}  // namespace

}  // namespace ecl

extern "C" ecl_status ecl_nbody_energy_noalloc(const void *pos4, int32_t n, float eps2, double *out_energy,
                                               void *cuda_stream)
{
    using namespace ecl;
    if (!pos4 || !out_energy || n <= 0 || (uintptr_t)pos4 % 16 || (uintptr_t)out_energy % 8) return ECL_ERR_ARG;
    const uint64_t G = ((uint64_t)n + kNoAllocLws - 1) / kNoAllocLws;
    if (G * kESeg > kNoAllocPartials) return ECL_ERR_SIZE;  // more than 524288 bodies
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        return ECL_ERR_CUDA;
    }
    void *scratch = nullptr;
    {
        // once per device, with that device current: the scratch array's device address
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_energy_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return ECL_ERR_CUDA;
            }
            g_scratch_ptr[dev] = ptr;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the chunk counter must start at zero (a previous call that failed may have left it set)
    if (cudaMemsetAsync(scratch, 0, 256, st) != cudaSuccess) {
        cudaGetLastError();
        return ECL_ERR_CUDA;
    }
    EnergyParams p{};
    p.pos = (const float4 *)pos4;
    p.n = n;
    p.eps2 = eps2;
    p.out_E = out_energy;
    p.counter = (unsigned *)scratch;
    p.partial = (double *)((char *)scratch + 256);
    p.G = G;
    p.lws = kNoAllocLws;
    SchedArgs s{};  // a monolithic launch: no package queue, so no engine memory either
    s.mode = MODE_MONO;
    s.G = G;
    s.grain = 1;
    s.units = G;
    s.mono_nchunks = (uint32_t)(G * kESeg);
    k_nbody_energy<DRIVE_MONO><<<(unsigned)(G * kESeg), kBlock + 32, 0, st>>>(p, s);
    if (cudaGetLastError() != cudaSuccess) return ECL_ERR_CUDA;
    return ECL_OK;
}

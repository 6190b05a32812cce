// Binomial option pricing (Listing 1 workload: one work-group per option
// lattice, out pattern 1:lws) for a batch of European calls of uneven depth
// N = 1..2048 on a Cox-Ross-Rubinstein lattice, FP32.
//
// One warp (the work-group, lws 32) prices one option.  Level t of the
// lattice holds nodes j = 0..t; node j lives in lane j / R, register slot
// j % R, where the width R steps down 64, 56, 48, ..., 2, 1 as the lattice
// shrinks; a lattice starts at the narrowest width that holds its leaves
// (each width's code exists once and is entered by index).  A backward step
// needs node j+1: in the same lane except for the last slot, which one
// shuffle per level brings from the next lane.  When the live nodes fit in
// the next width the warp repacks its registers through a padded shared
// buffer, so ~90% of the computed slots stay live.
//
// Arithmetic (exact in real numbers, arranged for FP32):
//   p = 1/2 + q,  q = (expm1(r dt) - 2 sinh^2(a/2)) / (2 sinh a),  a = sigma sqrt(dt)
// is the CRR probability (e^{r dt} - d)/(u - d) written so that the large
// part 1/2 is exact and only the small q carries rounding.  With v = 2q the
// level is V'_j = disc (p V_{j+1} + (1 - p) V_j); divided by disc (1 - p)
// per level it becomes
//   C'_j = C_j + rho C_{j+1},  rho = p / (1 - p) = 1 + eta,  eta = 2v / (1 - v),
// and one node update is  C_j <- fma(eta, C_{j+1}, C_{j+1} + C_j)  (add,
// FMA): the coefficient 1 is exact and only the small eta carries rounding,
// so the lattice is that of a probability within ~1e-9 of p.  The root is
// the price times (2 + eta)^N / disc^N; the factor is removed at the end
// from its logarithm in pairs of FP32 values.  The largest node grows by at
// most 2 + eta per level, so every K levels (K = 64, fewer when eta > 0:
// K log2(2 + eta) <= 64) all nodes are multiplied by 2^-E, E = the ceiling
// of K log2(2 + eta) (exact); leaves stay below ~1e16 (S = 100,
// sigma = 0.5, T = 2, N = 2048), so the lattice stays below ~2e35, inside
// the FP32 range.
// In-the-money calls (S > K) are priced through the put on the same lattice
// and put-call parity, which holds exactly on a CRR lattice:
//   C = P + S - K e^{-rT},  dC/dS = dP/dS + 1,  dC/dsigma = dP/dsigma.
// The put lattice of a deep in-the-money call holds small values, while the
// call lattice would carry two large vega terms (leaf and dq/dsigma parts)
// that cancel, losing several digits in FP32.
// Greeks are the exact derivatives of this discrete price.  In terms of the
// lattice scaled by 2 / disc per level, B'_j = (1 + v) B_{j+1} + (1 - v) B_j
// (B = (1 - v)^k C after k levels), forward mode through one level gives
//   delta tree: the same recursion, leaves u^j d^(N-j) for in-the-money leaves;
//   vega tree:  dB_j <- (dB_{j+1} + dB_j) + 2q (dB_{j+1} - dB_j) + 2q' (B_{j+1} - B_j),
//               q' = dq/dsigma = sqrt(dt) (-1/2 - q coth a),
//               leaves S_T (2j - N) sqrt(dt) for in-the-money leaves.
// The level operator L = (1 + 2q) shift + (1 - 2q) identity and the
// difference operator (shift - identity) are both shift-invariant, so they
// commute, and the N coefficient terms of the vega tree add up to
//   N 2q' (B_1 - B_0)   (B_1, B_0: the two nodes of level 1, same scaling).
// So delta and the leaf part of vega are the same recursion applied to the
// leaf derivatives, linear functionals of the leaves.  One reverse (adjoint)
// pass gives the weights A of every node of level N - 1 in the root
// (A = 1 at the root, A'_j = A_j + rho A_{j-1} outwards on the C lattice),
// and both become dot products of A with the leaf derivatives pushed back
// one level; with B_1 - B_0 kept from the price pass,
//   vega = <A, vega leaves'> + N 2q' (B_1 - B_0).
// Stored in reverse node order the adjoint recursion is the backward level
// itself, so the price pass and the adjoint pass run on one copy of the
// level code.
// Only the out-of-the-money side is priced, so its nonzero leaves form one
// contiguous run: j < b for the put, j > N - b for the call.  The call's
// lattice is stored reflected (node j at index N - j), where its level is
// the same operator with v = -2q in place of 2q (and eta from that v), so
// both sides have their nonzero leaves at indices 0 .. b - 1.  Nodes at index >= b stay exactly
// zero while the lattice is wider than b, so the backward induction runs at
// the width that holds min(t + 1, b) nodes of level t, and the adjoint pass
// stops widening once it holds the b weights the dot products use.  For the
// near-the-money options of the workload b is about N / 2: a quarter of the
// node updates of each pass are exact zeros that are never computed.
// The adjoint in closed form: the level operator B' = 2p shift(B) + 2(1-p) B
// applied N times gives every leaf j the weight 2^N C(N,j) p^j (1-p)^(N-j)
// in the root (each path from leaf j up to the root takes j up-steps and
// N - j down-steps), so the adjoint pass's weights, pushed back to the
// leaves, are the binomial probabilities.  Delta and the leaf part of vega
// are then sums over the b nonzero leaves, O(b) per option instead of the
// adjoint lattice's O(N b): ln C(N,j) + j ln p + (N-j) ln(1-p) in pairs of
// FP32 values (a log-factorial table generated at build time, the
// per-option logs from their series, in FP64 on coarse lattices), then one
// expf.  "binomial_full" keeps the adjoint lattice
// pass, the reference form this evaluation is tested against.
// In FP32 emulation of this arithmetic against the FP64 oracle,
// options of depth 1900..2048 show ~1.7e-6 relative error in the price,
// ~0.9e-6 in delta and ~1.8e-6 in vega.
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
    float eta;     // level coefficient: C'_i = C_i + (1 + eta) C_{i+1} (storage order)
    float f;       // 2^-E, one rescale
    int K;         // levels between rescales
    int E;
    int rescale;   // levels since the last rescale
    int shift;     // power of two still to remove from the result
};

constexpr int kRescale = 64;  // at most 64 levels (growth at most 2^64) between rescales

// ln k! for k = 0..2048 as (hi, lo) FP32 pairs, hi + lo = the double value
// (generated by build.py from math.lgamma).
__device__ const float2 g_lfact[] = {
#include "lfact_table.inc"
};

// Pairs of FP32 values (hi, lo) with about 48 significant bits: TwoSum and
// the FMA-based TwoProd (Dekker, Knuth), exact error-free transformations in
// round-to-nearest.
__device__ __forceinline__ float2 two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return make_float2(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    const float2 s = two_sum(a.x, b.x);
    const float lo = s.y + (a.y + b.y);
    const float hi = s.x + lo;
    return make_float2(hi, lo - (hi - s.x));
}

__device__ __forceinline__ float2 df_split(double x)
{
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}

// j * v for a small integer j (exact in FP32) and a pair v.
__device__ __forceinline__ float2 df_scale(float j, float2 v)
{
    const float p = j * v.x;
    const float e = fmaf(j, v.x, -p);
    const float lo = fmaf(j, v.y, e);
    const float hi = p + lo;
    return make_float2(hi, lo - (hi - p));
}

// ln(1 + x) as a pair for |x| <= 1/4 from the Mercator series
//   ln(1 + x) = x - x^2/2 + x^3 (1/3 - x/4 + x^2/5 - ...):
// x - x^2/2 carried exactly (TwoProd of x*x), the cubic tail (below
// 0.03 |x|) in FP32 with 16 terms, the rest below |x|^19 / 19.
__device__ __forceinline__ float2 df_log1p(float x)
{
    float t = 1.0f / 18.0f;
#pragma unroll
    for (int k = 17; k >= 3; --k) t = fmaf(t, -x, 1.0f / (float)k);
    const float x2 = x * x;
    const float x2e = fmaf(x, x, -x2);
    const float tail = x2 * x * t;
    const float2 s = two_sum(x, -0.5f * x2);
    const float lo = s.y + fmaf(-0.5f, x2e, tail);
    const float hi = s.x + lo;
    return make_float2(hi, lo - (hi - s.x));
}

// Lane widths (nodes per lane) the warp steps through as the lattice shrinks.
// Going from width R to the next width R' happens when the live nodes fit in
// 32 R'.  Every width is a fully unrolled level loop plus a repack, so the
// list trades computed-but-dead slots against code size: measured on the
// 2^20-option batch (price + greeks), finer lists (33 widths: ~96% live
// slots) ran up to 2x slower on instruction fetch, and this list (~88%
// live; the banded lattice uses it from 40 down) was the fastest of eight
// candidates; with the banded lattice at two instructions per node, adding
// 6, or 14, 10 and 6, or dropping 28 measured 1.5-2% slower.
constexpr int kWidths[] = {64, 56, 48, 40, 32, 28, 24, 20, 16, 12, 8, 4, 2, 1};
constexpr int kNWidths = sizeof(kWidths) / sizeof(kWidths[0]);
__host__ __device__ constexpr int width_at(int i) { return i < kNWidths ? kWidths[i] : 0; }
constexpr int kMaxR = 64;
constexpr int kMaxSteps = kWarp * kMaxR;               // deepest lattice: 2048 steps
// The banded lattice starts at width 40: its band, the out-of-the-money
// side's nonzero leaves, holds at most N/2 + 1 <= 1025 nodes (for sigma,
// T >= 0), so it never needs the three widest widths, which only the full
// lattice (up to 2049 leaves) runs.  Its level code and its registers stop
// at 40 slots per lane.
constexpr int kW0Band = 3;
static_assert(width_at(kW0Band) == 40, "banded lattice starts at width 40");
constexpr int kShNodes = kMaxSteps + 1 + kMaxSteps / 32 + 32;  // leaves 0..N with padding

// Resident one-warp CTAs per SM the register budget is set for.  A node
// update is an add and an FMA that depends on it, so a warp waits on its own
// FP32 latency unless the scheduler has other warps: the banded lattice (at
// most 40 slots a lane, inlined) runs at 16 per SM (128 registers, no
// spills).  Measured on the 2^20-option batch with greeks: 8 per SM 63.8 ms,
// 10 61.3, 12 51.4, 16 49.4, 20 (96 registers, spills) 51.9.  The full
// lattice (64 slots a lane) keeps 8 (255 registers).
constexpr int kMinCtas = 16;
constexpr int kMinCtasFull = 8;

__device__ __forceinline__ int shidx(int j) { return j + (j >> 5); }  // avoids bank conflicts

// One level of the recursion C'_k = C_k + (1 + eta) C_{k+1} on the first R
// slots of every lane (lane l holds nodes l*R .. l*R + R - 1), two FP32
// instructions per node.  The last lane's last slot has zero above it: the
// node above the top of the backward induction (a dead slot), above the
// nonzero band of a lattice wider than the band (which keeps the nodes
// there at zero), and the not-yet-reached node before node 0 in the adjoint
// (stored reversed).  With a zero neighbour the update leaves a node as it
// is (fma(eta, 0, 0 + x) = x exactly), so that lane skips it.
template <int R>
__device__ __forceinline__ void level(float (&B)[kMaxR], float eta, int src, bool top)
{
    const float bn = __shfl_sync(kFull, B[0], src);
#pragma unroll
    for (int s = 0; s + 1 < R; ++s) B[s] = fmaf(eta, B[s + 1], B[s + 1] + B[s]);
    if (!top) B[R - 1] = fmaf(eta, bn, bn + B[R - 1]);
}

// B[0..R) <- shared nodes lane*R .. lane*R + R - 1 at width R = width_at(WI),
// zero below node `lo`.
template <int WI>
__device__ __forceinline__ void load_width(float (&B)[kMaxR], const float *sh, int lane, int lo)
{
    constexpr int R = width_at(WI);
#pragma unroll
    for (int s = 0; s < R; ++s) {
        const int j = lane * R + s;
        B[s] = (j >= lo) ? sh[shidx(j)] : 0.f;
    }
}

// `n` levels at width width_at(WI); then, unless soff < 0, every lane's R
// slots to the warp's shared buffer at nodes soff + lane*R + s.
template <int WI>
__device__ __forceinline__ void levels(float (&B)[kMaxR], Lat &L, float *sh, int lane, int n, int soff)
{
    constexpr int R = width_at(WI);
    const int src = (lane + 1) & (kWarp - 1);
    const bool top = lane == kWarp - 1;
    // in runs up to the next rescale (every L.K levels, by 2^-L.E: exact)
    while (n > 0) {
        const int m = min(n, L.K - L.rescale);
        // one level per iteration: with four warps per scheduler at different
        // widths the level code's size costs more than the loop control
        // (measured: two levels per iteration at widths up to 16 / 32 / 40:
        // 45.4 / 57.7 / 60.0 ms against 44.7)
#pragma unroll 1
        for (int i = 0; i < m; ++i) level<R>(B, L.eta, src, top);
        n -= m;
        L.rescale += m;
        if (L.rescale == L.K) {
            L.rescale = 0;
            L.shift -= L.E;
#pragma unroll
            for (int s = 0; s < R; ++s) B[s] *= L.f;
        }
    }
    if (soff < 0) return;
    __syncwarp();
#pragma unroll
    for (int s = 0; s < R; ++s) sh[shidx(soff + lane * R + s)] = B[s];
    __syncwarp();
}

// Runtime width index -> the width's code.  Both the backward induction and
// its adjoint go through these, so each width's level code exists once
// (the instruction footprint, not the arithmetic, limits the deep lattices).
template <int WI>
__device__ __forceinline__ void levels_at(int wi, float (&B)[kMaxR], Lat &L, float *sh, int lane, int n, int soff)
{
    if constexpr (WI < kNWidths) {
        if (wi == WI) levels<WI>(B, L, sh, lane, n, soff);
        else levels_at<WI + 1>(wi, B, L, sh, lane, n, soff);
    }
}

template <int WI>
__device__ __forceinline__ void load_width_at(int wi, float (&B)[kMaxR], const float *sh, int lane, int lo)
{
    if constexpr (WI < kNWidths) {
        if (wi == WI) load_width<WI>(B, sh, lane, lo);
        else load_width_at<WI + 1>(wi, B, sh, lane, lo);
    }
}

template <int WI>
__device__ __forceinline__ int width_rt(int wi)
{
    if constexpr (WI + 1 < kNWidths) {
        if (wi != WI) return width_rt<WI + 1>(wi);
    }
    return width_at(WI);
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
    float S, K, sdt, a, q2;  // q2: v = 2q in storage order, -2q when reflected
    float eta, f;            // the level coefficient 2v / (1 - v); 2^-E
    int rk, re;              // a rescale by 2^-re every rk levels
    int N;
    bool put;
    bool refl;  // the lattice is stored reflected (node j at index N - j)
};

// Leaf at index i (0..N) of the priced side: its payoff and, for the greeks,
// its derivatives dS_T/dS (delta) and dS_T/dsigma (vega leaf part); all zero
// out of the money.  One exp per leaf.
__device__ __forceinline__ float leaf(const Opt &o, int i, float &dl, float &vg)
{
    const int j = o.refl ? o.N - i : i;
    const float m = (float)(2 * j - o.N);
    const float g = expf(o.a * m);
    const float ST = o.S * g;
    float b = 0.f;
    dl = vg = 0.f;
    if (o.put ? (ST < o.K) : (ST > o.K)) {
        b = o.put ? o.K - ST : ST - o.K;
        dl = o.put ? -g : g;
        vg = o.put ? -(ST * m * o.sdt) : ST * m * o.sdt;
    }
    return b;
}

// The payoffs of leaves 0..N into the warp's shared buffer, zero beyond N.
// Returns b, one past the last nonzero leaf (0 when every leaf is zero): the
// nonzero leaves are exactly 0..b-1, the priced side being out of the money.
__device__ __forceinline__ int leaves(const Opt &o, float *sh, int lane)
{
    __syncwarp();
    int last = -1;
    for (int j = lane; j <= kMaxSteps; j += kWarp) {
        float dl, vg;
        const float v = (j <= o.N) ? leaf(o, j, dl, vg) : 0.f;
        sh[shidx(j)] = v;
        if (v != 0.f) last = j;
    }
    __syncwarp();
    return __reduce_max_sync(kFull, last) + 1;
}

// The lattice passes of one option over the leaves in shared buffer 0,
// which each pass then uses as its repack buffer.
//
// Pass 0, the backward induction: from the N + 1 leaves (level N) down to
// the root.  The widths are walked downwards, starting at the width that
// holds min(N + 1, b) nodes (nodes from b up are zero): at width R the levels
// run until the level's nodes fit the next width, then the nodes are
// repacked through the shared buffer, down to level 1; the root follows
// from its two nodes.  Gives the root on lane 0 (the undiscounted price
// divided by lattice_scale(N, eta, shift)) and, on lane 0, d1 = C_1 - C_0 of
// level 1 (stored order) at the root's scaling.
//
// Pass 1 (greeks), its adjoint: weights A on the nodes of level N - 1 with
// root = sum_j A_j x_j for any level N - 1 of this recursion.  From the root
// (A = 1) outwards A'_j = A_j + (1 + eta) A_{j-1}, one node more
// per level.  Stored reversed (node j at slot 32R - 1 - j) this is the
// backward level itself, with the slots not reached yet at zero, so it runs
// on the same code while the widths are walked upwards, until the width
// holds the min(b, N) weights the dot products use (a node's weight depends
// only on nodes of lower index, so the rest of the level can be left out).
// Leaves node j < min(b, N) of level N - 1 at shared node 32 Rf - 1 - j
// (Rf returned in `rf`), with the
// power of two in A in shift_a: N - 1 levels here, and the one that pushes
// the leaves back to level N - 1, applied by the caller, counted too.
//
// Both passes go through one call of levels_at and one of load_width_at, so
// each width's code exists once in the kernel: the instruction footprint,
// not the arithmetic, limits the deep lattices.
//
// Inlined into the kernel (a call of its own cost the caller's saves and
// restores around it); the greeks, which need more registers, are the call.
template <bool FULL>
__device__ __forceinline__ float lattice(const Opt &o, int band, float *sh, int lane, bool adj, int &shift,
                                      float &d1, int &shift_a, int &rf)
{
    constexpr int W0 = FULL ? 0 : kW0Band;  // the widest width index this form runs
    constexpr int MR = width_at(W0);
    Lat L;
    L.eta = o.eta;
    L.f = o.f;
    L.K = o.rk;
    L.E = o.re;
    float B[kMaxR];
    float root = 0.f;
#pragma unroll 1
    for (int pass = 0; pass < (FULL && adj ? 2 : 1); ++pass) {
        L.shift = o.N;
        L.rescale = 0;
        int wi, active, lo = 0;
        bool load = false;
        if (pass == 0) {
            if (!FULL || min(o.N + 1, band) <= kMaxSteps) {
                // level N at the narrowest width that holds its nonzero band
                // (the caller guarantees that the banded form's widest holds it)
                wi = width_for<W0>(min(o.N + 1, band));
                load = true;
                active = o.N + 1;
            } else if constexpr (FULL) {
                // N = 2048: 2049 leaves do not fit 32 x 64 slots; level N-1 from the leaves
                wi = 0;
#pragma unroll
                for (int s = 0; s < kMaxR; ++s) {
                    const int j = lane * kMaxR + s;
                    const float lb = sh[shidx(j + 1)], b = sh[shidx(j)];
                    B[s] = fmaf(L.eta, lb, lb + b);
                }
                active = o.N;
                L.rescale = 1;
            }
        } else {
#pragma unroll
            for (int s = 0; s < MR; ++s) B[s] = 0.f;
            if (lane == kWarp - 1) B[0] = 1.0f;
            wi = kNWidths - 1;
            active = 1;
        }
        for (;;) {
            if (load) load_width_at<W0>(wi, B, sh, lane, lo);
            const int R = width_rt<W0>(wi);
            int n, soff = 0, next = wi;
            bool fin = false;
            if (pass == 0) {
                if (wi + 1 < kNWidths) {
                    n = active - kWarp * width_rt<W0>(wi + 1);
                    next = wi + 1;
                    load = true;
                    lo = 0;
                } else {  // width 1: down to level 1 (its two nodes on lanes 0, 1)
                    n = active - 2;
                    soff = -1;
                    fin = true;
                }
            } else {
                if (kWarp * R >= min(band, o.N)) {  // holds the weights used: the rest at this width
                    n = o.N - active;
                    fin = true;
                } else {
                    n = kWarp * R - active;
                    next = wi - 1;
                    soff = kWarp * (width_rt<W0>(next) - R);
                    load = true;
                    lo = soff;
                }
            }
            levels_at<W0>(wi, B, L, sh, lane, n, soff);
            active += pass == 0 ? -n : n;
            if (fin) break;
            wi = next;
        }
        if (pass == 0) {
            // the root from level 1, as the level code computes it, and d1
            const float c1 = __shfl_down_sync(kFull, B[0], 1);
            root = fmaf(L.eta, c1, c1 + B[0]);
            d1 = c1 - B[0];
            if (++L.rescale == L.K) {
                L.shift -= L.E;
                root *= L.f;
                d1 *= L.f;
            }
            shift = L.shift;
        } else {
            shift_a = L.shift;
            rf = width_rt<W0>(wi);
        }
    }
    return root;
}

constexpr float kLn2Hi = 0.693147182464599609375f;  // ln 2 = hi + lo
constexpr float kLn2Lo = (float)(0.69314718055994530942 - 0.693147182464599609375);

// 2^-sh (1 + eta/2)^-N: a root of the lattice C (rescaled to 2^sh) times
// this is the undiscounted value, since C = (2 + eta)^N V / disc^N.  The
// logarithm N ln(1 + eta/2) + sh ln 2 (two terms of up to ~1e3 that cancel
// to the rescales' rounding, below ~80) is formed in pairs of FP32 values,
// and its exponential is e^hi (1 - lo).
__device__ __forceinline__ float lattice_scale(int N, float eta, int sh)
{
    const float x = 0.5f * eta;
    const float2 l = (fabsf(x) <= 0.25f) ? df_scale((float)N, df_log1p(x))
                                         : df_split((double)N * log1p((double)x));
    const float2 t = df_add(l, df_scale((float)sh, make_float2(kLn2Hi, kLn2Lo)));
    return expf(-t.x) * (1.0f - t.y);
}

// Per-option values of the CRR lattice in FP32 (see the header).
struct Crr {
    float sdt, a, s1, q;
};

// LAT: also the lattice's coefficient and rescaling (eta, rk, re, f); the
// greeks pass needs only the CRR values.
template <bool LAT = true>
__device__ __forceinline__ Opt make_opt(float S, float K, float T, float sig, int N, float r, Crr &c)
{
    const float dt = T / (float)N;
    c.sdt = sqrtf(dt);
    c.a = sig * c.sdt;
    const float sh2 = sinhf(0.5f * c.a);
    const float num = expm1f(r * dt) - 2.0f * sh2 * sh2;
    c.s1 = sinhf(c.a);
    c.q = num / (2.0f * c.s1);
    Opt op;
    op.S = S;
    op.K = K;
    op.sdt = c.sdt;
    op.a = c.a;
    op.N = N;
    op.put = S > K;     // price the out-of-the-money side, then parity
    op.refl = !op.put;  // the call's nonzero leaves are the high ones: reflect
    op.q2 = op.refl ? -2.0f * c.q : 2.0f * c.q;
    op.eta = 0.f;
    op.rk = op.re = 0;
    op.f = 0.f;
    if (LAT) {
        op.eta = (2.0f * op.q2) / (1.0f - op.q2);
        // the largest node grows by at most 2 + eta per level: rk levels grow
        // it by at most 2^64, and the rescale removes the ceiling of that
        const float lg = log2f(2.0f + op.eta);
        op.rk = lg <= 1.0f ? kRescale : max(1, (int)((float)kRescale / lg));
        op.re = (int)ceilf((float)op.rk * lg);
        op.f = ldexpf(1.0f, -op.re);
    }
    return op;
}

// The per-option constants of the closed-form greeks' leaf sums: the high
// and low parts of C (see below) and the FP32 pair L.
struct GreeksConsts {
    float Ch, Cl, Lx, Ly;
};

__device__ __forceinline__ GreeksConsts greeks_consts(const Opt &op)
{
    // stored leaf i's weight in the root is the binomial pmf
    // C(N,i) w^i (1-w)^(N-i), w = (1 + v)/2 with v the lattice's own FP32
    // 2q in storage order (negated when reflected); its exponential g =
    // e^(a m), m = 2j - N = s (2i - N) (s = -1 when reflected), is folded
    // into the same logarithm:
    //   ln(pmf g) = C - ln i! - ln (N-i)! + i L,
    //   C = ln N! + N ln((1-v)/2) - s a N,  L = ln((1+v)/(1-v)) + 2 s a
    const float v = op.q2;
    const float sa = op.refl ? -op.a : op.a;
    float2 C, L;
    if (fabsf(v) <= 0.25f) {
        // FP32 pairs from the series (all lanes alike: no FP64)
        const float2 lp = df_log1p(v), lm = df_log1p(-v);
        const float2 lh = df_add(lm, make_float2(-kLn2Hi, -kLn2Lo));
        const float na = (float)op.N * sa;
        C = df_add(g_lfact[op.N], df_scale((float)op.N, lh));
        C = df_add(C, make_float2(-na, -fmaf((float)op.N, sa, -na)));
        L = df_add(df_add(lp, make_float2(-lm.x, -lm.y)), make_float2(2.0f * sa, 0.f));
    } else {
        // coarse lattices (|2q| > 1/4, a few steps): FP64 logs (no
        // shuffle here: a warp-synchronous call under this branch made
        // the compiler treat the whole kernel as divergent, +7%)
        const double lq = log1p(-(double)v);
        const float2 lfn = g_lfact[op.N];
        L = df_split(log1p((double)v) - lq + 2.0 * (double)sa);
        C = df_split((double)lfn.x + (double)lfn.y + (double)op.N * (lq - 0.69314718055994530942 - (double)sa));
    }
    // leaf in the money (exactly the first nz stored leaves): dS_T/dS =
    // g, dS_T/dsigma = S g m sqrt(dt) (both negated on the put side), so
    // one exponential gives the weighted g of both sums.
    // The high parts of C, of the table and of i L are multiples of 2^-10,
    // and so are their partial sums, exact in FP32 while below 2^14: ln
    // 2048! < 13572, and with |v| <= 1/4 |i L| < N (0.52 + 2a) < 1300 (a N
    // < 88 keeps the leaves finite).  The low parts (each below 2^-10)
    // are added in FP32, and the exponential of the exact high sum is
    // corrected by (1 + low sum).
    GreeksConsts k;
    k.Ch = rintf(C.x * 1024.f) * (1.0f / 1024.f);
    k.Cl = (C.x - k.Ch) + C.y;
    k.Lx = L.x;
    k.Ly = L.y;
    return k;
}

// This lane's part of the two leaf sums of an option with N steps and nz
// in-the-money leaves (leaves lane, lane + 32, ...), scaled by sgn and fv.
__device__ __forceinline__ float2 greeks_leaf_sums(const GreeksConsts &k, int N, int nz, float sgn, float fv, int lane)
{
    float sd = 0.f, sv = 0.f;
#pragma unroll 2
    for (int i = lane; i < nz; i += kWarp) {
        const float2 x = g_lfact[i], y = g_lfact[N - i];
        const float fi = (float)i;
        const float pr = fi * k.Lx;
        const float ph = rintf(pr * 1024.f) * (1.0f / 1024.f);
        const float pl = (pr - ph) + fmaf(fi, k.Ly, fmaf(fi, k.Lx, -pr));
        const float h = ((k.Ch - x.x) - y.x) + ph;
        const float lo = ((k.Cl - x.y) - y.y) + pl;
        const float e = expf(h);
        const float wg = fmaf(e, lo, e);
        sd += wg;
        sv = fmaf(wg, (float)(2 * i - N), sv);
    }
    return make_float2(sd * sgn, sv * fv);
}

// Sums of a pair over the warp (xor butterfly, a fixed order; every lane
// gets the sums).
__device__ __forceinline__ float2 warp_sum2(float2 v)
{
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        v.x += __shfl_xor_sync(kFull, v.x, o2);
        v.y += __shfl_xor_sync(kFull, v.y, o2);
    }
    return v;
}

// The vega sum's factor: dS_T/dsigma = S g m sqrt(dt), m in storage order
// (negated when reflected), both sums negated on the put side.
__device__ __forceinline__ float vega_factor(const Opt &op)
{
    const float sgn = op.put ? -1.f : 1.f;
    return (op.refl ? -sgn : sgn) * op.S * op.sdt;
}

// The greeks of the banded form in two launches: the lattice kernel leaves
// in greeks[o] the scratch pair (nz as int bits, the vega term through p),
// and the greeks kernel turns it into (delta, vega).  nz = -1 marks an
// option whose results are NaN.
__device__ __forceinline__ float2 greeks_scratch(int nz, float d1v) { return make_float2(__int_as_float(nz), d1v); }

// One option by one warp.  FULL: every node, and with greeks the adjoint
// lattice.  Otherwise the banded lattice and the price; with greeks the
// scratch pair for k_binomial_greeks.
template <bool FULL>
__device__ __forceinline__ void price_option(const BinoParams &p, int64_t o, float *sh)
{
    const float kNaN = __int_as_float(0x7fc00000);
    const int lane = threadIdx.x & 31;
    const int N = __ldg(p.steps + o);
    if (N < 1 || N > kMaxSteps) {  // outside the supported depths: NaN results
        if (lane == 0) {
            p.price[o] = kNaN;
            if (p.greeks) p.greeks[o] = FULL ? make_float2(kNaN, kNaN) : greeks_scratch(-1, kNaN);
        }
        return;
    }
    Crr c;
    const Opt op = make_opt(__ldg(p.S + o), __ldg(p.K + o), __ldg(p.T + o), __ldg(p.sigma + o), N, p.r, c);
    const bool greeks = p.greeks != nullptr;
    int shift = 0;
    float d1 = 0.f;
    int shift_a = 0, rf = 0;
    const int nz = leaves(op, sh, lane);
    const int band = FULL ? N + 1 : max(nz, 1);
    if (!FULL && min(N + 1, band) > kWarp * width_at(kW0Band)) {
        // a band wider than N/2 + 1 (sigma or T negative): outside the inputs
        if (lane == 0) {
            p.price[o] = kNaN;
            if (greeks) p.greeks[o] = greeks_scratch(-1, kNaN);
        }
        return;
    }
    const float b = lattice<FULL>(op, band, sh, lane, greeks && FULL, shift, d1, shift_a, rf);
    const float eta = op.eta, S = op.S, K = op.K, T = __ldg(p.T + o);
    if (op.refl) d1 = -d1;  // C_1 - C_0 in node order
    float delta = 0.f, vega = 0.f;
    if (FULL && greeks) {
        const int top = kWarp * rf - 1;  // node j of level N - 1 at shared node top - j
        // leaf derivatives pushed back one level (x'_j from x_j, x_{j+1}),
        // dotted with A; the leaves are evaluated again here rather than kept
        // in shared memory (two buffers would halve the resident warps)
        float sd = 0.f, sv = 0.f;
        const int need = min(band, N);  // the pushed-back leaf derivatives are zero from there on
        for (int j = lane; j < need; j += kWarp) {
            const float w = sh[shidx(top - j)];
            float d0, v0, d1l, v1;
            leaf(op, j, d0, v0);
            leaf(op, j + 1, d1l, v1);
            sd = fmaf(w, fmaf(eta, d1l, d1l + d0), sd);
            sv = fmaf(w, fmaf(eta, v1, v1 + v0), sv);
        }
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            sd += __shfl_xor_sync(kFull, sd, o2);
            sv += __shfl_xor_sync(kFull, sv, o2);
        }
        delta = sd;
        vega = sv;
    }
    if (lane == 0) {
        // remove the lattice's scaling, then discount
        const float disc = expf(-p.r * T);
        const float ls = lattice_scale(N, eta, shift);
        float price = (b * ls) * disc;
        if (op.put) price += S - K * disc;
        p.price[o] = price;
        if (greeks) {
            // B_1 - B_0 of the lattice scaled by 2 per level is (1 - v')^(N-1)
            // (C_1 - C_0), where 1 / (1 - v') = 1 + eta/2
            const float d1v = (d1 * fmaf(0.5f, eta, 1.0f)) * ls * disc;
            if (FULL) {
                // the adjoint weights carry the scaling of the N levels and 2^shift_a
                const float scale_a = lattice_scale(N, eta, shift_a) * disc;
                const float q2p = 2.0f * c.sdt * (-0.5f - c.q * (coshf(c.a) / c.s1));  // 2 dq/dsigma
                delta *= scale_a;
                if (op.put) delta += 1.0f;
                vega = fmaf((float)N * q2p, d1v, vega * scale_a);
                p.greeks[o] = make_float2(delta, vega);
            } else {
                p.greeks[o] = greeks_scratch(nz, d1v);
            }
        }
    }
}

template <bool FULL>
struct BinoBody {
    using Params = BinoParams;
    Params p;
    float *sh;

    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const int64_t o = (int64_t)(off + t);
        if (o < p.n) price_option<FULL>(p, o, sh);
    }
};

// FULL: every node of every level and the adjoint lattice (the reference
// form of the banded lattice and of the closed-form greeks).
template <bool FULL>
__global__ void __launch_bounds__(kWarp, FULL ? kMinCtasFull : kMinCtas) k_binomial(BinoParams prm, SchedArgs s)
{
    __shared__ float sh[kShNodes];
    BinoBody<FULL> b;
    b.p = prm;
    b.sh = sh;
    drive(s, b);
}

// The banded form's greeks pass: a plain launch after the lattice kernel on
// the same stream, `per` (1..32) options per warp, 8 warps per CTA.  Lane l
// < per sets up option l of its warp (its CRR values and the leaf sums'
// constants: a few hundred instructions that a warp per option computed 32
// times over), then the warp sums each option's leaves in turn (lane i of
// the warp takes leaves i, i + 32, ..., and the warp adds the lanes' sums
// in a fixed order), and each lane finishes its own option: delta and
// vega from the closed-form sums over the nz nonzero leaves (binomial
// probabilities, discounted), plus 1 for the calls priced through the put,
// and the vega term through p that the lattice left in the scratch pair.
// The batched launch takes the same path, so both agree bit for bit.  The
// launcher picks per so that the warps still fill the GPU (32 for 2^20
// options; 2 for 16384).
constexpr int kGreeksWarps = 8;

// One lane's option in the greeks pass.
struct GreeksLane {
    float2 *out;  // greeks[o] of the option, or nullptr: no option
    bool ok;      // a valid scratch pair (else NaN results)
    bool put;
    int N, nz;
    float d1v, T, r, sgn, fv;
    Crr c;
    GreeksConsts k;
};

// Reads option o's scratch pair and sets up its constants.
__device__ __forceinline__ void greeks_lane_setup(GreeksLane &g, const BinoParams &p, int64_t o)
{
    g.out = p.greeks + o;
    g.N = __ldg(p.steps + o);
    const float2 sc = *g.out;
    g.nz = __float_as_int(sc.x);
    g.d1v = sc.y;
    g.r = p.r;
    // nz outside 0..N+1: a marked option, or a scratch pair that no lattice
    // wrote (a run that ended with an error): NaN, nothing indexed by it
    g.ok = !(g.N < 1 || g.N > kMaxSteps || g.nz < 0 || g.nz > g.N + 1);
    if (g.ok) {
        g.T = __ldg(p.T + o);
        const Opt op = make_opt<false>(__ldg(p.S + o), __ldg(p.K + o), g.T, __ldg(p.sigma + o), g.N, p.r, g.c);
        g.k = greeks_consts(op);
        g.put = op.put;
        g.sgn = op.put ? -1.f : 1.f;
        g.fv = vega_factor(op);
    }
}

// The warp sums the leaves of the valid options of lanes 0..per-1 in turn;
// each lane gets its own option's sums.
__device__ __forceinline__ float2 greeks_warp_sums(const GreeksLane &g, int per, int lane)
{
    float2 sums = make_float2(0.f, 0.f);
    for (int j = 0; j < per; ++j) {
        if (!__shfl_sync(kFull, (int)g.ok, j)) continue;  // warp-uniform
        GreeksConsts kj;
        kj.Ch = __shfl_sync(kFull, g.k.Ch, j);
        kj.Cl = __shfl_sync(kFull, g.k.Cl, j);
        kj.Lx = __shfl_sync(kFull, g.k.Lx, j);
        kj.Ly = __shfl_sync(kFull, g.k.Ly, j);
        const int Nj = __shfl_sync(kFull, g.N, j), nzj = __shfl_sync(kFull, g.nz, j);
        const float sgnj = __shfl_sync(kFull, g.sgn, j), fvj = __shfl_sync(kFull, g.fv, j);
        const float2 dv = warp_sum2(greeks_leaf_sums(kj, Nj, nzj, sgnj, fvj, lane));
        if (lane == j) sums = dv;
    }
    return sums;
}

// (delta, vega) of the lane's option from its sums.
__device__ __forceinline__ void greeks_lane_finish(const GreeksLane &g, float2 sums)
{
    const float kNaN = __int_as_float(0x7fc00000);
    if (!g.ok) {
        *g.out = make_float2(kNaN, kNaN);
        return;
    }
    const float disc = expf(-g.r * g.T);
    const float q2p = 2.0f * g.c.sdt * (-0.5f - g.c.q * (coshf(g.c.a) / g.c.s1));  // 2 dq/dsigma
    float delta = sums.x * disc;
    if (g.put) delta += 1.0f;
    *g.out = make_float2(delta, fmaf((float)g.N * q2p, g.d1v, sums.y * disc));
}

__global__ void __launch_bounds__(kWarp * kGreeksWarps) k_binomial_greeks(BinoParams p, int per)
{
    const int lane = threadIdx.x & 31;
    const int64_t o = ((int64_t)blockIdx.x * kGreeksWarps + threadIdx.x / kWarp) * per + lane;
    GreeksLane g{};
    if (lane < per && o < p.n) greeks_lane_setup(g, p, o);
    const float2 sums = greeks_warp_sums(g, per, lane);
    if (g.out) greeks_lane_finish(g, sums);
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
    int32_t greeks;  // with_greeks
    int64_t total;
};

// Instance of global option o (binary search over `first`) as the
// parameters of one plain batch; false outside every instance.
__device__ __forceinline__ bool batch_option(const BinoBatchParams &p, int64_t o, BinoParams &bp, int64_t &local)
{
    if (o >= p.total) return false;
    int lo = 0, hi = p.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&p.inst[mid].first) <= o) lo = mid;
        else hi = mid - 1;
    }
    const BinoInstance &in = p.inst[lo];
    local = o - in.first;
    if (local < 0 || local >= in.n) return false;
    bp.S = in.S;
    bp.K = in.K;
    bp.T = in.T;
    bp.sigma = in.sigma;
    bp.steps = in.steps;
    bp.r = in.r;
    bp.n = in.n;
    bp.price = in.price;
    bp.greeks = p.greeks ? in.greeks : nullptr;
    return true;
}

struct BinoBatchBody {
    using Params = BinoBatchParams;
    Params p;
    float *sh;

    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        BinoParams bp;
        int64_t local;
        if (batch_option(p, (int64_t)(off + t), bp, local)) price_option<false>(bp, local, sh);
    }
};

__global__ void __launch_bounds__(kWarp, kMinCtas) k_binomial_batch(BinoBatchParams prm, SchedArgs s)
{
    __shared__ float sh[kShNodes];
    BinoBatchBody b;
    b.p = prm;
    b.sh = sh;
    drive(s, b);
}

// The batch's greeks pass (instances with a greeks array), as for one batch.
__global__ void __launch_bounds__(kWarp * kGreeksWarps) k_binomial_batch_greeks(BinoBatchParams prm, int per)
{
    const int lane = threadIdx.x & 31;
    const int64_t o = ((int64_t)blockIdx.x * kGreeksWarps + threadIdx.x / kWarp) * per + lane;
    GreeksLane g{};
    BinoParams bp;
    int64_t local;
    if (lane < per && batch_option(prm, o, bp, local) && bp.greeks) greeks_lane_setup(g, bp, local);
    const float2 sums = greeks_warp_sums(g, per, lane);
    if (g.out) greeks_lane_finish(g, sums);
}

// Options per warp of the greeks pass: as many as keep every resident warp
// slot of the GPU busy, at most 32.
int greeks_per_warp(int64_t n)
{
    static int slots = 0;  // resident warps of k_binomial_greeks on device 0
    if (!slots) {
        int sms = 0, ctas = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, k_binomial_greeks, kWarp * kGreeksWarps, 0) !=
                cudaSuccess) {
            cudaGetLastError();
            sms = 152;
            ctas = 5;
        }
        slots = sms * ctas * kGreeksWarps;
    }
    const int64_t per = n / (slots > 0 ? slots : 1);
    return (int)(per < 1 ? 1 : (per > kWarp ? kWarp : per));
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

int ctas_per_sm() { return occ((const void *)k_binomial<false>); }

template <bool FULL>
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
    k_binomial<FULL><<<c.grid, kWarp, 0, c.stream>>>(p, s);
    mark_main_end(c);
    if (!FULL && p.greeks && p.n > 0) {
        const int per = greeks_per_warp(p.n);
        const int64_t warps = ((int64_t)p.n + per - 1) / per;
        k_binomial_greeks<<<(unsigned)((warps + kGreeksWarps - 1) / kGreeksWarps), kWarp * kGreeksWarps, 0,
                            c.stream>>>(p, per);
    }
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

int batch_ctas_per_sm() { return occ((const void *)k_binomial_batch); }

ecl_status l_batch(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    BinoBatchParams p;
    p.inst = a.buf<const BinoInstance>(0);
    p.count = a.i32(1);
    p.total = a.i64(2);
    p.greeks = a.i32(3) ? 1 : 0;
    k_binomial_batch<<<c.grid, kWarp, 0, c.stream>>>(p, s);
    mark_main_end(c);
    if (p.greeks && p.total > 0) {
        const int per = greeks_per_warp(p.total);
        const int64_t warps = (p.total + per - 1) / per;
        k_binomial_batch_greeks<<<(unsigned)((warps + kGreeksWarps - 1) / kGreeksWarps), kWarp * kGreeksWarps, 0,
                                  c.stream>>>(p, per);
    }
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
    1, 0, kWarp, 0, validate, grain, nchunks, ctas_per_sm, launch<false>,
};

// The same program computing every node of every level, with the top
// neighbour of the last lane set to zero, and the greeks from the adjoint
// lattice: the reference form of the banded lattice (identical prices) and
// of the closed-form greeks (within ~1e-6).
extern const KernelDesc kBinomialFull = {
    "binomial_full", 9,
    {{"S", A_BUF_IN}, {"K", A_BUF_IN}, {"T", A_BUF_IN}, {"sigma", A_BUF_IN}, {"steps", A_BUF_IN},
     {"r", A_F32}, {"n", A_I32}, {"price", A_BUF_OUT}, {"greeks", A_BUF_OUT_OPT}},
    1, 0, kWarp, 0, validate, grain, nchunks, ctas_per_sm, launch<true>,
};

}  // namespace ecl

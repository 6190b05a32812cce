// Row-tiled GEMM on the 5th-generation tensor cores (tcgen05) of sm_103a.
//
//   C[M x N] (FP32, row-major) = A[M x K] (bf16, row-major) * Bt[N x K]^T
//
// The NDRange is the grid of 128 x 256 output tiles: one work-group = one
// tile (the config's 128-row tiles).  A chunk is a pair of vertically
// adjacent tiles, one 256 x 256 block computed together: each staged slice
// of Bt feeds two MMAs, twice the MMA work per staged byte of a single
// tile (measured at 8192^3: 0.749 -> 0.649 ms).  Pairs are numbered in
// column groups (tc::tile_at: the pairs of W tile columns row by row, then
// the next W columns), so that a wave of concurrent pairs reads few strips
// of A and Bt; with an odd number of tile rows the last row's tiles follow
// as single-tile chunks.  The scheduling unit is two tile rows, so Static /
// Dynamic / HGuided hand out packages of whole pairs of tile rows.
//
// Each persistent CTA (192 threads, one per SM) is warp-specialised:
//   warp 0    claims chunks from the package queue and feeds a ring of
//             chunk slots; its lane 0 issues the TMA loads (128B swizzle)
//             of the 64-wide K slices of A (256 rows) and Bt (256 rows)
//             into a 3-stage ring of 64 KB stages;
//   warp 1    allocates 512 TMEM columns (the pair's two 128 x 256 FP32
//             accumulators) and its lane 0 issues tcgen05.mma (M128 N256
//             K16, BF16 inputs, FP32 accumulation), two per K16 step, one
//             per tile of the pair, committing each stage back to the
//             loader and the finished pair to the epilogue;
//   warps 2-5 read both accumulators with tcgen05.ld (each warp its 32-lane
//             quarter of TMEM), store FP32 to C with 128-bit stores, free the
//             accumulators and account for the finished chunk.
// The loads of the next pair's first stages overlap the epilogue; its MMAs
// wait for the accumulators to be free.
//
// Split mode (gemm_split3): A and Bt are FP32; a first kernel splits every
// value x into hi = bf16(x) and lo = bf16(x - hi) (the subtraction is exact
// in FP32), then the main loop runs three K sweeps, hi*hi, hi*lo, lo*hi,
// into the same FP32 accumulator.
//
// Every wait on an mbarrier is bounded in time; a wait that gives up sets
// the queue's error word (ECL_ERR_TIMEOUT), the CTA drains its own copies in
// flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ecl_internal.h"
#include "sched.cuh"
#include "tc.cuh"

namespace ecl {
namespace {

using namespace tc;

// A work-group is one BM x BN output tile; a chunk is a pair of vertically
// adjacent tiles (CM = 2 BM rows), computed together so that each staged
// slice of Bt feeds two MMAs: twice the MMA work per staged byte of a
// single tile.
constexpr int BM = 128, BN = 256, BK = 64, PAIR = 2, CM = PAIR * BM, NSTAGE = 3, RING = 4;
constexpr int STAGE_A = CM * BK * 2;  // 32 KB
constexpr int STAGE_B = BN * BK * 2;  // 32 KB
constexpr int NTHREADS = 192;
constexpr uint32_t TMEM_COLS = 512;   // the pair's two 128 x 256 FP32 accumulators
constexpr int64_t TILE_DONE = -1;
constexpr uint32_t IDESC = idesc_bf16(BM, BN);

struct __align__(1024) GemmSmem {
    uint8_t a[NSTAGE][STAGE_A];
    uint8_t b[NSTAGE][STAGE_B];
    uint64_t full[NSTAGE], empty[NSTAGE];
    uint64_t tfull, tempty;  // the accumulators (one pair at a time)
    uint64_t rfull[RING], rempty[RING];
    uint64_t drain;
    uint64_t stored;  // the four epilogue warps finished storing a tile
    int64_t ring_tile[RING];
    uint32_t ring_pkg[RING], ring_nch[RING];
    uint32_t tmem_base;
    uint32_t err;
    uint32_t flag;
    uint32_t chunks;
    uint64_t t_first, t_last;
};

constexpr size_t SMEM_BYTES = sizeof(GemmSmem) + 1024;  // + alignment slack

struct GemmParams {
    float *C;
    int64_t M, N, K;
    int64_t tiles_n;
    int64_t tmf;          // full pairs of tile rows (floor(tile rows / 2))
    tc::TileOrder order;  // pair id -> pair row, tile column
    uint32_t kblocks;   // K slices per sweep
    uint32_t sweeps;    // 1 (bf16) or 3 (split)
};

// Work-groups and chunks.  The first F = 2 tmf tn work-groups (tmf full
// pairs of tile rows, tn tile columns) are the tile pairs, two work-groups
// each, numbered in column groups (tc::tile_at over the tmf x tn grid of
// pairs); with an odd number of tile rows the last row's tn tiles follow,
// one work-group and one chunk each.  Packages hold whole pairs of tile rows
// (grain 2 tn), so a package starts at an even work-group, and only the
// last package reaches past F.
__host__ __device__ inline uint32_t gemm_chunks(int64_t F, uint64_t off, uint64_t len)
{
    const uint64_t b = off + len, f = (uint64_t)F;
    const uint64_t pairs = off < f ? ((b < f ? b : f) - off) / PAIR : 0;
    const uint64_t singles = b > f ? b - (off > f ? off : f) : 0;
    return (uint32_t)(pairs + singles);
}

// Chunk code of chunk t of the package at `off`: a pair id below tmf tn, a
// single tile of the last row (tmf tn + its column) from there on.
__host__ __device__ inline int64_t gemm_chunk_code(int64_t F, int64_t tmf_tn, uint64_t off, uint64_t t)
{
    const uint64_t f = (uint64_t)F;
    const uint64_t cp = off < f ? (f - off) / PAIR : 0;  // pairs from off up to F
    if (t < cp) return (int64_t)(off / PAIR + t);
    const uint64_t w = (off > f ? off : f) + (t - cp);   // a work-group of the last row
    return tmf_tn + (int64_t)(w - f);
}

struct GemmBody {  // chunk bookkeeping for the scheduler
    using Params = GemmParams;
    static __host__ __device__ uint32_t nchunks(const Params &q, uint64_t off, uint64_t len)
    {
        return gemm_chunks(2 * q.tmf * q.tiles_n, off, len);
    }
};

// First row and column of chunk `code` (its 256 rows; the rows from M on are
// neither loaded, TMA fills them with zeros, nor stored).
__device__ __forceinline__ void chunk_origin(const GemmParams &p, int64_t code, int &m0, int &n0)
{
    const int64_t full = p.tmf * p.tiles_n;
    if (code < full) {
        int64_t pr, nt;
        tc::tile_at(p.order, code, pr, nt);
        m0 = (int)(pr * CM);
        n0 = (int)(nt * BN);
    } else {
        m0 = (int)(p.tmf * CM);
        n0 = (int)((code - full) * BN);
    }
}

// ---------------------------------------------------------------- kernel
struct Maps {
    CUtensorMap a[2];  // [0] bf16 A (or A_hi), [1] A_lo
    CUtensorMap b[2];  // [0] bf16 Bt (or B_hi), [1] B_lo
};

__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm(const __grid_constant__ Maps maps, GemmParams p, SchedArgs s)
{
    extern __shared__ uint8_t smem_raw[];
    GemmSmem &sm = *reinterpret_cast<GemmSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const bool mono = (s.mode == MODE_MONO);
    const uint32_t d = mono ? 0u : blockIdx.x / s.C;
    unsigned int *gerr = &s.q->error;
    volatile uint32_t *err = &sm.err;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NSTAGE; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.empty[i], 1);
        }
        mbar_init(&sm.tfull, 1);
        mbar_init(&sm.tempty, 4);
        for (int i = 0; i < RING; ++i) {
            mbar_init(&sm.rfull[i], 1);
            mbar_init(&sm.rempty[i], 5);  // MMA lane + one lane per epilogue warp
        }
        mbar_init(&sm.drain, 1);
        mbar_init(&sm.stored, 4);
        sm.err = 0;
        sm.chunks = 0;
        sm.t_first = 0;
        sm.t_last = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    const uint32_t ksteps = p.kblocks * p.sweeps;

    if (warp == 0) {
        // ------------------------------------------------ claims + TMA producer
        if (lane == 0) {
            uint32_t ri = 0, kq = 0;  // ring slots used, K steps issued
            bool more = true;
            while (more && !*err) {
                Claim c{};
                if (mono) {
                    c.off = 0;
                    c.t_begin = blockIdx.x;
                    c.t_end = blockIdx.x + 1;
                    c.nchunks = 0;
                    more = false;
                } else {
                    c = claim_chunks<GemmBody>(s, p, d);
                    if (c.done) break;
                    if (!sm.t_first) sm.t_first = gtime();
                }
                for (uint32_t t = c.t_begin; t < c.t_end && !*err; ++t) {
                    const int64_t code = gemm_chunk_code(2 * p.tmf * p.tiles_n, p.tmf * p.tiles_n, c.off, t);
                    const uint32_t r = ri % RING;
                    if (!mbar_wait(&sm.rempty[r], ((ri / RING) & 1) ^ 1, err, gerr)) break;
                    sm.ring_tile[r] = code;
                    sm.ring_pkg[r] = c.pkg;
                    sm.ring_nch[r] = c.nchunks;
                    mbar_arrive(&sm.rfull[r]);
                    ++ri;
                    int m0, n0;
                    chunk_origin(p, code, m0, n0);
                    for (uint32_t k = 0; k < ksteps; ++k, ++kq) {
                        const uint32_t st = kq % NSTAGE;
                        if (!mbar_wait(&sm.empty[st], ((kq / NSTAGE) & 1) ^ 1, err, gerr)) break;
                        const uint32_t sweep = k / p.kblocks;
                        const int kx = (int)((k % p.kblocks) * BK);
                        const CUtensorMap *am = &maps.a[sweep == 2 ? 1 : 0];
                        const CUtensorMap *bm = &maps.b[sweep == 1 ? 1 : 0];
                        mbar_expect_tx(&sm.full[st], STAGE_A + STAGE_B);
                        tma_load(sm.a[st], am, kx, m0, &sm.full[st]);
                        tma_load(sm.b[st], bm, kx, n0, &sm.full[st]);
                    }
                }
            }
            // tell the consumers there is no more work
            if (!*err) {
                const uint32_t r = ri % RING;
                if (mbar_wait(&sm.rempty[r], ((ri / RING) & 1) ^ 1, err, gerr)) {
                    sm.ring_tile[r] = TILE_DONE;
                    mbar_arrive(&sm.rfull[r]);
                }
            }
            // drain: every issued copy has landed before the CTA can exit
            const uint32_t last = kq < NSTAGE ? kq : NSTAGE;
            for (uint32_t i = 0; i < last; ++i) {
                const uint32_t q = kq - 1 - i;
                uint32_t e2 = 0;
                mbar_wait(&sm.full[q % NSTAGE], (q / NSTAGE) & 1, &e2, gerr);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t ri = 0, kq = 0, tc = 0;
            bool issued = false;
            for (;;) {
                const uint32_t r = ri % RING;
                if (!mbar_wait(&sm.rfull[r], (ri / RING) & 1, err, gerr)) break;
                const int64_t tile = sm.ring_tile[r];
                mbar_arrive(&sm.rempty[r]);
                ++ri;
                if (tile == TILE_DONE) break;
                // the epilogue of the previous pair has read both accumulators
                if (!mbar_wait(&sm.tempty, (tc & 1) ^ 1, err, gerr)) break;
                tc_fence_after();
                bool ok = true;
                for (uint32_t k = 0; k < ksteps; ++k, ++kq) {
                    const uint32_t st = kq % NSTAGE;
                    if (!mbar_wait(&sm.full[st], (kq / NSTAGE) & 1, err, gerr)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sm.a[st]), b0 = smem_u32(sm.b[st]);
                    // A rows h * 128 .. + 127 of the stage (16 KB apart, 128B swizzle
                    // atoms of 8 rows) into accumulator h, the Bt slice shared
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
#pragma unroll
                        for (int h = 0; h < PAIR; ++h)
                            umma(tmem + h * BN, sdesc(a0 + h * (BM * BK * 2) + kk * 32), sdesc(b0 + kk * 32), IDESC,
                                 (k | kk) != 0);
                    umma_commit(&sm.empty[st]);
                    issued = true;
                }
                if (!ok) break;
                umma_commit(&sm.tfull);
                ++tc;
            }
            if (issued) {  // every MMA issued by this CTA has completed
                umma_commit(&sm.drain);
                uint32_t e2 = 0;
                mbar_wait(&sm.drain, 0, &e2, gerr);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue (warps 2-5)
        const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
        uint32_t ri = 0, tc = 0;
        for (;;) {
            const uint32_t r = ri % RING;
            bool ok = true;
            long long tile = 0;
            uint32_t pkg = 0, nch = 0;
            if (lane == 0) {
                ok = mbar_wait(&sm.rfull[r], (ri / RING) & 1, err, gerr);
                if (ok) {
                    tile = sm.ring_tile[r];
                    pkg = sm.ring_pkg[r];
                    nch = sm.ring_nch[r];
                    mbar_arrive(&sm.rempty[r]);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tile = __shfl_sync(0xffffffffu, tile, 0);
            pkg = __shfl_sync(0xffffffffu, pkg, 0);
            nch = __shfl_sync(0xffffffffu, nch, 0);
            ++ri;
            if (tile == TILE_DONE) break;
            if (lane == 0) ok = mbar_wait(&sm.tfull, tc & 1, err, gerr);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            int cm0, cn0;
            chunk_origin(p, tile, cm0, cn0);
            const int64_t n0 = cn0;
            const bool vec = (p.N % 4) == 0;
#pragma unroll 1
            for (int q = 0; q < PAIR * (BN / 32); ++q) {
                const int h = q / (BN / 32), cc = q % (BN / 32);  // tile h of the pair, 32 columns cc
                const int64_t m = (int64_t)cm0 + h * BM + quarter * 32 + lane;
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + h * BN + cc * 32, v);
                const int64_t c0 = n0 + cc * 32;
                if (m < p.M) {
                    float *row = p.C + m * p.N;
                    if (vec && c0 + 31 < p.N) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4 *>(row + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (c0 + j < p.N) row[c0 + j] = v[j];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sm.tempty);
                mbar_arrive(&sm.stored);
            }
            // chunk accounting once all four warps stored the tile (bounded wait)
            if (threadIdx.x == 64 && !mono) {
                if (mbar_wait(&sm.stored, tc & 1, err, gerr)) {
                    const uint64_t te = gtime();
                    sm.t_last = te;
                    sm.chunks += 1;
                    if (finish_chunks(s, pkg, 1, nch, te) && s.coverage) {
                        const PkgRec rec = s.rec[pkg];
                        for (uint64_t w = rec.off; w < rec.off + rec.len; ++w) atomicAdd(&s.coverage[w], 1u);
                    }
                }
            }
            ++tc;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
    if (!mono) {
        const uint64_t tf = sm.t_first, tl = sm.t_last;
        exit_protocol(s, d, tf, tl, tl > tf ? tl - tf : 0, sm.chunks, &sm.flag);
    }
}

// ---------------------------------------------------------------- split / cast
// hi = bf16(x), lo = bf16(x - hi) for the A and Bt operands of the split mode.
__global__ void k_split(const float *A, const float *B, __nv_bfloat16 *ah, __nv_bfloat16 *al, __nv_bfloat16 *bh,
                        __nv_bfloat16 *bl, int64_t na, int64_t nb)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += stride) {
        const bool isa = i < na;
        const int64_t j = isa ? i : i - na;
        const float x = isa ? A[j] : B[j];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        if (isa) {
            ah[j] = h;
            al[j] = l;
        } else {
            bh[j] = h;
            bl[j] = l;
        }
    }
}

struct CastParams {
    const float *in;
    __nv_bfloat16 *out;
    int64_t n;
    uint32_t lws;
};

struct CastBody {
    using Params = CastParams;
    Params p;
    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }
    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const int64_t b = (int64_t)(off + t) * p.lws;
        for (int64_t i = b + threadIdx.x; i < b + p.lws && i < p.n; i += blockDim.x)
            p.out[i] = __float2bfloat16_rn(p.in[i]);
    }
};

__global__ void __launch_bounds__(256) k_cast(CastParams prm, SchedArgs s)
{
    CastBody b;
    b.p = prm;
    drive(s, b);
}

// ---------------------------------------------------------------- host side
bool set_smem()
{
    static std::atomic<unsigned long long> done{0};
    return smem_limit_once((const void *)k_gemm, (int)SMEM_BYTES, done);
}

int gemm_ctas_per_sm()
{
    if (!set_smem()) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gemm, NTHREADS, SMEM_BYTES) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ecl_status v_gemm_common(const KArgs &a, uint64_t gws, uint32_t lws, size_t esize, std::string &err)
{
    const int64_t M = a.i32(3), N = a.i32(4), K = a.i32(5);
    if (M <= 0 || N <= 0 || K <= 0) {
        err = "M, N and K must be positive";
        return ECL_ERR_ARG;
    }
    if (K % 8) {
        err = "K must be a multiple of 8 (16-byte rows for the tensor copies)";
        return ECL_ERR_ARG;
    }
    if (lws != (uint32_t)(BM * BN)) {
        err = "lws must be 32768 (one 128 x 256 output tile per work-group)";
        return ECL_ERR_SIZE;
    }
    const uint64_t tiles = (uint64_t)((M + BM - 1) / BM) * (uint64_t)((N + BN - 1) / BN);
    if (gws < tiles * lws) {
        err = "the NDRange does not cover the output tiles";
        return ECL_ERR_SIZE;
    }
    if (a.bytes[0] < (uint64_t)M * K * esize || a.bytes[1] < (uint64_t)N * K * esize ||
        a.bytes[2] < (uint64_t)M * N * 4) {
        err = "buffers smaller than the matrices";
        return ECL_ERR_BUFFER;
    }
    if ((uintptr_t)a.ptr[0] % 16 || (uintptr_t)a.ptr[1] % 16 || (uintptr_t)a.ptr[2] % 16) {
        err = "A, Bt and C must be 16-byte aligned";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

ecl_status v_bf16(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    return v_gemm_common(a, gws, lws, 2, err);
}

ecl_status v_split(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    return v_gemm_common(a, gws, lws, 4, err);
}

// Packages of whole pairs of tile rows: a chunk (two vertically adjacent
// tiles) never straddles two packages.
uint64_t grain_rows(const KArgs &a, uint64_t, uint32_t) { return (uint64_t)PAIR * ((a.i32(4) + BN - 1) / BN); }

uint32_t nchunks_pairs(const KArgs &a, uint64_t, uint32_t, uint64_t off, uint64_t len)
{
    const int64_t tm = (a.i32(3) + BM - 1) / BM, tn = (a.i32(4) + BN - 1) / BN;
    return gemm_chunks(2 * (tm / PAIR) * tn, off, len);
}

uint32_t nchunks_tiles(const KArgs &, uint64_t, uint32_t, uint64_t, uint64_t len) { return (uint32_t)len; }

ecl_status launch_main(const Maps &maps, const KArgs &a, const SchedArgs &s, const LaunchCtx &c, uint32_t sweeps,
                       std::string &err)
{
    if (!set_smem()) {
        err = "cannot raise the shared-memory limit";
        return ECL_ERR_CUDA;
    }
    GemmParams p;
    p.C = a.buf<float>(2);
    p.M = a.i32(3);
    p.N = a.i32(4);
    p.K = a.i32(5);
    p.tiles_n = (p.N + BN - 1) / BN;
    p.kblocks = (uint32_t)((p.K + BK - 1) / BK);
    p.sweeps = sweeps;
    // tile pairs numbered in column groups over the grid of full CM-row pairs
    p.tmf = ((p.M + BM - 1) / BM) / PAIR;
    p.order = tile_order(p.tmf > 0 ? p.tmf : 1, p.tiles_n, c.grid, (double)CM, (double)BN);  // strips of equal K
    k_gemm<<<c.grid, NTHREADS, SMEM_BYTES, c.stream>>>(maps, p, s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

ecl_status l_bf16(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    const int64_t M = a.i32(3), N = a.i32(4), K = a.i32(5);
    Maps maps;
    if (!make_map(&maps.a[0], a.ptr[0], M, K, CM, err) || !make_map(&maps.b[0], a.ptr[1], N, K, BN, err))
        return ECL_ERR_CUDA;
    maps.a[1] = maps.a[0];
    maps.b[1] = maps.b[0];
    return launch_main(maps, a, s, c, 1, err);
}

ecl_status l_split(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    const int64_t M = a.i32(3), N = a.i32(4), K = a.i32(5);
    const size_t na = (size_t)M * K, nb = (size_t)N * K;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t oa = al(na * 2), ob = al(nb * 2);
    char *ws = (char *)workspace_get(c.ws, 2 * oa + 2 * ob, err);
    if (!ws) return ECL_ERR_CUDA;
    __nv_bfloat16 *ah = (__nv_bfloat16 *)ws, *alo = (__nv_bfloat16 *)(ws + oa);
    __nv_bfloat16 *bh = (__nv_bfloat16 *)(ws + 2 * oa), *blo = (__nv_bfloat16 *)(ws + 2 * oa + ob);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    k_split<<<sms * 8, 256, 0, c.stream>>>(a.buf<const float>(0), a.buf<const float>(1), ah, alo, bh, blo,
                                           (int64_t)na, (int64_t)nb);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("split launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    mark_main_begin(c);
    Maps maps;
    if (!make_map(&maps.a[0], ah, M, K, CM, err) || !make_map(&maps.a[1], alo, M, K, CM, err) ||
        !make_map(&maps.b[0], bh, N, K, BN, err) || !make_map(&maps.b[1], blo, N, K, BN, err))
        return ECL_ERR_CUDA;
    return launch_main(maps, a, s, c, 3, err);
}

// ---- cast_bf16: in float[n], out bf16[n], n
ecl_status v_cast(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    const int64_t n = a.i64(2);
    if (n <= 0) {
        err = "n must be positive";
        return ECL_ERR_ARG;
    }
    if (gws < (uint64_t)n || lws > 1024) {
        err = "one element per work-item, lws <= 1024";
        return ECL_ERR_SIZE;
    }
    if (a.bytes[0] < (uint64_t)n * 4 || a.bytes[1] < (uint64_t)n * 2) {
        err = "buffers smaller than n elements";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

uint64_t grain1(const KArgs &, uint64_t, uint32_t) { return 1; }

int cast_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cast, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ecl_status l_cast(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    CastParams p;
    p.in = a.buf<const float>(0);
    p.out = a.buf<__nv_bfloat16>(1);
    p.n = a.i64(2);
    p.lws = c.lws;
    k_cast<<<c.grid, 256, 0, c.stream>>>(p, s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

}  // namespace

extern const KernelDesc kGemmBF16 = {
    "gemm_bf16", 6,
    {{"A", A_BUF_IN}, {"Bt", A_BUF_IN}, {"C", A_BUF_OUT}, {"M", A_I32}, {"N", A_I32}, {"K", A_I32}},
    1, 1, NTHREADS, 4, v_bf16, grain_rows, nchunks_pairs, gemm_ctas_per_sm, l_bf16, true,
};

extern const KernelDesc kGemmSplit3 = {
    "gemm_split3", 6,
    {{"A", A_BUF_IN}, {"Bt", A_BUF_IN}, {"C", A_BUF_OUT}, {"M", A_I32}, {"N", A_I32}, {"K", A_I32}},
    1, 1, NTHREADS, 4, v_split, grain_rows, nchunks_pairs, gemm_ctas_per_sm, l_split, true,
};

extern const KernelDesc kCastBF16 = {
    "cast_bf16", 3,
    {{"in", A_BUF_IN}, {"out", A_BUF_OUT}, {"n", A_I64}},
    1, 1, 256, 0, v_cast, grain1, nchunks_tiles, cast_ctas_per_sm, l_cast,
};

}  // namespace ecl

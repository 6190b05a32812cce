// Six-product split-BF16 GEMM on the tcgen05 tensor cores, for FP32 inputs:
//
//   C[M x N] (FP32) = A[M x K] (FP32, row-major) * Bt[N x K]^T (FP32, row-major)
//
// A first kernel splits every value x into three bf16 terms, x = h + m + l
// with h = bf16(x), m = bf16(x - h), l = bf16((x - h) - m) (the FP32
// subtractions are exact, so the three terms hold all 24 bits of x).  The
// main kernel sums the six products of order up to 2^-16 relative,
//   hh + (hm + mh + hl + lh + mm),
// and leaves out ml, lm and ll (below 2^-23 |a||b| per term).
//
// Accuracy is set by how partial sums are accumulated, so the two groups
// are kept apart:
//   * hh (the bulk) goes into a fresh TMEM accumulator for every chunk of
//     `chunk_kb` K slices of 64; the epilogue warps add each chunk into FP32
//     registers (round to nearest), so the tensor core never accumulates
//     more than 4 * chunk_kb products into a large running sum;
//   * the five cross products (2^-8 smaller) accumulate over the whole K in
//     a second TMEM accumulator, added to the running sum once per tile.
// Two hh buffers let the MMAs of chunk i+1 run while chunk i is promoted;
// two cross buffers let one tile's epilogue overlap the next tile.  TMEM
// columns: hh[0], hh[1], cross[0], cross[1], 128 each (512 in total).
//
// Tiles are 128 x 128 (one work-group each), numbered in column groups as
// in the plain GEMM; the scheduling unit is as many tiles as a tile row
// holds.  Each persistent CTA (192 threads, one per SM):
//   warp 0    claims tiles and issues the TMA loads of the six operand
//             pieces (A and Bt: h, m, l) of each 64-wide K slice into a
//             2-stage ring (96 KB per stage);
//   warp 1    allocates TMEM and issues the MMAs (M128 N128 K16);
//   warps 2-5 promote the hh chunks, add the cross sums, store C and
//             account for finished tiles.
// Every mbarrier wait is bounded; a wait that gives up sets ECL_ERR_TIMEOUT,
// the CTA drains its copies in flight, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ecl_internal.h"
#include "sched.cuh"
#include "tc.cuh"

namespace ecl {
namespace {

using namespace tc;

constexpr int BM = 128, BN = 128, BK = 64, NST = 2, RING = 4;
constexpr int PIECE = BM * BK * 2;  // 16 KB (BN == BM)
constexpr int NTHREADS = 192;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t COL_HH = 0, COL_X = 2 * BN;
constexpr int64_t TILE_DONE = -1;
constexpr uint32_t IDESC = idesc_bf16(BM, BN);
static_assert(BN == BM, "A and Bt pieces share one tile size");

struct __align__(1024) Smem6 {
    uint8_t a[NST][3][PIECE];  // h, m, l of A
    uint8_t b[NST][3][PIECE];  // h, m, l of Bt
    uint64_t full[NST], empty[NST];
    uint64_t hfull[2], hempty[2];  // hh chunk accumulators
    uint64_t xfull[2], xempty[2];  // cross accumulators (per tile)
    uint64_t rfull[RING], rempty[RING];
    uint64_t drain;
    uint64_t stored;
    int64_t ring_tile[RING];
    uint32_t ring_pkg[RING], ring_nch[RING];
    uint32_t tmem_base;
    uint32_t err;
    uint32_t flag;
    uint32_t chunks;
    uint64_t t_first, t_last;
};

constexpr size_t SMEM_BYTES = sizeof(Smem6) + 1024;  // + alignment slack

struct Gemm6Params {
    float *C;
    int64_t M, N, K;
    int64_t tiles_n;
    tc::TileOrder order;  // work-group id -> output tile
    uint32_t kblocks;   // K slices of 64
    uint32_t chunk_kb;  // K slices per hh chunk
};

struct Gemm6Body {  // chunk bookkeeping for the scheduler
    using Params = Gemm6Params;
    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }
};

struct Maps6 {
    CUtensorMap a[3];  // h, m, l
    CUtensorMap b[3];
};

// Chunks (hh promotions) of K slices [0, kblocks): ceil(kblocks / chunk_kb).
__device__ __forceinline__ uint32_t nchunk_of(const Gemm6Params &p) { return (p.kblocks + p.chunk_kb - 1) / p.chunk_kb; }

__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm6(const __grid_constant__ Maps6 maps, Gemm6Params p, SchedArgs s)
{
    extern __shared__ uint8_t smem_raw[];
    Smem6 &sm = *reinterpret_cast<Smem6 *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const bool mono = (s.mode == MODE_MONO);
    const uint32_t d = mono ? 0u : blockIdx.x / s.C;
    unsigned int *gerr = &s.q->error;
    volatile uint32_t *err = &sm.err;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NST; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.hfull[i], 1);
            mbar_init(&sm.hempty[i], 4);
            mbar_init(&sm.xfull[i], 1);
            mbar_init(&sm.xempty[i], 4);
        }
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

    if (warp == 0) {
        // ------------------------------------------------ claims + TMA producer
        if (lane == 0) {
            uint32_t ri = 0, kq = 0;  // ring slots used, K slices issued
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
                    c = claim_chunks<Gemm6Body>(s, p, d);
                    if (c.done) break;
                    if (!sm.t_first) sm.t_first = gtime();
                }
                for (uint32_t t = c.t_begin; t < c.t_end && !*err; ++t) {
                    const int64_t tile = (int64_t)(c.off + t);
                    const uint32_t r = ri % RING;
                    if (!mbar_wait(&sm.rempty[r], ((ri / RING) & 1) ^ 1, err, gerr)) break;
                    sm.ring_tile[r] = tile;
                    sm.ring_pkg[r] = c.pkg;
                    sm.ring_nch[r] = c.nchunks;
                    mbar_arrive(&sm.rfull[r]);
                    ++ri;
                    int64_t mt, nt;
                    tc::tile_at(p.order, tile, mt, nt);
                    const int m0 = (int)(mt * BM);
                    const int n0 = (int)(nt * BN);
                    for (uint32_t k = 0; k < p.kblocks; ++k, ++kq) {
                        const uint32_t st = kq % NST;
                        if (!mbar_wait(&sm.empty[st], ((kq / NST) & 1) ^ 1, err, gerr)) break;
                        const int kx = (int)(k * BK);
                        mbar_expect_tx(&sm.full[st], 6 * PIECE);
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            tma_load(sm.a[st][q], &maps.a[q], kx, m0, &sm.full[st]);
                            tma_load(sm.b[st][q], &maps.b[q], kx, n0, &sm.full[st]);
                        }
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
            const uint32_t last = kq < NST ? kq : NST;
            for (uint32_t i = 0; i < last; ++i) {
                const uint32_t q = kq - 1 - i;
                uint32_t e2 = 0;
                mbar_wait(&sm.full[q % NST], (q / NST) & 1, &e2, gerr);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t ri = 0, kq = 0, hc = 0, tc_ = 0;
            bool issued = false;
            for (;;) {
                const uint32_t r = ri % RING;
                if (!mbar_wait(&sm.rfull[r], (ri / RING) & 1, err, gerr)) break;
                const int64_t tile = sm.ring_tile[r];
                mbar_arrive(&sm.rempty[r]);
                ++ri;
                if (tile == TILE_DONE) break;
                const uint32_t xb = tc_ & 1;
                if (!mbar_wait(&sm.xempty[xb], ((tc_ >> 1) & 1) ^ 1, err, gerr)) break;
                const uint32_t dx = tmem + COL_X + xb * BN;
                bool ok = true;
                for (uint32_t k = 0; k < p.kblocks; ++k, ++kq) {
                    const uint32_t st = kq % NST;
                    const uint32_t in_chunk = k % p.chunk_kb;
                    const uint32_t hb = hc & 1;
                    if (in_chunk == 0 && !mbar_wait(&sm.hempty[hb], ((hc >> 1) & 1) ^ 1, err, gerr)) {
                        ok = false;
                        break;
                    }
                    if (!mbar_wait(&sm.full[st], (kq / NST) & 1, err, gerr)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dh = tmem + COL_HH + hb * BN;
                    const uint32_t ah = smem_u32(sm.a[st][0]), am = smem_u32(sm.a[st][1]), al = smem_u32(sm.a[st][2]);
                    const uint32_t bh = smem_u32(sm.b[st][0]), bm = smem_u32(sm.b[st][1]), bl = smem_u32(sm.b[st][2]);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t o = kk * 32;
                        umma(dh, sdesc(ah + o), sdesc(bh + o), IDESC, (in_chunk | kk) != 0);
                        umma(dx, sdesc(al + o), sdesc(bh + o), IDESC, (k | kk) != 0);
                        umma(dx, sdesc(ah + o), sdesc(bl + o), IDESC, 1);
                        umma(dx, sdesc(am + o), sdesc(bm + o), IDESC, 1);
                        umma(dx, sdesc(am + o), sdesc(bh + o), IDESC, 1);
                        umma(dx, sdesc(ah + o), sdesc(bm + o), IDESC, 1);
                    }
                    umma_commit(&sm.empty[st]);
                    issued = true;
                    if (in_chunk + 1 == p.chunk_kb || k + 1 == p.kblocks) {
                        umma_commit(&sm.hfull[hb]);
                        ++hc;
                    }
                }
                if (!ok) break;
                umma_commit(&sm.xfull[xb]);
                ++tc_;
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
        const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31 (one output row per thread)
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        uint32_t ri = 0, hc = 0, tc_ = 0;
        const uint32_t nch = nchunk_of(p);
        for (;;) {
            const uint32_t r = ri % RING;
            bool ok = true;
            long long tile = 0;
            uint32_t pkg = 0, pnch = 0;
            if (lane == 0) {
                ok = mbar_wait(&sm.rfull[r], (ri / RING) & 1, err, gerr);
                if (ok) {
                    tile = sm.ring_tile[r];
                    pkg = sm.ring_pkg[r];
                    pnch = sm.ring_nch[r];
                    mbar_arrive(&sm.rempty[r]);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tile = __shfl_sync(0xffffffffu, tile, 0);
            pkg = __shfl_sync(0xffffffffu, pkg, 0);
            pnch = __shfl_sync(0xffffffffu, pnch, 0);
            ++ri;
            if (tile == TILE_DONE) break;
            float run[BN];
#pragma unroll
            for (int j = 0; j < BN; ++j) run[j] = 0.f;
            for (uint32_t c = 0; c < nch && ok; ++c, ++hc) {
                const uint32_t hb = hc & 1;
                if (lane == 0) ok = mbar_wait(&sm.hfull[hb], (hc >> 1) & 1, err, gerr);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
                tc_fence_after();
#pragma unroll
                for (int cc = 0; cc < BN / 32; ++cc) {
                    float v[32];
                    tmem_ld32(tmem + lane_off + COL_HH + hb * BN + cc * 32, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) run[cc * 32 + j] += v[j];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.hempty[hb]);
            }
            if (!ok) break;
            const uint32_t xb = tc_ & 1;
            if (lane == 0) ok = mbar_wait(&sm.xfull[xb], (tc_ >> 1) & 1, err, gerr);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            int64_t mt, nt;
            tc::tile_at(p.order, tile, mt, nt);
            const int64_t m = mt * BM + quarter * 32 + lane;
            const int64_t n0 = nt * BN;
            const bool vec = (p.N % 4) == 0;
#pragma unroll
            for (int cc = 0; cc < BN / 32; ++cc) {
                float v[32];
                tmem_ld32(tmem + lane_off + COL_X + xb * BN + cc * 32, v);
                const int64_t c0 = n0 + cc * 32;
                if (m < p.M) {
                    float *row = p.C + m * p.N;
                    if (vec && c0 + 31 < p.N) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4 *>(row + c0 + j) =
                                make_float4(run[cc * 32 + j] + v[j], run[cc * 32 + j + 1] + v[j + 1],
                                            run[cc * 32 + j + 2] + v[j + 2], run[cc * 32 + j + 3] + v[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (c0 + j < p.N) row[c0 + j] = run[cc * 32 + j] + v[j];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sm.xempty[xb]);
                mbar_arrive(&sm.stored);
            }
            // chunk accounting once all four warps stored the tile (bounded wait)
            if (threadIdx.x == 64 && !mono) {
                if (mbar_wait(&sm.stored, tc_ & 1, err, gerr)) {
                    const uint64_t te = gtime();
                    sm.t_last = te;
                    sm.chunks += 1;
                    if (finish_chunks(s, pkg, 1, pnch, te) && s.coverage) {
                        const PkgRec rec = s.rec[pkg];
                        for (uint64_t w = rec.off; w < rec.off + rec.len; ++w) atomicAdd(&s.coverage[w], 1u);
                    }
                }
            }
            ++tc_;
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

// x = h + m + l for the A and Bt operands: h = bf16(x), m = bf16(x - h),
// l = bf16((x - h) - m).
__global__ void k_split6(const float *A, const float *B, __nv_bfloat16 *a3, __nv_bfloat16 *b3, int64_t na, int64_t nb)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + nb; i += stride) {
        const bool isa = i < na;
        const int64_t j = isa ? i : i - na;
        const float x = isa ? A[j] : B[j];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const float r = x - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r);
        const __nv_bfloat16 l = __float2bfloat16_rn(r - __bfloat162float(m));
        __nv_bfloat16 *o = isa ? a3 : b3;
        const int64_t n = isa ? na : nb;
        o[j] = h;
        o[n + j] = m;
        o[2 * n + j] = l;
    }
}

// ---------------------------------------------------------------- host side
bool set_smem()
{
    static std::atomic<unsigned long long> done{0};
    return smem_limit_once((const void *)k_gemm6, (int)SMEM_BYTES, done);
}

int ctas_per_sm()
{
    if (!set_smem()) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gemm6, NTHREADS, SMEM_BYTES) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ecl_status validate(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    const int64_t M = a.i32(3), N = a.i32(4), K = a.i32(5), ck = a.i32(6);
    if (M <= 0 || N <= 0 || K <= 0) {
        err = "M, N and K must be positive";
        return ECL_ERR_ARG;
    }
    if (K % 8) {
        err = "K must be a multiple of 8 (16-byte rows for the tensor copies)";
        return ECL_ERR_ARG;
    }
    if (ck < 0 || ck > 1 << 20) {
        err = "chunk_k must be 0 (default) or a positive number of K slices of 64";
        return ECL_ERR_ARG;
    }
    if (lws != (uint32_t)(BM * BN)) {
        err = "lws must be 16384 (one 128 x 128 output tile per work-group)";
        return ECL_ERR_SIZE;
    }
    const uint64_t tiles = (uint64_t)((M + BM - 1) / BM) * (uint64_t)((N + BN - 1) / BN);
    if (gws < tiles * lws) {
        err = "the NDRange does not cover the output tiles";
        return ECL_ERR_SIZE;
    }
    if (a.bytes[0] < (uint64_t)M * K * 4 || a.bytes[1] < (uint64_t)N * K * 4 || a.bytes[2] < (uint64_t)M * N * 4) {
        err = "buffers smaller than the matrices";
        return ECL_ERR_BUFFER;
    }
    if ((uintptr_t)a.ptr[2] % 16) {
        err = "C must be 16-byte aligned";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

uint64_t grain_rows(const KArgs &a, uint64_t, uint32_t) { return (uint64_t)((a.i32(4) + BN - 1) / BN); }

uint32_t nchunks_tiles(const KArgs &, uint64_t, uint32_t, uint64_t, uint64_t len) { return (uint32_t)len; }

ecl_status launch(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    const int64_t M = a.i32(3), N = a.i32(4), K = a.i32(5);
    const size_t na = (size_t)M * K, nb = (size_t)N * K;
    const size_t oa = (3 * na * 2 + 255) & ~(size_t)255;
    char *ws = (char *)workspace_get(c.ws, oa + 3 * nb * 2, err);
    if (!ws) return ECL_ERR_CUDA;
    __nv_bfloat16 *a3 = (__nv_bfloat16 *)ws, *b3 = (__nv_bfloat16 *)(ws + oa);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    k_split6<<<sms * 8, 256, 0, c.stream>>>(a.buf<const float>(0), a.buf<const float>(1), a3, b3, (int64_t)na,
                                            (int64_t)nb);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("split launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    mark_main_begin(c);
    Maps6 maps;
    for (int q = 0; q < 3; ++q)
        if (!make_map(&maps.a[q], a3 + q * na, M, K, BM, err) || !make_map(&maps.b[q], b3 + q * nb, N, K, BN, err))
            return ECL_ERR_CUDA;
    if (!set_smem()) {
        err = "cannot raise the shared-memory limit";
        cudaGetLastError();
        return ECL_ERR_CUDA;
    }
    Gemm6Params p;
    p.C = a.buf<float>(2);
    p.M = M;
    p.N = N;
    p.K = K;
    p.tiles_n = (N + BN - 1) / BN;
    p.kblocks = (uint32_t)((K + BK - 1) / BK);
    p.order = tc::tile_order((M + BM - 1) / BM, p.tiles_n, c.grid, (double)BM, (double)BN);  // strips of equal K
    const int32_t ck = a.i32(6);
    p.chunk_kb = ck > 0 ? (uint32_t)ck : 1u;
    if (p.chunk_kb > p.kblocks) p.chunk_kb = p.kblocks;
    k_gemm6<<<c.grid, NTHREADS, SMEM_BYTES, c.stream>>>(maps, p, s);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

}  // namespace

extern const KernelDesc kGemmSplit6 = {
    "gemm_split6", 7,
    {{"A", A_BUF_IN}, {"Bt", A_BUF_IN}, {"C", A_BUF_OUT}, {"M", A_I32}, {"N", A_I32}, {"K", A_I32},
     {"chunk_k", A_I32}},
    1, 1, NTHREADS, 4, validate, grain_rows, nchunks_tiles, ctas_per_sm, launch, true,
};

}  // namespace ecl

// Separable Gaussian blur (Table 2: lws 128, image + filter-weight buffers,
// out pattern 1:1), clamp-to-edge borders, FP32.
//
// Work-item g produces pixel g of the row-major image, so a package of
// work-groups is a range of pixels: a band of rows with possibly partial
// first and last rows.  The kernel splits a package into chunks of
// (32-row band) x (224 output columns; 256 staged with the halo).  A chunk
// runs the vertical pass first (one thread per column of the tile plus its
// 2r halo columns; the 32 outputs of a column slide down the input rows in
// registers, each staged value read once) into a shared-memory tile, then
// the horizontal pass (four consecutive outputs per thread, 128-bit shared
// loads and 128-bit stores).  Only pixels inside the package's range are
// written, so packages that split a row are handled exactly.
//
// The 31-tap case has a fully unrolled path with the weights in
// registers; other odd tap counts up to 63 use a plain loop path.
#include <cuda_runtime.h>

#include "ecl_internal.h"
#include "sched.cuh"

namespace ecl {
namespace {

constexpr int kBlock = 256;
constexpr int kRB = 32;        // output rows per chunk
constexpr int kTW = 224;       // output columns per chunk (vertical pass: 256 columns = 8 warps)
constexpr int kMaxTaps = 63;
constexpr int kSW = kTW + 32;  // staged / vertical tile width: 224 + 2*15 halo + 2 pad = 256

struct GaussParams {
    const float *in;
    const float *w;
    float *out;
    int64_t W, H;
    int32_t taps;
    uint32_t lws;
};

struct ChunkGeom {
    int64_t p0, p1;    // pixel range of the package
    int64_t y0, rows;  // band
    int64_t x0;        // tile
};

__host__ __device__ inline uint32_t gauss_nchunks(const GaussParams &p, uint64_t off, uint64_t len)
{
    const int64_t npx = p.W * p.H;
    const int64_t p0 = (int64_t)(off * p.lws);
    int64_t p1 = (int64_t)((off + len) * p.lws);
    if (p1 > npx) p1 = npx;
    if (p0 >= p1) return 0;
    const int64_t r0 = p0 / p.W, r1 = (p1 - 1) / p.W;
    const int64_t nb = (r1 - r0 + kRB) / kRB;
    const int64_t nt = (p.W + kTW - 1) / kTW;
    return (uint32_t)(nb * nt);
}

__device__ __forceinline__ ChunkGeom geom(const GaussParams &p, uint64_t off, uint64_t len, uint32_t t)
{
    ChunkGeom g;
    const int64_t npx = p.W * p.H;
    g.p0 = (int64_t)(off * p.lws);
    g.p1 = (int64_t)((off + len) * p.lws);
    if (g.p1 > npx) g.p1 = npx;
    const uint32_t nt = (uint32_t)((p.W + kTW - 1) / kTW);
    int64_t r0, r1;
    if (npx < (int64_t)0x7fffffff) {  // 32-bit divisions: a few instructions instead of ~100
        const uint32_t W = (uint32_t)p.W;
        r0 = (uint32_t)g.p0 / W;
        r1 = (uint32_t)(g.p1 - 1) / W;
    } else {
        r0 = g.p0 / p.W;
        r1 = (g.p1 - 1) / p.W;
    }
    const uint32_t b = t / nt, c = t % nt;
    g.y0 = r0 + (int64_t)b * kRB;
    g.rows = min((int64_t)kRB, r1 + 1 - g.y0);
    g.x0 = (int64_t)c * kTW;
    return g;
}

__device__ __forceinline__ int64_t clampl(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

// Horizontal pass + store for one chunk.  Shared tile row o, column c holds
// the vertical result at image column x0 - BASE + c (row stride SW floats).
// T > 0: unrolled with the weights in registers; T == 0: any tap count,
// weights in shared memory.
template <int T, int SW, int BASE>
__device__ __forceinline__ void horizontal_store(const GaussParams &p, const ChunkGeom &g, const float *sv,
                                                 const float *wreg, const float *wsh)
{
    const int taps = T ? T : p.taps;
    const int r = taps / 2;
    const bool vec = (p.W % 4) == 0;
    constexpr int NCB = kTW / 4;  // 4-column blocks per row
    for (int q = threadIdx.x; q < g.rows * NCB; q += kBlock) {
        const int o = q / NCB, cb = q % NCB;
        const int64_t x = g.x0 + 4 * cb;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const float *row = sv + o * SW + 4 * cb + (BASE - r);  // T == 0 path
        if (T) {
            // aligned 128-bit loads from column 4*cb + OFF0, values shifted by OFFR
            constexpr int OFF = BASE - (T ? T : 1) / 2;
            constexpr int OFF0 = OFF & ~3, OFFR = OFF & 3;
            constexpr int NV = (OFFR + T + 3 + 3) / 4 * 4;
            const float *arow = sv + o * SW + 4 * cb + OFF0;
            float v[NV];
#pragma unroll
            for (int q = 0; q < NV / 4; ++q) {
                const float4 f = *reinterpret_cast<const float4 *>(arow + 4 * q);
                v[4 * q] = f.x;
                v[4 * q + 1] = f.y;
                v[4 * q + 2] = f.z;
                v[4 * q + 3] = f.w;
            }
#pragma unroll
            for (int u = 0; u < (T ? T : 1); ++u)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] = fmaf(wreg[u], v[OFFR + j + u], acc[j]);
        } else {
            for (int u = 0; u < taps; ++u) {
                const float wu = wsh[u];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] = fmaf(wu, row[j + u], acc[j]);
            }
        }
        const int64_t y = g.y0 + o;
        const int64_t lin = y * p.W + x;
        if (vec && x + 3 < p.W && lin >= g.p0 && lin + 3 < g.p1) {
            *reinterpret_cast<float4 *>(p.out + lin) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x + j < p.W && lin + j >= g.p0 && lin + j < g.p1) p.out[lin + j] = acc[j];
        }
    }
}

// 31-tap path.  The chunk's input tile (62 rows x 256 columns: image
// columns x0-16 .. x0+239, rows clamped to the image) is staged in shared
// memory with 16-byte cp.async copies (element-wise clamped loads at the
// left/right borders), in two groups of rows (0..31, 32..61) so that the
// vertical pass starts on the first while the second is in flight.  The
// vertical pass reads shared memory at compile-time offsets, with the 31
// weights and the 32 outputs of a column in registers; its results
// overwrite the staged rows and feed the horizontal pass.
constexpr int kNIN = kRB + 30;   // staged input rows
constexpr int kSC = kSW / 4;     // 16-byte chunks per staged row

__device__ __forceinline__ void cp_async16(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

struct Gauss31Body {
    static constexpr uint32_t kThreads = kBlock;
    using Params = GaussParams;
    Params p;
    float (*st)[kSW];  // [kNIN][kSW] staged input, then [kRB][kSW] vertical results
    float wr[31];

    static __host__ __device__ uint32_t nchunks(const Params &q, uint64_t off, uint64_t len)
    {
        return gauss_nchunks(q, off, len);
    }

    // Staged rows [kb, ke) (kb a multiple of 4) as one group of copies.
    __device__ __forceinline__ void stage(const ChunkGeom &g, int kb, int ke)
    {
        const bool vec_ok = (p.W % 4) == 0 && ((uintptr_t)p.in % 16) == 0;
        const int c4 = threadIdx.x % kSC;  // fixed 16-byte column chunk per thread
        const int64_t xs = g.x0 - 16 + 4 * c4;
        const bool vec = vec_ok && xs >= 0 && xs + 4 <= p.W;
        const int k0 = kb + threadIdx.x / kSC;
        const int64_t ylo = g.y0 - 15 + k0;
        if (vec && g.y0 - 15 + kb >= 0 && g.y0 - 15 + ke <= p.H) {  // interior rows: pointer steps, no clamps
            const float *src = p.in + ylo * p.W + xs;
            const int64_t step = (int64_t)(kBlock / kSC) * p.W;
            for (int k = k0; k < ke; k += kBlock / kSC, src += step) cp_async16(&st[k][4 * c4], src);
        } else {
            for (int k = k0; k < ke; k += kBlock / kSC) {
                const int64_t ys = clampl(g.y0 - 15 + k, 0, p.H - 1);
                const float *row = p.in + ys * p.W;
                float *dst = &st[k][4 * c4];
                if (vec) {
                    cp_async16(dst, row + xs);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = __ldg(row + clampl(xs + j, 0, p.W - 1));
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    __device__ __forceinline__ void run(uint64_t off, uint64_t len, uint32_t t, uint32_t) { tile(geom(p, off, len, t)); }

    // One 32-row x 224-column output tile of the image p.
    __device__ __forceinline__ void tile(const ChunkGeom &g)
    {
        // the staged rows in two groups of copies: the vertical pass starts on
        // the first while the second is in flight
        constexpr int kHalf = 32;
        stage(g, 0, kHalf);
        stage(g, kHalf, kNIN);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        body_sync(kBlock);
        // vertical pass: staged column c <-> image column x0 - 16 + c, one column per thread
        float acc[kRB];
        const int c1 = threadIdx.x;
#pragma unroll
        for (int o = 0; o < kRB; ++o) acc[o] = 0.f;
#pragma unroll
        for (int k = 0; k < kHalf; ++k) {
            const float v = st[k][c1];
#pragma unroll
            for (int o = 0; o < kRB; ++o)
                if (k - o >= 0 && k - o < 31) acc[o] = fmaf(wr[k - o], v, acc[o]);
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        body_sync(kBlock);
#pragma unroll
        for (int k = kHalf; k < kNIN; ++k) {
            const float v = st[k][c1];
#pragma unroll
            for (int o = 0; o < kRB; ++o)
                if (k - o >= 0 && k - o < 31) acc[o] = fmaf(wr[k - o], v, acc[o]);
        }
        body_sync(kBlock);  // every staged row has been read
#pragma unroll
        for (int o = 0; o < kRB; ++o) st[o][c1] = acc[o];
        body_sync(kBlock);
        // horizontal pass: output x needs vertical results at staged columns x - x0 + 1 .. + 31
        horizontal_store<31, kSW, 16>(p, g, &st[0][0], wr, nullptr);
        body_sync(kBlock);
    }
};

// Any odd tap count up to 63: plain loops, weights in shared memory.  Shared
// tile column c holds image column x0 - 31 + c (room for radius 31).
constexpr int kSWA = kTW + 64;

struct GaussAnyBody {
    static constexpr uint32_t kThreads = kBlock;
    using Params = GaussParams;
    Params p;
    float *sv;  // [kRB][kSWA]
    const float *wsh;

    static __host__ __device__ uint32_t nchunks(const Params &q, uint64_t off, uint64_t len)
    {
        return gauss_nchunks(q, off, len);
    }

    __device__ __forceinline__ void run(uint64_t off, uint64_t len, uint32_t t, uint32_t)
    {
        const ChunkGeom g = geom(p, off, len, t);
        const int r = p.taps / 2;
        for (int c = threadIdx.x; c < kTW + 2 * r; c += kBlock) {
            const int col = c + (31 - r);
            const int64_t xs = clampl(g.x0 - r + c, 0, p.W - 1);
            for (int o = 0; o < g.rows; ++o) {
                float acc = 0.f;
                for (int v = 0; v < p.taps; ++v) {
                    const int64_t ys = clampl(g.y0 + o - r + v, 0, p.H - 1);
                    acc = fmaf(wsh[v], __ldg(p.in + ys * p.W + xs), acc);
                }
                sv[o * kSWA + col] = acc;
            }
        }
        body_sync(kBlock);
        horizontal_store<0, kSWA, 31>(p, g, sv, nullptr, wsh);
        body_sync(kBlock);
    }
};

__global__ void __launch_bounds__(kBlock + 32, 3) k_gauss31(GaussParams prm, SchedArgs s)
{
    extern __shared__ __align__(16) float smem_g[];
    Gauss31Body b;
    b.p = prm;
    b.st = reinterpret_cast<float(*)[kSW]>(smem_g);
#pragma unroll
    for (int u = 0; u < 31; ++u) b.wr[u] = __ldg(prm.w + u);
    drive_ws(s, b);
}

// ---------------------------------------------------------------- batches
// Many images of uneven size (31 taps each, own weights) as one NDRange of
// tiles: image i owns work-groups [first_i, first_i + tiles_i), one per
// 32-row x 224-column output tile (row-major over the image's tile grid);
// a work-group finds its image by binary search over `first`.  Mirrors
// ecl_gaussian_image in include/ecl.h.
struct GaussImage {
    const float *in;
    float *out;
    const float *w;
    int32_t W, H;
    int64_t first;
    int64_t tiles;
};
static_assert(sizeof(GaussImage) == 48, "ecl_gaussian_image layout");

__host__ __device__ inline int64_t gauss_tiles(int64_t W, int64_t H)
{
    return ((H + kRB - 1) / kRB) * ((W + kTW - 1) / kTW);
}

struct GaussBatchParams {
    const GaussImage *img;
    int32_t count;
    int64_t total;
};

struct Gauss31BatchBody {
    static constexpr uint32_t kThreads = kBlock;
    using Params = GaussBatchParams;
    Params p;
    Gauss31Body b;

    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const int64_t wg = (int64_t)(off + t);
        if (wg >= p.total) return;
        int lo = 0, hi = p.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&p.img[mid].first) <= wg) lo = mid;
            else hi = mid - 1;
        }
        const GaussImage &im = p.img[lo];
        const int64_t local = wg - im.first;
        // out of range, empty, or an output the 128-bit stores cannot use: skipped
        if (local < 0 || local >= im.tiles || im.W <= 0 || im.H <= 0 || ((uintptr_t)im.out & 15) ||
            local >= gauss_tiles(im.W, im.H))
            return;
        b.p.in = im.in;
        b.p.out = im.out;
        b.p.w = im.w;
        b.p.W = im.W;
        b.p.H = im.H;
        b.p.taps = 31;
        b.p.lws = 1;
#pragma unroll
        for (int u = 0; u < 31; ++u) b.wr[u] = __ldg(im.w + u);
        const int64_t ntx = (im.W + kTW - 1) / kTW;
        ChunkGeom g;
        g.p0 = 0;
        g.p1 = (int64_t)im.W * im.H;
        g.y0 = (local / ntx) * kRB;
        g.rows = min((int64_t)kRB, (int64_t)im.H - g.y0);
        g.x0 = (local % ntx) * kTW;
        b.tile(g);
    }
};

__global__ void __launch_bounds__(kBlock + 32, 3) k_gauss31_batch(GaussBatchParams prm, SchedArgs s)
{
    extern __shared__ __align__(16) float smem_g[];
    Gauss31BatchBody b;
    b.p = prm;
    b.b.st = reinterpret_cast<float(*)[kSW]>(smem_g);
    drive_ws(s, b);
}

__global__ void __launch_bounds__(kBlock + 32) k_gauss_any(GaussParams prm, SchedArgs s)
{
    __shared__ __align__(16) float sv[kRB][kSWA];
    __shared__ float wsh[kMaxTaps];
    for (int u = threadIdx.x; u < prm.taps; u += blockDim.x) wsh[u] = prm.w[u];
    __syncthreads();
    GaussAnyBody b;
    b.p = prm;
    b.sv = &sv[0][0];
    b.wsh = wsh;
    drive_ws(s, b);
}

GaussParams params_of(const KArgs &a, uint32_t lws)
{
    GaussParams p;
    p.in = a.buf<const float>(0);
    p.w = a.buf<const float>(1);
    p.out = a.buf<float>(2);
    p.W = a.i32(3);
    p.H = a.i32(4);
    p.taps = a.i32(5);
    p.lws = lws;
    return p;
}

ecl_status validate(const KArgs &a, uint64_t gws, uint32_t, std::string &err)
{
    const int64_t W = a.i32(3), H = a.i32(4), T = a.i32(5);
    if (W <= 0 || H <= 0) {
        err = "width and height must be positive";
        return ECL_ERR_ARG;
    }
    if (T < 1 || T > kMaxTaps || T % 2 == 0) {
        err = "taps must be odd, 1..63";
        return ECL_ERR_ARG;
    }
    const uint64_t npx = (uint64_t)W * (uint64_t)H;
    if (a.bytes[0] < npx * 4 || a.bytes[2] < npx * 4) {
        err = "image buffers smaller than width*height floats";
        return ECL_ERR_BUFFER;
    }
    if (a.bytes[1] < (uint64_t)T * 4) {
        err = "weight buffer smaller than taps floats";
        return ECL_ERR_BUFFER;
    }
    if ((uintptr_t)a.ptr[2] % 16) {
        err = "output buffer must be 16-byte aligned";
        return ECL_ERR_BUFFER;
    }
    if (gws < npx) {
        err = "the NDRange (one pixel per work-item) does not cover the image";
        return ECL_ERR_SIZE;
    }
    return ECL_OK;
}

uint64_t grain(const KArgs &, uint64_t, uint32_t) { return 1; }

uint32_t nchunks(const KArgs &a, uint64_t, uint32_t lws, uint64_t off, uint64_t len)
{
    return gauss_nchunks(params_of(a, lws), off, len);
}

constexpr size_t kSmem31 = sizeof(float) * kNIN * kSW;

bool set_smem_attr()
{
    static std::atomic<unsigned long long> done{0};
    return smem_limit_once((const void *)k_gauss31, (int)kSmem31, done);
}

int ctas_per_sm()
{
    if (!set_smem_attr()) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gauss31, kBlock + 32, kSmem31) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ecl_status launch(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    const GaussParams p = params_of(a, c.lws);
    if (p.taps == 31) {
        if (!set_smem_attr()) {
            err = "cannot raise the shared-memory limit";
            return ECL_ERR_CUDA;
        }
        k_gauss31<<<c.grid, kBlock + 32, kSmem31, c.stream>>>(p, s);
    } else {
        // the generic path keeps a smaller resident count; the plan used the fast path's
        // count, so it is clamped here: more CTAs than resident is still correct
        k_gauss_any<<<c.grid, kBlock + 32, 0, c.stream>>>(p, s);
    }
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

// ---- gaussian_batch: table of images, count, total tiles
ecl_status v_batch(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    const int64_t count = a.i32(1), total = a.i64(2);
    if (count <= 0 || total <= 0) {
        err = "count and total must be positive";
        return ECL_ERR_ARG;
    }
    if (a.bytes[0] < (uint64_t)count * sizeof(GaussImage) || (uintptr_t)a.ptr[0] % 16) {
        err = "the image table must hold count 16-byte aligned entries of 48 bytes";
        return ECL_ERR_BUFFER;
    }
    if (lws != kBlock) {
        err = "lws must be 256 (one work-group per output tile)";
        return ECL_ERR_SIZE;
    }
    if (gws < (uint64_t)total * kBlock) {
        err = "the NDRange does not cover the images' tiles";
        return ECL_ERR_SIZE;
    }
    return ECL_OK;
}

uint32_t nchunks_batch(const KArgs &, uint64_t, uint32_t, uint64_t, uint64_t len) { return (uint32_t)len; }

bool set_smem_attr_batch()
{
    static std::atomic<unsigned long long> done{0};
    return smem_limit_once((const void *)k_gauss31_batch, (int)kSmem31, done);
}

int batch_ctas_per_sm()
{
    if (!set_smem_attr_batch()) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gauss31_batch, kBlock + 32, kSmem31) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ecl_status l_batch(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    if (!set_smem_attr_batch()) {
        err = "cannot raise the shared-memory limit";
        return ECL_ERR_CUDA;
    }
    GaussBatchParams p;
    p.img = a.buf<const GaussImage>(0);
    p.count = a.i32(1);
    p.total = a.i64(2);
    k_gauss31_batch<<<c.grid, kBlock + 32, kSmem31, c.stream>>>(p, s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

}  // namespace

extern const KernelDesc kGaussianBatch = {
    "gaussian_batch", 3, {{"images", A_BUF_IN}, {"count", A_I32}, {"total", A_I64}},
    1, 0, kBlock + 32, 0, v_batch, grain, nchunks_batch, batch_ctas_per_sm, l_batch,
};

extern const KernelDesc kGaussian = {
    "gaussian",
    6,
    {{"in", A_BUF_IN}, {"weights", A_BUF_IN}, {"out", A_BUF_OUT}, {"width", A_I32}, {"height", A_I32},
     {"taps", A_I32}},
    1,
    1,
    kBlock + 32,
    0,
    validate,
    grain,
    nchunks,
    ctas_per_sm,
    launch,
};

}  // namespace ecl

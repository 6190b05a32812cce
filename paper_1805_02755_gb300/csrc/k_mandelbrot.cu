// Mandelbrot escape counts (Sec. 5.3 Fig. 6 workload; Table 2: lws 256, no
// input buffer, out pattern 4:1).  This translation unit is compiled with
// -fmad=false and every operation is written with an explicit round-to-
// nearest intrinsic, so the FP32 arithmetic is exactly the correctly
// rounded sequence of the definition and the counts match a host
// evaluation bit for bit.
//
// Work-item g computes pixels 4g .. 4g+3 of the row-major image and writes
// them with one 128-bit store.  One chunk = one work-group; the CTA's 256
// compute threads stride over the work-group's work-items (plus one warp
// that claims chunks ahead).  The four pixels of a
// thread iterate interleaved so that four independent dependency chains
// are in flight.
#include <cuda_runtime.h>

#include "ecl_internal.h"
#include "sched.cuh"

namespace ecl {
namespace {

constexpr int kBlock = 256;

struct MandelbrotBody {
    static constexpr uint32_t kThreads = kBlock;
    struct Params {
        uint32_t *out;
        int64_t W, H;
        float x0, y0, dx, dy;
        int32_t max_iter;
        uint32_t lws;
    };
    Params p;

    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len)
    {
        return (uint32_t)len;
    }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t) { workgroup(p, off + t); }

    // Work-group wg of the view p: its lws work-items, 4 pixels each.
    static __device__ __forceinline__ void workgroup(const Params &p, uint64_t wg)
    {
        const uint64_t npx = (uint64_t)p.W * (uint64_t)p.H;
        const uint64_t wi_end = (wg + 1) * p.lws;
        for (uint64_t wi = wg * p.lws + threadIdx.x; wi < wi_end; wi += kBlock) {
            const uint64_t px0 = wi * 4;
            if (px0 >= npx) break;
            float cx[4], cy[4], x[4], y[4];
            uint32_t n[4];
            bool live[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t px = px0 + k;
                const uint64_t i = px % (uint64_t)p.W, j = px / (uint64_t)p.W;
                cx[k] = __fadd_rn(p.x0, __fmul_rn((float)i, p.dx));
                cy[k] = __fadd_rn(p.y0, __fmul_rn((float)j, p.dy));
                x[k] = 0.0f;
                y[k] = 0.0f;
                n[k] = 0;
                live[k] = px < npx;
            }
            for (int32_t it = 0; it < p.max_iter; ++it) {
                bool any = false;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float x2 = __fmul_rn(x[k], x[k]);
                    const float y2 = __fmul_rn(y[k], y[k]);
                    const bool go = live[k] && !(__fadd_rn(x2, y2) > 4.0f);
                    const float xt = __fadd_rn(__fsub_rn(x2, y2), cx[k]);
                    const float yt = __fadd_rn(__fmul_rn(__fmul_rn(2.0f, x[k]), y[k]), cy[k]);
                    x[k] = go ? xt : x[k];
                    y[k] = go ? yt : y[k];
                    n[k] += go ? 1u : 0u;
                    live[k] = go;
                    any |= go;
                }
                if (!any) break;
            }
            if (px0 + 3 < npx) {
                *reinterpret_cast<uint4 *>(p.out + px0) = make_uint4(n[0], n[1], n[2], n[3]);
            } else {
                for (int k = 0; k < 4; ++k)
                    if (px0 + k < npx) p.out[px0 + k] = n[k];
            }
        }
    }
};

__global__ void __launch_bounds__(kBlock + 32) k_mandelbrot(MandelbrotBody::Params prm, SchedArgs s)
{
    MandelbrotBody b{prm};
    drive_ws(s, b);
}

// ---------------------------------------------------------------- batches
// Many views of uneven size as one NDRange: view i owns work-groups
// [first_i, first_i + wgs_i) of lws 256; a work-group finds its view by
// binary search over `first` (ascending, first_0 = 0).  Mirrors
// ecl_mandelbrot_view in include/ecl.h.
struct MandelView {
    uint32_t *out;
    int32_t W, H;
    float x0, y0, dx, dy;
    int32_t max_iter;
    int32_t pad;
    int64_t first;
    int64_t wgs;
};
static_assert(sizeof(MandelView) == 56, "ecl_mandelbrot_view layout");

struct MandelBatchBody {
    static constexpr uint32_t kThreads = kBlock;
    struct Params {
        const MandelView *views;
        int32_t count;
        int64_t total;
    };
    Params p;

    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const int64_t wg = (int64_t)(off + t);
        if (wg >= p.total) return;
        int lo = 0, hi = p.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&p.views[mid].first) <= wg) lo = mid;
            else hi = mid - 1;
        }
        const MandelView &v = p.views[lo];
        const int64_t local = wg - v.first;
        // out of range, empty, or an output the 128-bit stores cannot use: skipped
        if (local < 0 || local >= v.wgs || v.W <= 0 || v.H <= 0 || ((uintptr_t)v.out & 15)) return;
        MandelbrotBody::Params q;
        q.out = v.out;
        q.W = v.W;
        q.H = v.H;
        q.x0 = v.x0;
        q.y0 = v.y0;
        q.dx = v.dx;
        q.dy = v.dy;
        q.max_iter = v.max_iter;
        q.lws = kBlock;
        MandelbrotBody::workgroup(q, (uint64_t)local);
    }
};

__global__ void __launch_bounds__(kBlock + 32) k_mandelbrot_batch(MandelBatchBody::Params prm, SchedArgs s)
{
    MandelBatchBody b{prm};
    drive_ws(s, b);
}

MandelbrotBody::Params params_of(const KArgs &a, uint32_t lws)
{
    MandelbrotBody::Params p;
    p.out = a.buf<uint32_t>(0);
    p.W = a.i32(1);
    p.H = a.i32(2);
    p.x0 = a.f32(3);
    p.y0 = a.f32(4);
    p.dx = a.f32(5);
    p.dy = a.f32(6);
    p.max_iter = a.i32(7);
    p.lws = lws;
    return p;
}

ecl_status validate(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    const int64_t W = a.i32(1), H = a.i32(2);
    if (W <= 0 || H <= 0) {
        err = "width and height must be positive";
        return ECL_ERR_ARG;
    }
    if (a.i32(7) < 0) {
        err = "max_iter must be >= 0";
        return ECL_ERR_ARG;
    }
    if (lws > 1024) {
        err = "lws must be <= 1024";
        return ECL_ERR_SIZE;
    }
    const uint64_t npx = (uint64_t)W * (uint64_t)H;
    if (a.bytes[0] < npx * 4) {
        err = "output buffer smaller than width*height uint32";
        return ECL_ERR_BUFFER;
    }
    if ((uintptr_t)a.ptr[0] % 16) {
        err = "output buffer must be 16-byte aligned";
        return ECL_ERR_BUFFER;
    }
    if (gws * 4 < npx) {
        err = "the NDRange (4 pixels per work-item) does not cover the image";
        return ECL_ERR_SIZE;
    }
    return ECL_OK;
}

uint64_t grain(const KArgs &, uint64_t, uint32_t) { return 1; }

uint32_t nchunks(const KArgs &a, uint64_t, uint32_t lws, uint64_t off, uint64_t len)
{
    return MandelbrotBody::nchunks(params_of(a, lws), off, len);
}

int ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mandelbrot, kBlock + 32, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ecl_status launch(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    k_mandelbrot<<<c.grid, kBlock + 32, 0, c.stream>>>(params_of(a, c.lws), s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

// ---- mandelbrot_batch: table of views, count, total work-groups
ecl_status v_batch(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    const int64_t count = a.i32(1), total = a.i64(2);
    if (count <= 0 || total <= 0) {
        err = "count and total must be positive";
        return ECL_ERR_ARG;
    }
    if (a.bytes[0] < (uint64_t)count * sizeof(MandelView) || (uintptr_t)a.ptr[0] % 16) {
        err = "the view table must hold count 16-byte aligned entries of 56 bytes";
        return ECL_ERR_BUFFER;
    }
    if (lws != kBlock) {
        err = "lws must be 256";
        return ECL_ERR_SIZE;
    }
    if (gws < (uint64_t)total * kBlock) {
        err = "the NDRange does not cover the views' work-groups";
        return ECL_ERR_SIZE;
    }
    return ECL_OK;
}

uint32_t nchunks_batch(const KArgs &, uint64_t, uint32_t, uint64_t, uint64_t len) { return (uint32_t)len; }

int batch_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mandelbrot_batch, kBlock + 32, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ecl_status l_batch(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    MandelBatchBody::Params p;
    p.views = a.buf<const MandelView>(0);
    p.count = a.i32(1);
    p.total = a.i64(2);
    k_mandelbrot_batch<<<c.grid, kBlock + 32, 0, c.stream>>>(p, s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

}  // namespace

extern const KernelDesc kMandelbrotBatch = {
    "mandelbrot_batch", 3, {{"views", A_BUF_IN}, {"count", A_I32}, {"total", A_I64}},
    1, 0, kBlock + 32, 0, v_batch, grain, nchunks_batch, batch_ctas_per_sm, l_batch,
};

extern const KernelDesc kMandelbrot = {
    "mandelbrot",
    8,
    {{"out", A_BUF_OUT}, {"width", A_I32}, {"height", A_I32}, {"x0", A_F32}, {"y0", A_F32},
     {"dx", A_F32}, {"dy", A_F32}, {"max_iter", A_I32}},
    4,
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

// Ray tracing (Sec. 7 "Ray" workload; Table 2: lws 128, scene buffer in,
// image out, out pattern 1:1, scene kept in local memory).  The paper's
// tracer and scenes are not available: this is a Whitted tracer over
// spheres and point lights (camera rays, hard shadows, Phong shading,
// mirror reflections up to a depth), the same definition as the oracle's.
//
// This translation unit is compiled with -fmad=false and every expression
// has the operand order of the definition, with IEEE division and square
// root, so colours and ray counts match a host evaluation bit for bit.
//
// Work-item g traces pixel g of the row-major W x H image and writes one
// float4 (r, g, b, rays traced).  One chunk = one work-group; a CTA is one
// warp that strides over the work-group's pixels.  Pixel costs vary by an
// order of magnitude (sky: one ray; reflective spheres: up to 16), so
// workers are kept small: with 128-thread CTAs the warps of a chunk waited
// for its most expensive pixels and the older CTAs on an SM out-ran the
// younger ones, 23-45% slower than a monolithic launch against 6-8% with
// one-warp CTAs (measured at 2048^2).  The scene (at most
// 128 spheres and 16 lights) is staged in shared memory once per CTA:
// sphere geometry as float4 (centre, r^2), materials separately.
#include <cuda_runtime.h>

#include "ecl_internal.h"
#include "sched.cuh"

namespace ecl {
namespace {

constexpr int kBlock = 32;
constexpr int kMaxSpheres = 128;
constexpr int kMaxLights = 16;
constexpr float kEps = 1e-3f;

struct RayParams {
    const float *scene;
    int32_t ns, nl;
    int64_t W, H;
    float ka, bg_r, bg_g, bg_b;
    int32_t max_depth;
    float4 *out;
    uint32_t lws;
};

struct RayScene {
    float4 geo[kMaxSpheres];     // centre x y z, r^2
    float4 mat[kMaxSpheres];     // colour r g b, reflectivity
    float4 shade[kMaxSpheres];   // kd, ks, log2 specular exponent, r
    float4 lpos[kMaxLights];     // position
    float4 lint[kMaxLights];     // intensity
};

// Nearest hit of the ray (o, d): index or -1, and t.  Spheres in index order,
// the first of equal t wins.
__device__ __forceinline__ int nearest(const RayScene &sc, int ns, float ox, float oy, float oz, float dx, float dy,
                                       float dz, float &t_out)
{
    int best = -1;
    float tb = 3.0e38f;
    for (int k = 0; k < ns; ++k) {
        const float4 g = sc.geo[k];
        const float ocx = ox - g.x, ocy = oy - g.y, ocz = oz - g.z;
        const float b = ocx * dx + ocy * dy + ocz * dz;
        const float c = (ocx * ocx + ocy * ocy + ocz * ocz) - g.w;
        const float disc = b * b - c;
        if (disc < 0.0f) continue;
        const float sq = sqrtf(disc);
        float t = -b - sq;
        if (!(t > kEps)) t = -b + sq;
        if (t > kEps && t < tb) {
            tb = t;
            best = k;
        }
    }
    t_out = tb;
    return best;
}

// Whether a sphere blocks (o, d) before dist; every sphere is tested (the
// answer does not depend on the order, and the work per shadow ray is fixed).
__device__ __forceinline__ bool blocked(const RayScene &sc, int ns, float ox, float oy, float oz, float dx, float dy,
                                        float dz, float dist)
{
    bool hit = false;
    for (int k = 0; k < ns; ++k) {
        const float4 g = sc.geo[k];
        const float ocx = ox - g.x, ocy = oy - g.y, ocz = oz - g.z;
        const float b = ocx * dx + ocy * dy + ocz * dz;
        const float c = (ocx * ocx + ocy * ocy + ocz * ocz) - g.w;
        const float disc = b * b - c;
        if (disc < 0.0f) continue;
        const float sq = sqrtf(disc);
        float t = -b - sq;
        if (!(t > kEps)) t = -b + sq;
        hit |= (t > kEps && t < dist);
    }
    return hit;
}

struct RayBody {
    using Params = RayParams;
    Params p;
    const RayScene *sc;

    static __host__ __device__ uint32_t nchunks(const Params &, uint64_t, uint64_t len) { return (uint32_t)len; }

    __device__ __forceinline__ float4 trace(int64_t i, int64_t j) const
    {
        const RayScene &s = *sc;
        const float inv = 1.0f / (float)p.H;
        const float u = (float)(2 * i + 1 - p.W) * inv;
        const float v = (float)(p.H - 2 * j - 1) * inv;
        const float len = sqrtf(u * u + v * v + 1.0f);
        float dx = u / len, dy = v / len, dz = -1.0f / len;
        float ox = 0.0f, oy = 0.0f, oz = 0.0f;
        float cr = 0.0f, cg = 0.0f, cb = 0.0f, w = 1.0f;
        int rays = 1;
        for (int depth = 0;; ++depth) {
            float t;
            const int k = nearest(s, p.ns, ox, oy, oz, dx, dy, dz, t);
            if (k < 0) {
                cr += w * p.bg_r;
                cg += w * p.bg_g;
                cb += w * p.bg_b;
                break;
            }
            const float4 g = s.geo[k], m = s.mat[k], sh = s.shade[k];
            const float px = ox + t * dx, py = oy + t * dy, pz = oz + t * dz;
            const float qx = px - g.x, qy = py - g.y, qz = pz - g.z;
            const float ql = sqrtf(qx * qx + qy * qy + qz * qz);
            const float nx = qx / ql, ny = qy / ql, nz = qz / ql;
            const float sox = px + nx * kEps, soy = py + ny * kEps, soz = pz + nz * kEps;
            float lr = p.ka * m.x, lg = p.ka * m.y, lb = p.ka * m.z;
            const int e = (int)sh.z;
            for (int l = 0; l < p.nl; ++l) {
                const float4 L = s.lpos[l], I = s.lint[l];
                float lx = L.x - px, ly = L.y - py, lz = L.z - pz;
                const float dist = sqrtf(lx * lx + ly * ly + lz * lz);
                lx = lx / dist;
                ly = ly / dist;
                lz = lz / dist;
                ++rays;
                if (blocked(s, p.ns, sox, soy, soz, lx, ly, lz, dist)) continue;
                const float ndl = nx * lx + ny * ly + nz * lz;
                if (!(ndl > 0.0f)) continue;
                const float dif = sh.x * ndl;
                lr += (dif * m.x) * I.x;
                lg += (dif * m.y) * I.y;
                lb += (dif * m.z) * I.z;
                const float rx = (2.0f * ndl) * nx - lx, ry = (2.0f * ndl) * ny - ly, rz = (2.0f * ndl) * nz - lz;
                const float rdv = -(rx * dx + ry * dy + rz * dz);
                if (rdv > 0.0f) {
                    float sp = rdv;
                    for (int q = 0; q < e; ++q) sp = sp * sp;
                    const float spec = sh.y * sp;
                    lr += spec * I.x;
                    lg += spec * I.y;
                    lb += spec * I.z;
                }
            }
            const float refl = m.w;
            if (refl > 0.0f && depth < p.max_depth) {
                const float wl = w * (1.0f - refl);
                cr += wl * lr;
                cg += wl * lg;
                cb += wl * lb;
                w = w * refl;
                const float dn = dx * nx + dy * ny + dz * nz;
                const float rx = dx - (2.0f * dn) * nx, ry = dy - (2.0f * dn) * ny, rz = dz - (2.0f * dn) * nz;
                const float rl = sqrtf(rx * rx + ry * ry + rz * rz);
                dx = rx / rl;
                dy = ry / rl;
                dz = rz / rl;
                ox = sox;
                oy = soy;
                oz = soz;
                ++rays;
            } else {
                cr += w * lr;
                cg += w * lg;
                cb += w * lb;
                break;
            }
        }
        return make_float4(cr, cg, cb, (float)rays);
    }

    __device__ __forceinline__ void run(uint64_t off, uint64_t, uint32_t t, uint32_t)
    {
        const int64_t npx = p.W * p.H;
        const int64_t g0 = (int64_t)(off + t) * p.lws;
        for (int64_t g = g0 + threadIdx.x; g < g0 + p.lws && g < npx; g += kBlock) {
            const int64_t j = g / p.W, i = g - j * p.W;
            p.out[g] = trace(i, j);
        }
    }
};

__global__ void __launch_bounds__(kBlock, 24) k_ray(RayParams prm, SchedArgs s)
{
    __shared__ RayScene sc;
    const float *lights = prm.scene + 12 * (int64_t)prm.ns;
    for (int k = threadIdx.x; k < prm.ns; k += blockDim.x) {
        const float *q = prm.scene + 12 * k;
        sc.geo[k] = make_float4(q[0], q[1], q[2], q[3] * q[3]);
        sc.mat[k] = make_float4(q[4], q[5], q[6], q[7]);
        sc.shade[k] = make_float4(q[8], q[9], q[10], q[3]);
    }
    for (int l = threadIdx.x; l < prm.nl; l += blockDim.x) {
        const float *q = lights + 8 * l;
        sc.lpos[l] = make_float4(q[0], q[1], q[2], 0.0f);
        sc.lint[l] = make_float4(q[4], q[5], q[6], 0.0f);
    }
    __syncthreads();
    RayBody b;
    b.p = prm;
    b.sc = &sc;
    drive(s, b);
}

RayParams params_of(const KArgs &a, uint32_t lws)
{
    RayParams p;
    p.scene = a.buf<const float>(0);
    p.ns = a.i32(1);
    p.nl = a.i32(2);
    p.W = a.i32(3);
    p.H = a.i32(4);
    p.ka = a.f32(5);
    p.bg_r = a.f32(6);
    p.bg_g = a.f32(7);
    p.bg_b = a.f32(8);
    p.max_depth = a.i32(9);
    p.out = a.buf<float4>(10);
    p.lws = lws;
    return p;
}

ecl_status validate(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err)
{
    const int64_t ns = a.i32(1), nl = a.i32(2), W = a.i32(3), H = a.i32(4), depth = a.i32(9);
    if (ns < 0 || ns > kMaxSpheres || nl < 0 || nl > kMaxLights) {
        err = "0..128 spheres and 0..16 lights";
        return ECL_ERR_ARG;
    }
    if (W <= 0 || H <= 0 || depth < 0 || depth > 64) {
        err = "width and height must be positive, max_depth 0..64";
        return ECL_ERR_ARG;
    }
    if (lws == 0 || lws > 1024) {
        err = "lws must be 1..1024";
        return ECL_ERR_SIZE;
    }
    if (gws < (uint64_t)W * (uint64_t)H) {
        err = "the NDRange (one pixel per work-item) does not cover the image";
        return ECL_ERR_SIZE;
    }
    if (a.bytes[0] < (uint64_t)(12 * ns + 8 * nl) * 4) {
        err = "scene buffer smaller than 12 floats per sphere + 8 per light";
        return ECL_ERR_BUFFER;
    }
    if (a.bytes[10] < (uint64_t)W * H * 16 || (uintptr_t)a.ptr[10] % 16) {
        err = "output must be a 16-byte aligned float4[width * height]";
        return ECL_ERR_BUFFER;
    }
    return ECL_OK;
}

uint64_t grain(const KArgs &, uint64_t, uint32_t) { return 1; }

uint32_t nchunks(const KArgs &a, uint64_t, uint32_t lws, uint64_t off, uint64_t len)
{
    return RayBody::nchunks(params_of(a, lws), off, len);
}

int ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ray, kBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

ecl_status launch(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err)
{
    k_ray<<<c.grid, kBlock, 0, c.stream>>>(params_of(a, c.lws), s);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(ce);
        return ECL_ERR_CUDA;
    }
    return ECL_OK;
}

}  // namespace

extern const KernelDesc kRay = {
    "ray",
    11,
    {{"scene", A_BUF_IN}, {"spheres", A_I32}, {"lights", A_I32}, {"width", A_I32}, {"height", A_I32},
     {"ambient", A_F32}, {"bg_r", A_F32}, {"bg_g", A_F32}, {"bg_b", A_F32}, {"max_depth", A_I32},
     {"out", A_BUF_OUT}},
    1,
    1,
    kBlock,
    0,
    validate,
    grain,
    nchunks,
    ctas_per_sm,
    launch,
};

}  // namespace ecl

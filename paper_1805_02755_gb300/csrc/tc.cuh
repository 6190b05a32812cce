// tcgen05 / TMA / mbarrier building blocks shared by the GEMM kernels
// (inline PTX for sm_103a), and the host-side tensor-map encoder.
//
// Operand tiles are K-major bf16 with 128-byte rows (64 elements) in the
// 128-byte swizzled layout TMA writes; 8-row groups lie 1024 bytes apart.
// Every mbarrier wait is bounded in time: a wait that gives up sets the
// CTA's error word and the queue's ECL_ERR_TIMEOUT.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "ecl_internal.h"
#include "sched.cuh"

namespace ecl {
namespace tc {

constexpr int kBoxK = 64;                    // K extent of one TMA box (128 bytes of bf16)
constexpr uint64_t kWaitNs = 2000000000ull;  // a wait gives up after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false when it gave up (or another role already did).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile uint32_t *err,
                                          unsigned int *gerr)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtime();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 0) {
            if (*err) return false;
            if (gtime() - t0 > kWaitNs) {
                *err = 1;
                atomicExch(gerr, (unsigned int)ECL_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major tile with 128-byte rows, 128B
// swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3ffffu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: A = B = BF16, D = FP32,
// both operands K-major, M x N tile.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) = A (shared) * B (shared) [+ D when accumulate != 0]; issued by one thread.
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}


// ---------------------------------------------------------------- host side
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}

inline bool make_map(CUtensorMap *m, const void *base, int64_t rows, int64_t K, int box_rows, std::string &err)
{
    auto fn = encode_fn();
    if (!fn) {
        err = "cuTensorMapEncodeTiled unavailable";
        return false;
    }
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBoxK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}

// Output-tile order of the work-group ids: column groups of W tile columns,
// each group's tiles row by row (W tiles per row, the last group narrower
// when W does not divide the tile columns).  A wave of `ctas` concurrent
// tiles then covers about ctas / W tile rows and W tile columns, so it reads
// ctas / W A strips and W Bt strips instead of one or two tile rows' A
// strips and every Bt strip.
struct TileOrder {
    int64_t tm, tn, w;  // tile rows, tile columns, group width
};

__host__ __device__ __forceinline__ void tile_at(const TileOrder &o, int64_t t, int64_t &mt, int64_t &nt)
{
    const int64_t gsz = o.tm * o.w;
    const int64_t g = t / gsz;
    const int64_t r = t - g * gsz;
    const int64_t rest = o.tn - g * o.w;
    const int64_t wg = rest < o.w ? rest : o.w;
    mt = r / wg;
    nt = g * o.w + (r - (r / wg) * wg);
}

// The group width that minimises one wave's strip bytes W b + (ctas / W) a
// (A and Bt strips of a_bytes and b_bytes): W = sqrt(ctas a / b).  Measured
// at M = N = K = 8192 (152 CTAs, 128 x 256 tiles, W = 9): DRAM reads of the
// plain BF16 GEMM 2.06 -> 1.27 GB and 0.785 -> 0.746 ms against the
// row-major order; wider groups sized for a group's Bt strips to stay in L2
// across waves (W = 17, 24) read 1.46 and 1.53 GB.
inline TileOrder tile_order(int64_t tm, int64_t tn, int64_t ctas, double a_bytes, double b_bytes)
{
    const int64_t w = (int64_t)(std::sqrt((double)ctas * a_bytes / b_bytes) + 0.5);
    return TileOrder{tm, tn, w < 1 ? 1 : (w > tn ? tn : w)};
}

}  // namespace tc
}  // namespace ecl

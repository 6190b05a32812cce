// Internal interfaces between the host runtime (runtime.cu) and the kernel
// translation units.  Not part of the public ABI (include/ecl.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <string>

#include "../../include/ecl.h"

namespace ecl {

// ------------------------------------------------------------------ device
// One package of the plan: a contiguous work-group range and the number of
// chunks the kernel splits it into (the unit a CTA of a device claims).
struct Pkg {
    uint64_t off;
    uint64_t len;
    uint32_t nchunks;
    uint32_t pad;
};

// Per-package record written on the device.  The first 48 bytes mirror
// ecl_pkg_stat; `done` counts finished chunks so that the CTA finishing the
// last chunk stamps t1.
struct PkgRec {
    uint64_t off, len, t0, t1;
    uint32_t pkg, device, cta, smid;
    uint32_t done, nchunks;
};

// Per-device claim word: high 32 bits = package slot + 1 (0 = none yet,
// 0xffffffff = finished), low 32 bits = chunk claims made on that slot.
struct DevState {
    unsigned long long word;
    unsigned int fetches;  // packages this device has taken (Static)
    unsigned int pad;
};

// Queue header.  Zero at allocation; the last CTA of every run puts the
// cursor, the device words and the exit count back to zero, so a run needs
// no memset beforehand.  `error` is sticky until the host clears it.
struct Queue {
    unsigned long long cursor;     // next package index (table modes)
    unsigned long long consumed;   // units handed out (device-side HGuided)
    unsigned int exit_count;
    unsigned int error;            // 0 or ECL_ERR_TIMEOUT
    unsigned long long error_info; // CTA id | spin count of the wait that gave up
    unsigned long long last_npkg;  // packages handed out by the last run
};

enum Mode : uint32_t {
    MODE_STATIC = 0,    // device d takes table[d] once
    MODE_QUEUE = 1,     // packages table[0..npkg) in order, one atomicAdd each
    MODE_HGUIDED = 2,   // HGuided with unequal powers: sizes cut on the device
    MODE_MONO = 3       // no queue: CTA b computes chunk b of the whole range
};

constexpr uint32_t kSlotDone = 0xffffffffu;

// Everything a persistent kernel needs from the scheduler, by value.
struct SchedArgs {
    Pkg *table;            // npkg entries (written by the device in MODE_HGUIDED)
    Queue *q;
    DevState *dev;         // D entries
    PkgRec *rec;           // one per package
    ecl_worker_stat *wst;  // one per CTA
    uint32_t *coverage;    // optional per-work-group counters
    uint64_t G;            // work-groups
    uint64_t grain;        // work-groups per scheduling unit
    uint64_t units;        // ceil(G / grain)
    uint64_t table_cap;    // capacity of table/rec
    uint32_t npkg;         // packages in the table (table modes)
    uint32_t mode;
    uint32_t D, C;
    uint32_t mono_nchunks; // MODE_MONO: chunks of the whole range (= grid)
    uint32_t spin_limit;   // iterations of a bounded wait before giving up
    uint32_t withhold;     // fault injection: fetchers do not publish packages
    uint32_t records;      // MODE_MONO run for Static over one device: keep the
                           // package record (table entry 0) and one worker record per CTA
    // HGuided with unequal powers (MODE_HGUIDED)
    double hg_k;
    double hg_sum_p;
    const double *hg_p;    // D powers (device memory)
    const uint32_t *hg_min;// D minimum sizes in units (device memory)
};

// ------------------------------------------------------------------ host
enum ArgKind : uint32_t { A_BUF_IN, A_BUF_OUT, A_BUF_OUT_OPT, A_I32, A_I64, A_F32 };

struct ArgSpec {
    const char *name;
    ArgKind kind;
};

// Resolved kernel arguments: device address and size for buffers, raw bits
// for scalars.
struct KArgs {
    int n = 0;
    void *ptr[16] = {};
    size_t bytes[16] = {};
    uint64_t raw[16] = {};
    int i32(int i) const { return (int)(int32_t)(uint32_t)raw[i]; }
    long long i64(int i) const { return (long long)raw[i]; }
    float f32(int i) const {
        uint32_t b = (uint32_t)raw[i];
        float f;
        memcpy(&f, &b, 4);
        return f;
    }
    template <class T> T *buf(int i) const { return (T *)ptr[i]; }
};

struct Workspace;  // engine-owned scratch (runtime.cu)

struct LaunchCtx {
    cudaStream_t stream;
    uint32_t lws;
    uint64_t gws;
    uint32_t grid;
    Workspace *ws;
    // ecl_engine_kernel_events: a launcher that follows its main kernel with
    // another (the binomial's greeks pass) records mark_end right after the
    // main kernel and sets *marked; otherwise the run records it after the
    // launcher returns
    cudaEvent_t mark_end = nullptr;
    bool *marked = nullptr;
    // the same for the begin mark, recorded before the launcher; a launcher
    // with a pass before its main kernel (the split GEMMs' operand split)
    // records it again after that pass (the later record counts)
    cudaEvent_t mark_begin = nullptr;
};

// Records c.mark_begin on the launch's stream before a program's main kernel.
inline void mark_main_begin(const LaunchCtx &c)
{
    if (c.mark_begin) cudaEventRecord(c.mark_begin, c.stream);
}

// Records c.mark_end on the launch's stream after a program's main kernel.
inline void mark_main_end(const LaunchCtx &c)
{
    if (c.mark_end && c.marked) {
        cudaEventRecord(c.mark_end, c.stream);
        *c.marked = true;
    }
}

struct KernelDesc {
    const char *name;
    int nargs;
    ArgSpec args[12];
    uint32_t out_outs;     // output pattern outs : work_items; work_items 0
    uint32_t out_wis;      //   means "lws" (one output per work-group)
    int block;             // threads per CTA
    int default_D;         // 0 = one device per resident CTA
    // Checks sizes; fills err and returns a status.
    ecl_status (*validate)(const KArgs &a, uint64_t gws, uint32_t lws, std::string &err);
    // Work-groups per scheduling unit (1 except the row-tiled GEMM).
    uint64_t (*grain)(const KArgs &a, uint64_t gws, uint32_t lws);
    // Chunks a package [off, off+len) is split into.
    uint32_t (*nchunks)(const KArgs &a, uint64_t gws, uint32_t lws, uint64_t off, uint64_t len);
    // Resident CTAs per SM of the persistent kernel.
    int (*ctas_per_sm)();
    // Launches the persistent (or monolithic) kernel.
    ecl_status (*launch)(const KArgs &a, const SchedArgs &s, const LaunchCtx &c, std::string &err);
    // The kernel runs its own claim loop instead of drive/drive_ws (the
    // tcgen05 GEMMs): Static over one device then stays on the queue.
    bool own_claims;
};

const KernelDesc *find_kernel(const char *name);

// Engine-owned scratch memory, grown on demand (device memory).  Fresh memory
// is zeroed.  A kernel that keeps counters in it passes itself as `owner`:
// when the previous user was a different kernel the memory is zeroed on
// `stream` first, so counters start at zero; kernels reset their counters
// before they exit.
void *workspace_get(Workspace *ws, size_t bytes, std::string &err, const void *owner = nullptr,
                    cudaStream_t stream = 0);

// Raises kernel `fn`'s dynamic shared-memory limit to `bytes` on the current
// device, once per device: the attribute belongs to the function on one
// device, so a process with engines on several GPUs sets it on each.  `done`
// holds one bit per device ordinal (ordinals from 64 up are set every call).
// Setting it twice is harmless, so host threads that race here need no lock.
// Returns false, with the CUDA error cleared, when the driver refuses.
bool smem_limit_once(const void *fn, int bytes, std::atomic<unsigned long long> &done);

}  // namespace ecl

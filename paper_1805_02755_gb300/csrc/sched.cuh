// Device side of the package scheduler: the persistent-CTA driver that every
// kernel body runs under.
//
// The paper's devices (Sec. 5.1: one host thread per OpenCL device, the
// Scheduler thread handing out packages) become groups of C persistent CTAs.
// A package taken by a device is split into chunks; the device's CTAs claim
// chunks through one 64-bit word per device.  The CTA whose claim lands
// exactly one past the last chunk is the one that fetches the device's next
// package (Static: its own range once; Dynamic/HGuided: the next entry of
// the queue).  Other CTAs of the device that overshoot wait, with a bounded
// spin, for the new package to be published.  Nothing else waits, so the
// queue cannot deadlock: the CTA being waited for is running.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ecl_internal.h"

namespace ecl {

__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smid()
{
    uint32_t s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

struct Claim {
    uint64_t off, len;   // package range (work-groups)
    uint32_t pkg;        // package index
    uint32_t t_begin;    // chunks [t_begin, t_end) of nchunks
    uint32_t t_end;
    uint32_t nchunks;
    uint32_t done;       // no more work for this CTA
    uint32_t last;       // (exit) this CTA is the last to leave
};

// HGuided packet size of device d for G_r pending units (Sec. 5.3 equation),
// evaluated in double in the order (G_r * P_i) / ((k * n) * sum P), raised
// to the device minimum and clipped to G_r.
__device__ __forceinline__ uint64_t hguided_units(const SchedArgs &s, uint32_t d, uint64_t gr)
{
    const double q = ((double)gr * s.hg_p[d]) / ((s.hg_k * (double)s.D) * s.hg_sum_p);
    uint64_t sz = (uint64_t)floor(q);
    const uint64_t mn = s.hg_min[d];
    if (sz < mn) sz = mn;
    if (sz > gr) sz = gr;
    return sz;
}

// Takes the next package for device d; returns its slot or -1 when none is
// left.  Called by one thread of one CTA of the device at a time.
template <class Body>
__device__ int64_t fetch_package(const SchedArgs &s, const typename Body::Params &bp, uint32_t d)
{
    int64_t p = -1;
    if (s.mode == MODE_STATIC) {
        if (atomicAdd(&s.dev[d].fetches, 1u) == 0u) p = d;
    } else if (s.mode == MODE_QUEUE) {
        const unsigned long long i = atomicAdd(&s.q->cursor, 1ull);
        if (i < s.npkg) p = (int64_t)i;
    } else {  // MODE_HGUIDED: cut the package from the pending units
        unsigned long long used = ld_relaxed(&s.q->consumed);
        while (used < s.units) {
            const uint64_t gr = s.units - used;
            const uint64_t sz = hguided_units(s, d, gr);
            const unsigned long long seen = atomicCAS(&s.q->consumed, used, used + sz);
            if (seen == used) {
                const uint64_t off = used * s.grain;
                uint64_t end = (used + sz) * s.grain;
                if (end > s.G) end = s.G;
                const unsigned long long i = atomicAdd(&s.q->cursor, 1ull);
                if (i >= s.table_cap) break;  // cannot happen: every package has >= 1 unit
                Pkg pk;
                pk.off = off;
                pk.len = end - off;
                pk.nchunks = Body::nchunks(bp, off, end - off);
                pk.pad = 0;
                s.table[i] = pk;
                p = (int64_t)i;
                break;
            }
            used = seen;
        }
    }
    if (p >= 0) {
        const Pkg pk = s.table[p];
        PkgRec r;
        r.off = pk.off;
        r.len = pk.len;
        r.t0 = gtime();
        r.t1 = 0;
        r.pkg = (uint32_t)p;
        r.device = d;
        r.cta = blockIdx.x;
        r.smid = smid();
        r.done = 0;
        r.nchunks = pk.nchunks;
        s.rec[p] = r;
        __threadfence();
    }
    return p;
}

// The package slot a claimer last found in its device's chunk word, with
// that package's table entry.  A package's entry is written before its slot
// is published and not changed during the run, so a claim that finds the
// same slot again needs neither the acquire fence nor the table read.
struct ClaimCache {
    uint32_t slot;  // 0: none yet
    Pkg pk;
};

// cc: the claimer's cache (kept by the one thread that claims for the CTA,
// in shared memory), or nullptr: every claim fences and reads the table (the
// warp-specialised and GEMM drivers, where a cache held by the claiming
// lane measured more registers for the whole kernel: the NBody energy 56 ->
// 65, one CTA per SM fewer).
template <class Body>
__device__ Claim claim_chunks(const SchedArgs &s, const typename Body::Params &bp, uint32_t d,
                              ClaimCache *cc = nullptr)
{
    Claim c{};
    if (s.C == 1) {
        const int64_t p = fetch_package<Body>(s, bp, d);
        if (p < 0) {
            c.done = 1;
            return c;
        }
        const Pkg pk = s.table[p];
        c.off = pk.off;
        c.len = pk.len;
        c.pkg = (uint32_t)p;
        c.t_begin = 0;
        c.t_end = pk.nchunks;
        c.nchunks = pk.nchunks;
        return c;
    }
    if (s.mode == MODE_STATIC && !s.coverage) {
        // Static: device d's package is table entry d, fixed before the launch,
        // so a claim is one atomic on the device's chunk counter and no CTA
        // waits for an election.  The claimer of chunk 0 stamps the record (t1
        // is a running maximum of chunk end times, so it is left alone).
        if (d >= s.npkg) {
            c.done = 1;
            return c;
        }
        const Pkg pk = s.table[d];
        const uint32_t t = (uint32_t)atomicAdd(&s.dev[d].word, 1ull);
        if (t >= pk.nchunks) {
            c.done = 1;
            return c;
        }
        if (t == 0) {
            PkgRec *r = s.rec + d;
            r->off = pk.off;
            r->len = pk.len;
            r->t0 = gtime();
            r->pkg = d;
            r->device = d;
            r->cta = blockIdx.x;
            r->smid = smid();
            r->nchunks = pk.nchunks;
        }
        c.off = pk.off;
        c.len = pk.len;
        c.pkg = d;
        c.t_begin = t;
        c.t_end = t + 1;
        c.nchunks = pk.nchunks;
        return c;
    }
    uint32_t spins = 0;
    for (;;) {
        const unsigned long long w = atomicAdd(&s.dev[d].word, 1ull);
        const uint32_t slot = (uint32_t)(w >> 32);
        const uint32_t t = (uint32_t)w;
        if (slot == kSlotDone) {
            c.done = 1;
            return c;
        }
        Pkg pk{};
        if (!cc) {
            __threadfence();
            if (slot) pk = s.table[slot - 1];
        } else if (slot == cc->slot) {
            pk = cc->pk;
        } else {
            // acquire: pairs with the publisher's fence before its exchange,
            // so the new package's table entry is read after the slot
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            if (slot) pk = s.table[slot - 1];
            cc->slot = slot;
            cc->pk = pk;
        }
        const uint32_t nch = slot ? pk.nchunks : 0u;
        if (t < nch) {
            c.off = pk.off;
            c.len = pk.len;
            c.pkg = slot - 1;
            c.t_begin = t;
            c.t_end = t + 1;
            c.nchunks = nch;
            return c;
        }
        if (t == nch) {  // this CTA fetches the device's next package
            const int64_t p = fetch_package<Body>(s, bp, d);
            if (s.withhold) {  // fault injection: never publish; the others time out
                c.done = 1;
                return c;
            }
            if (p < 0) {
                atomicExch(&s.dev[d].word, (unsigned long long)kSlotDone << 32);
                c.done = 1;
                return c;
            }
            atomicExch(&s.dev[d].word, (unsigned long long)(p + 1) << 32);
            continue;
        }
        // another CTA of the device is fetching: wait for the new slot, with
        // a doubling back-off (a fetch takes a few microseconds, and up to C - 1
        // CTAs of the device poll meanwhile)
        uint32_t ns = 128;
        while ((uint32_t)(ld_relaxed(&s.dev[d].word) >> 32) == slot) {
            __nanosleep(ns);
            if (ns < 2048) ns <<= 1;
            if (++spins > s.spin_limit) {
                atomicExch(&s.q->error, (unsigned int)ECL_ERR_TIMEOUT);
                atomicExch(&s.q->error_info, ((unsigned long long)blockIdx.x << 32) | spins);
                c.done = 1;
                return c;
            }
        }
    }
}

// Chunk accounting after a CTA finished chunks [t_begin, t_end) of c.pkg:
// returns true when this completed the package (then t1 is stamped).
__device__ __forceinline__ bool finish_chunks(const SchedArgs &s, uint32_t pkg, uint32_t n, uint32_t nchunks,
                                              uint64_t te)
{
    const uint32_t prev = (s.C == 1) ? 0u : atomicAdd(&s.rec[pkg].done, n);
    const bool finished = (prev + n == nchunks);
    if (finished) {
        s.rec[pkg].t1 = te;
        s.rec[pkg].done = nchunks;
    }
    return finished;
}

// The same accounting without waiting for an atomic's result: t1 becomes
// the latest chunk end (a reduction the CTA does not wait for).  Used when
// no coverage is requested, so nobody needs to know which CTA finished the
// package.
__device__ __forceinline__ void finish_chunks_async(const SchedArgs &s, uint32_t pkg, uint64_t te)
{
    if (s.C == 1)
        s.rec[pkg].t1 = te;
    else
        atomicMax((unsigned long long *)&s.rec[pkg].t1, (unsigned long long)te);
}

// End of a persistent CTA (all threads call it): writes the per-CTA record,
// and the last CTA to leave puts the queue back to its initial state.
__device__ __forceinline__ void exit_protocol(const SchedArgs &s, uint32_t d, uint64_t t_first, uint64_t t_last,
                                              uint64_t busy, uint32_t nchunks_done, uint32_t *flag)
{
    if (threadIdx.x == 0) {
        ecl_worker_stat w;
        w.t_first_ns = t_first;
        w.t_last_ns = t_last;
        w.busy_ns = busy;
        w.cta = blockIdx.x;
        w.device = d;
        w.smid = smid();
        w.chunks = nchunks_done;
        s.wst[blockIdx.x] = w;
        __threadfence();
        const unsigned int ticket = atomicAdd(&s.q->exit_count, 1u);
        *flag = (ticket == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (*flag) {
        __threadfence();
        for (uint32_t i = threadIdx.x; i < s.D; i += blockDim.x) {
            s.dev[i].word = 0ull;
            s.dev[i].fetches = 0u;
        }
        if (threadIdx.x == 0) {
            s.q->last_npkg = s.q->cursor;
            s.q->cursor = 0ull;
            s.q->consumed = 0ull;
            s.q->exit_count = 0u;
        }
        __threadfence();
    }
}

// Barrier among the compute warps only (warp-specialised driver).
__device__ __forceinline__ void body_sync(uint32_t nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Records of a monolithic run of Static over one device (s.records): CTA b
// ran chunk b of the single package, table entry 0.  The package's t0 is
// chunk 0's start and t1 the running maximum of chunk end times (as in the
// persistent Static path); every CTA writes its worker record.  With
// coverage the last CTA to finish (a ticket on the queue's exit counter,
// zero at the start of every run) counts the package's work-groups.  Called
// by all NT threads that ran the body; WS selects the compute-warp barrier
// of the warp-specialised driver.
template <bool WS>
__device__ __forceinline__ void grid_records(const SchedArgs &s, uint64_t ts, uint32_t *flag, uint32_t nt)
{
    if (WS) body_sync(nt);
    else __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t te = gtime();
        ecl_worker_stat w;
        w.t_first_ns = ts;
        w.t_last_ns = te;
        w.busy_ns = te - ts;
        w.cta = blockIdx.x;
        w.device = 0;
        w.smid = smid();
        w.chunks = 1;
        s.wst[blockIdx.x] = w;
        PkgRec *r = s.rec;
        if (blockIdx.x == 0) {
            r->off = 0;
            r->len = s.G;
            r->t0 = ts;
            r->pkg = 0;
            r->device = 0;
            r->cta = 0;
            r->smid = w.smid;
            r->nchunks = s.mono_nchunks;
        }
        atomicMax((unsigned long long *)&r->t1, (unsigned long long)te);
        *flag = 0;
        if (s.coverage) {
            __threadfence();
            if (atomicAdd(&s.q->exit_count, 1u) == gridDim.x - 1) {
                s.q->exit_count = 0u;
                *flag = 1;
            }
        }
    }
    if (s.coverage) {
        if (WS) body_sync(nt);
        else __syncthreads();
        if (*flag)
            for (uint64_t w = threadIdx.x; w < s.G; w += nt) atomicAdd(&s.coverage[w], 1u);
    }
}

// The persistent driver.  Body must provide
//   struct Params;                                   (kernel arguments)
//   static __host__ __device__ uint32_t nchunks(const Params&, off, len);
//   __device__ void run(off, len, t, nchunks);        (all threads, uniform)
template <class Body>
__device__ __forceinline__ void drive(const SchedArgs &s, Body &body)
{
    __shared__ Claim sc;
    __shared__ ClaimCache cache;  // thread 0's, in shared memory: no registers across the body
    if (threadIdx.x == 0) cache.slot = 0;
    // MODE_MONO: the whole range is one package, CTA b = chunk b.  It goes
    // through the same call of body.run, so that a large body is inlined once.
    const bool mono = s.mode == MODE_MONO;
    const uint32_t d = mono ? 0u : blockIdx.x / s.C;
    uint64_t t_first = 0, t_last = 0, busy = 0;
    uint32_t nchunks_done = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            if (mono) {
                Claim m{};
                m.len = s.G;
                m.t_begin = blockIdx.x;
                m.t_end = blockIdx.x + 1;
                m.nchunks = s.mono_nchunks;
                sc = m;
            } else {
                sc = claim_chunks<Body>(s, body.p, d, &cache);
            }
        }
        __syncthreads();
        const Claim c = sc;
        __syncthreads();
        if (c.done) break;
        uint64_t ts = 0;
        if (threadIdx.x == 0) ts = gtime();
        for (uint32_t t = c.t_begin; t < c.t_end; ++t) body.run(c.off, c.len, t, c.nchunks);
        if (mono) {
            if (s.records) grid_records<false>(s, ts, &sc.last, blockDim.x);
            return;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint64_t te = gtime();
            if (!t_first) t_first = ts;
            t_last = te;
            busy += te - ts;
            nchunks_done += c.t_end - c.t_begin;
            const uint32_t n = c.t_end - c.t_begin;
            if (s.coverage) {
                sc.last = finish_chunks(s, c.pkg, n, c.nchunks, te) ? 1u : 0u;
            } else {
                // nobody needs to know which CTA finished the package: t1
                // becomes the latest chunk end without waiting for an atomic
                finish_chunks_async(s, c.pkg, te);
                sc.last = 0u;
            }
        }
        if (s.coverage) {  // debug: count every work-group of a finished package
            __syncthreads();
            if (sc.last)
                for (uint64_t w = c.off + threadIdx.x; w < c.off + c.len; w += blockDim.x)
                    atomicAdd(&s.coverage[w], 1u);
            __syncthreads();
        }
    }
    exit_protocol(s, d, t_first, t_last, busy, nchunks_done, &sc.last);
}

// ------------------------------------------------------------------ mbarrier helpers
__device__ __forceinline__ uint32_t sh_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void sbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sh_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void sbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sh_addr(bar)) : "memory");
}

// Bounded wait on phase `parity`; false (and the queue's error word set)
// when it gave up after about two seconds.  The thread waits suspended in
// try_wait, which returns when the phase completes or after the suspend-time
// hint (1 ms), so a waiting warp takes no issue slots from the compute warps
// (the scheduler warp waits out a whole chunk here).  Measured against polls
// separated by a doubling nanosleep back-off: Mandelbrot 53.6 -> 51.6 us, the
// Gaussian 0.2373 -> 0.2355 ms, the NBody energy 0.7253 -> 0.7232 ms.
constexpr uint32_t kWaitHintNs = 1000000;

__device__ __forceinline__ bool sbar_wait(uint64_t *bar, uint32_t parity, unsigned int *gerr)
{
    uint64_t t0 = 0;
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            "selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(sh_addr(bar)), "r"(parity), "r"(kWaitHintNs)
            : "memory");
        if (ok) return true;
        const uint64_t now = gtime();
        if (!t0) t0 = now;
        if (now - t0 > 2000000000ull) {
            atomicExch(gerr, (unsigned int)ECL_ERR_TIMEOUT);
            return false;
        }
    }
}

// Warp-specialised persistent driver: the CTA has Body::kThreads compute
// threads plus one scheduler warp.  The scheduler warp claims chunks into a
// two-slot ring ahead of the compute warps, so the atomic round trips of a
// claim (and a device's election to fetch its next package) overlap the
// previous chunk's work.  Bodies synchronise with body_sync(kThreads), never
// __syncthreads.  Every wait is bounded; a wait that gives up sets the queue's
// error word and ends the CTA's work.
// FORM selects the launch forms compiled into the kernel: DRIVE_ANY both
// (chosen by s.mode at run time), DRIVE_MONO the monolithic launch only,
// DRIVE_QUEUE the persistent queue only.  A kernel with a large body can be
// instantiated once per form so that each holds a single inlined copy of the
// body, with a register allocation of its own (measured on the NBody force:
// the claim-loop copy then executed 5% fewer instructions).
enum DriveForm { DRIVE_ANY = 0, DRIVE_MONO = 1, DRIVE_QUEUE = 2 };

template <class Body, int FORM = DRIVE_ANY>
__device__ __forceinline__ void drive_ws(const SchedArgs &s, Body &body)
{
    constexpr uint32_t NC = Body::kThreads;
    __shared__ Claim ring[2];
    __shared__ uint64_t full[2], empty[2];
    __shared__ uint32_t flag;
    if (FORM == DRIVE_MONO || (FORM == DRIVE_ANY && s.mode == MODE_MONO)) {
        // the whole range is one package, CTA b = chunk b
        if (threadIdx.x < NC) {
            uint64_t ts = 0;
            if (s.records && threadIdx.x == 0) ts = gtime();
            body.run(0, s.G, blockIdx.x, s.mono_nchunks);
            if (s.records) grid_records<true>(s, ts, &flag, NC);
        }
        return;
    }
    unsigned int *gerr = &s.q->error;
    const uint32_t d = blockIdx.x / s.C;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            sbar_init(&full[i], 1);
            sbar_init(&empty[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // Loop state of thread 0 lives in shared memory and the claim is read from
    // its ring slot when needed: registers held across body.run would come out
    // of the body's budget (measured: a register copy of the claim and 64-bit
    // timers cost a force run a quarter more instructions).
    __shared__ uint64_t st_ts, st_first, st_last, st_busy;
    __shared__ uint32_t st_n;
    if (threadIdx.x == 0) {
        st_first = st_last = st_busy = 0;
        st_n = 0;
    }
    __syncthreads();
    if (threadIdx.x >= NC) {
        if (threadIdx.x == NC) {  // scheduler: lane 0 of the last warp
            // Claiming a chunk ahead fixes which CTA takes it before anyone
            // knows which CTA will be free first.  Under Static (direct
            // claims on the device's chunk counter), when fewer chunks are
            // left in the device's package than it has CTAs, the scheduler
            // claims only after the chunk it handed out last is done (lazy),
            // so the package's tail goes to the CTAs that finish first.
            const bool counted = s.mode == MODE_STATIC && s.C > 1 && !s.coverage;
            uint32_t nch = 0;
            for (uint32_t i = 0;; ++i) {
                const uint32_t r = i & 1;
                if (counted && i > 0) {
                    const unsigned long long claimed = ld_relaxed(&s.dev[d].word);
                    const bool lazy = claimed >= nch || nch - claimed < s.C;
                    if (lazy && !sbar_wait(&empty[r ^ 1], ((i - 1) >> 1) & 1, gerr)) break;
                }
                if (!sbar_wait(&empty[r], ((i >> 1) & 1) ^ 1, gerr)) break;
                Claim c = (*(volatile unsigned int *)gerr) ? Claim{} : claim_chunks<Body>(s, body.p, d);
                if (*(volatile unsigned int *)gerr) c.done = 1;
                nch = c.nchunks;
                ring[r] = c;
                sbar_arrive(&full[r]);
                if (c.done) break;
            }
        }
    } else {
        for (uint32_t i = 0;; ++i) {
            const uint32_t r = i & 1;
            if (threadIdx.x == 0) flag = sbar_wait(&full[r], (i >> 1) & 1, gerr) ? 0u : 1u;
            body_sync(NC);
            if (flag || ring[r].done) break;
            if (threadIdx.x == 0) st_ts = gtime();
            const uint32_t tb = ring[r].t_begin, tz = ring[r].t_end;
            for (uint32_t t = tb; t < tz; ++t) body.run(ring[r].off, ring[r].len, t, ring[r].nchunks);
            body_sync(NC);  // all compute threads are done with the chunk
            if (threadIdx.x == 0) {
                const uint64_t te = gtime();
                if (!st_first) st_first = st_ts;
                st_last = te;
                st_busy += te - st_ts;
                st_n += tz - tb;
                if (!s.coverage) {
                    finish_chunks_async(s, ring[r].pkg, te);
                    sbar_arrive(&empty[r]);  // the slot is no longer read
                    flag = 0;
                } else {
                    flag = finish_chunks(s, ring[r].pkg, tz - tb, ring[r].nchunks, te) ? 1u : 0u;
                }
            }
            if (s.coverage) {  // debug: count every work-group of a finished package
                body_sync(NC);
                if (flag) {
                    const uint64_t o = ring[r].off, z = ring[r].off + ring[r].len;
                    for (uint64_t w = o + threadIdx.x; w < z; w += NC) atomicAdd(&s.coverage[w], 1u);
                }
                body_sync(NC);
                if (threadIdx.x == 0) {
                    flag = 0;
                    sbar_arrive(&empty[r]);
                }
            }
        }
    }
    __syncthreads();
    exit_protocol(s, d, st_first, st_last, st_busy, st_n, &flag);
}

}  // namespace ecl

// Host runtime behind include/ecl.h: engines, programs, the package planner
// (Static / Static rev / Dynamic / HGuided of Sec. 5.3) and the run path.
//
// A run is validated and planned on the host, then executes as ONE
// persistent launch on the engine's stream.  The package table is uploaded
// only when the plan changes, and the device queue resets itself at the end
// of every run, so repeated runs of one plan cost exactly one launch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "ecl_internal.h"

using namespace ecl;

namespace ecl {
struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
    const void *owner = nullptr;  // kernel whose counters the memory holds
};

bool smem_limit_once(const void *fn, int bytes, std::atomic<unsigned long long> &done)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return true;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    done.fetch_or(bit, std::memory_order_release);
    return true;
}

void *workspace_get(Workspace *ws, size_t bytes, std::string &err, const void *owner, cudaStream_t stream)
{
    if (ws->bytes >= bytes) {
        if (owner && owner != ws->owner) {  // another kernel's leftovers: zero before use
            cudaError_t ce = cudaMemsetAsync(ws->ptr, 0, bytes, stream);
            if (ce != cudaSuccess) {
                err = std::string("cudaMemsetAsync(workspace): ") + cudaGetErrorString(ce);
                return nullptr;
            }
        }
        ws->owner = owner;
        return ws->ptr;
    }
    if (ws->ptr) cudaFree(ws->ptr);
    ws->ptr = nullptr;
    ws->bytes = 0;
    ws->owner = nullptr;
    cudaError_t ce = cudaMalloc(&ws->ptr, bytes);
    if (ce != cudaSuccess) {
        err = std::string("cudaMalloc(workspace): ") + cudaGetErrorString(ce);
        ws->ptr = nullptr;
        return nullptr;
    }
    ce = cudaMemset(ws->ptr, 0, bytes);  // kernels rely on zeroed counters
    if (ce != cudaSuccess) {
        err = std::string("cudaMemset(workspace): ") + cudaGetErrorString(ce);
        cudaFree(ws->ptr);
        ws->ptr = nullptr;
        return nullptr;
    }
    ws->bytes = bytes;
    ws->owner = owner;
    return ws->ptr;
}
}  // namespace ecl

namespace {

struct Buf {
    void *ptr;
    size_t bytes;
    bool in;
    bool host;
    void *mirror;  // device copy of a host buffer
};

struct ArgVal {
    bool set = false;
    size_t bytes = 0;
    uint64_t raw = 0;
};

}  // namespace

struct ecl_program {
    const KernelDesc *k = nullptr;
    std::vector<Buf> bufs;
    ArgVal args[16];
    int next_arg = 0;
    uint32_t out_outs = 0, out_wis = 0;  // 0 = kernel default
    bool owned = false;
};

struct ecl_engine {
    int device = 0;
    cudaStream_t stream = nullptr;
    ecl_program *prog = nullptr;
    uint64_t gws = 0;
    uint32_t lws = 0;
    ecl_sched_kind kind = ECL_STATIC;
    std::vector<double> params;
    int D = 0, C = 0;
    int sms = 0;
    // errors
    std::string last_error;
    int nerrors = 0;
    // device memory
    Queue *q = nullptr;
    DevState *dev = nullptr;
    size_t dev_cap = 0;
    Pkg *table = nullptr;
    PkgRec *rec = nullptr;
    size_t table_cap = 0;
    ecl_worker_stat *wst = nullptr;
    size_t wst_cap = 0;
    double *hg_p = nullptr;
    uint32_t *hg_min = nullptr;
    size_t hg_cap = 0;
    Queue *q_host = nullptr;  // pinned
    Pkg *stage = nullptr;     // pinned staging for the table
    size_t stage_cap = 0;
    std::vector<Pkg> uploaded;
    uint32_t uploaded_mode = 0xffffffffu;
    std::vector<double> hg_uploaded_p;
    std::vector<uint32_t> hg_uploaded_min;
    uint32_t *coverage = nullptr;
    uint64_t coverage_n = 0;
    uint32_t spin_limit = 20000000u;  // ecl_debug knobs
    uint32_t withhold = 0;
    Workspace ws;
    // host buffers: optional copy streams, and whether a run returns before
    // its copies finish (ecl_engine_copy_streams)
    cudaStream_t h2d = nullptr, d2h = nullptr;
    bool copies_set = false, host_async = false;
    cudaEvent_t ev_in = nullptr, ev_done = nullptr, ev_out = nullptr;
    bool ev_pending = false;  // ev_done / ev_out record a run not yet waited for
    // caller's events around each run's main kernel (ecl_engine_kernel_events)
    cudaEvent_t kev_begin = nullptr, kev_end = nullptr;
    // facts of the last run
    uint64_t last_G = 0, last_npkg = 0;
    uint32_t last_D = 0, last_C = 0, last_grid = 0, last_mode = MODE_MONO;
    bool ran = false;
};

namespace {

ecl_status fail(ecl_engine *e, ecl_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (e) {
        e->last_error = buf;
        e->nerrors++;
    }
    return st;
}

ecl_status ferr(std::string &err, ecl_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return st;
}

#define CUDA_OR_FAIL(e, call)                                                          \
    do {                                                                               \
        cudaError_t ce_ = (call);                                                      \
        if (ce_ != cudaSuccess)                                                        \
            return fail((e), ECL_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(ce_));  \
    } while (0)

bool is_host_pointer(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

ecl_status grow(ecl_engine *e, void **p, size_t *cap, size_t need, size_t elem)
{
    if (*cap >= need) return ECL_OK;
    size_t n = std::max(need, (size_t)64);
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    CUDA_OR_FAIL(e, cudaMalloc(p, n * elem));
    CUDA_OR_FAIL(e, cudaMemset(*p, 0, n * elem));
    *cap = n;
    return ECL_OK;
}

// ------------------------------------------------------------------ planner
// The package rules restated from Sec. 5.3; every size is in scheduling
// units (ceil(G / grain)), converted to work-groups with the tail clipped.
struct Plan {
    uint32_t mode = MODE_QUEUE;
    std::vector<Pkg> table;
    std::vector<double> hg_p;
    std::vector<uint32_t> hg_min;
    double hg_k = 2.0, hg_sum_p = 0.0;
    uint64_t units = 0;
};

void push_units(Plan &pl, uint64_t G, uint64_t grain, uint64_t u0, uint64_t ul)
{
    Pkg p;
    uint64_t off = std::min(G, u0 * grain), end = std::min(G, (u0 + ul) * grain);
    p.off = off;
    p.len = end - off;
    p.nchunks = 0;
    p.pad = 0;
    pl.table.push_back(p);
}

ecl_status make_plan(ecl_sched_kind kind, const std::vector<double> &pr, uint64_t G, uint64_t grain, uint32_t D,
                     Plan &pl, std::string &err)
{
    const uint64_t U = (G + grain - 1) / grain;
    pl.units = U;
    switch (kind) {
    case ECL_STATIC:
    case ECL_STATIC_REV: {
        pl.mode = MODE_STATIC;
        std::vector<uint64_t> size(D, 0);
        uint64_t sum = 0;
        if (pr.empty()) {
            for (uint32_t d = 0; d + 1 < D; ++d) size[d] = U / D;
        } else {
            if (pr.size() != D - 1 && pr.size() != D)
                return ferr(err, ECL_ERR_SCHED, "Static: %zu proportions given for %u devices (need %u or %u)",
                            pr.size(), D, D - 1, D);
            double tot = 0.0;
            for (uint32_t d = 0; d + 1 < D; ++d) {
                if (!(pr[d] >= 0.0)) return ferr(err, ECL_ERR_SCHED, "Static: proportion %u is negative", d);
                tot += pr[d];
                size[d] = (uint64_t)floor(pr[d] * (double)U);
            }
            if (tot > 1.0 + 1e-12) return ferr(err, ECL_ERR_SCHED, "Static: proportions sum to %g > 1", tot);
        }
        for (uint32_t d = 0; d + 1 < D; ++d) sum += size[d];
        if (sum > U) return ferr(err, ECL_ERR_SCHED, "Static: proportions exceed the NDRange");
        size[D - 1] = U - sum;
        pl.table.assign(D, Pkg{});
        uint64_t u = 0;
        for (uint32_t i = 0; i < D; ++i) {
            const uint32_t d = (kind == ECL_STATIC_REV) ? D - 1 - i : i;
            Plan one;
            push_units(one, G, grain, u, size[d]);
            pl.table[d] = one.table[0];
            u += size[d];
        }
        return ECL_OK;
    }
    case ECL_DYNAMIC: {
        pl.mode = MODE_QUEUE;
        if (pr.size() != 1 || !(pr[0] >= 1.0) || pr[0] != floor(pr[0]))
            return ferr(err, ECL_ERR_SCHED, "Dynamic: params must be {num_packages >= 1}");
        const uint64_t np = (uint64_t)pr[0];
        if (U == 0) return ECL_OK;
        const uint64_t sz = (U + np - 1) / np;
        for (uint64_t u = 0; u < U; u += sz) push_units(pl, G, grain, u, std::min(sz, U - u));
        return ECL_OK;
    }
    case ECL_HGUIDED: {
        double k = pr.size() > 0 ? pr[0] : 2.0;
        double mb = pr.size() > 1 ? pr[1] : 1.0;
        if (!(k > 0.0) || !(mb >= 1.0) || mb != floor(mb))
            return ferr(err, ECL_ERR_SCHED, "HGuided: need k > 0 and an integer min_package >= 1");
        std::vector<double> P(D, 1.0);
        if (pr.size() > 2) {
            if (pr.size() != 2 + (size_t)D)
                return ferr(err, ECL_ERR_SCHED, "HGuided: %zu powers given for %u devices", pr.size() - 2, D);
            for (uint32_t d = 0; d < D; ++d) {
                P[d] = pr[2 + d];
                if (!(P[d] > 0.0)) return ferr(err, ECL_ERR_SCHED, "HGuided: power %u must be > 0", d);
            }
        }
        double sumP = 0.0, pmin = P[0];
        bool equal = true;
        for (uint32_t d = 0; d < D; ++d) {
            sumP += P[d];
            pmin = std::min(pmin, P[d]);
            equal = equal && (P[d] == P[0]);
        }
        std::vector<uint32_t> mins(D);
        for (uint32_t d = 0; d < D; ++d) {
            double m = floor(mb * P[d] / pmin + 0.5);
            mins[d] = (uint32_t)std::max(1.0, std::min(m, 4294967295.0));
        }
        pl.hg_k = k;
        pl.hg_sum_p = sumP;
        if (!equal) {  // sizes depend on which device asks: cut on the device
            pl.mode = MODE_HGUIDED;
            pl.hg_p = P;
            pl.hg_min = mins;
            return ECL_OK;
        }
        pl.mode = MODE_QUEUE;
        uint64_t gr = U, u = 0;
        while (gr > 0) {
            const double q = ((double)gr * P[0]) / ((k * (double)D) * sumP);
            uint64_t sz = (uint64_t)floor(q);
            sz = std::max<uint64_t>(sz, mins[0]);
            sz = std::min(sz, gr);
            push_units(pl, G, grain, u, sz);
            u += sz;
            gr -= sz;
        }
        return ECL_OK;
    }
    case ECL_MONOLITHIC:
        pl.mode = MODE_MONO;
        return ECL_OK;
    }
    return ferr(err, ECL_ERR_SCHED, "unknown scheduler kind %d", (int)kind);
}

bool same_table(const std::vector<Pkg> &a, const std::vector<Pkg> &b)
{
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i)
        if (a[i].off != b[i].off || a[i].len != b[i].len || a[i].nchunks != b[i].nchunks) return false;
    return true;
}

ecl_status check_device_error(ecl_engine *e)
{
    CUDA_OR_FAIL(e, cudaMemcpyAsync(e->q_host, e->q, sizeof(Queue), cudaMemcpyDeviceToHost, e->stream));
    CUDA_OR_FAIL(e, cudaStreamSynchronize(e->stream));
    if (e->ev_pending) {  // the output copies of the last run, on the copy stream
        CUDA_OR_FAIL(e, cudaEventSynchronize(e->ev_out));
        e->ev_pending = false;
    }
    if (e->q_host->error) {
        const unsigned long long info = e->q_host->error_info;
        // the run is void: put the queue back in its initial state
        CUDA_OR_FAIL(e, cudaMemsetAsync(e->q, 0, sizeof(Queue), e->stream));
        if (e->dev) CUDA_OR_FAIL(e, cudaMemsetAsync(e->dev, 0, e->dev_cap * sizeof(DevState), e->stream));
        if (e->ws.ptr) CUDA_OR_FAIL(e, cudaMemsetAsync(e->ws.ptr, 0, e->ws.bytes, e->stream));
        CUDA_OR_FAIL(e, cudaStreamSynchronize(e->stream));
        return fail(e, ECL_ERR_TIMEOUT, "device wait gave up (CTA %llu after %llu polls); the run is void",
                    info >> 32, info & 0xffffffffull);
    }
    return ECL_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

ecl_status ecl_engine_create(ecl_engine **out, int device_ordinal, void *cuda_stream)
{
    if (!out) return ECL_ERR_ARG;
    *out = nullptr;
    ecl_engine *e = new (std::nothrow) ecl_engine();
    if (!e) return ECL_ERR_ARG;
    e->device = device_ordinal;
    e->stream = (cudaStream_t)cuda_stream;
    cudaError_t ce = cudaSetDevice(device_ordinal);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, device_ordinal);
    if (ce == cudaSuccess) ce = cudaMalloc((void **)&e->q, sizeof(Queue));
    if (ce == cudaSuccess) ce = cudaMemset(e->q, 0, sizeof(Queue));
    if (ce == cudaSuccess) ce = cudaMallocHost((void **)&e->q_host, sizeof(Queue));
    if (ce != cudaSuccess) {
        ecl_status st = ECL_ERR_CUDA;
        if (e->q) cudaFree(e->q);
        delete e;
        cudaGetLastError();
        return st;
    }
    *out = e;
    return ECL_OK;
}

void ecl_program_destroy(ecl_program *p);

void ecl_engine_destroy(ecl_engine *e)
{
    if (!e) return;
    cudaSetDevice(e->device);
    cudaStreamSynchronize(e->stream);
    if (e->prog) {
        e->prog->owned = false;
        ecl_program_destroy(e->prog);
    }
    cudaFree(e->q);
    cudaFree(e->dev);
    cudaFree(e->table);
    cudaFree(e->rec);
    cudaFree(e->wst);
    cudaFree(e->hg_p);
    cudaFree(e->hg_min);
    cudaFree(e->ws.ptr);
    cudaFreeHost(e->q_host);
    cudaFreeHost(e->stage);
    if (e->ev_out) cudaEventSynchronize(e->ev_out);
    for (cudaEvent_t ev : {e->ev_in, e->ev_done, e->ev_out})
        if (ev) cudaEventDestroy(ev);
    delete e;
}

ecl_status ecl_engine_copy_streams(ecl_engine *e, void *h2d_stream, void *d2h_stream, int async)
{
    if (!e) return ECL_ERR_ARG;
    CUDA_OR_FAIL(e, cudaSetDevice(e->device));
    if (e->ev_pending) {
        CUDA_OR_FAIL(e, cudaEventSynchronize(e->ev_out));
        e->ev_pending = false;
    }
    for (cudaEvent_t *ev : {&e->ev_in, &e->ev_done, &e->ev_out})
        if (!*ev) CUDA_OR_FAIL(e, cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    e->h2d = (cudaStream_t)h2d_stream;
    e->d2h = (cudaStream_t)d2h_stream;
    e->copies_set = true;
    e->host_async = async != 0;
    return ECL_OK;
}

ecl_status ecl_engine_kernel_events(ecl_engine *e, void *begin, void *end)
{
    if (!e || (!begin) != (!end)) return ECL_ERR_ARG;
    e->kev_begin = (cudaEvent_t)begin;
    e->kev_end = (cudaEvent_t)end;
    return ECL_OK;
}

ecl_status ecl_engine_set_stream(ecl_engine *e, void *cuda_stream)
{
    if (!e) return ECL_ERR_ARG;
    e->stream = (cudaStream_t)cuda_stream;
    return ECL_OK;
}

ecl_status ecl_work_items(ecl_engine *e, uint64_t gws, uint32_t lws)
{
    if (!e) return ECL_ERR_ARG;
    if (gws == 0 || lws == 0)
        return fail(e, ECL_ERR_SIZE, "work_items: gws and lws must be positive (gws=%llu lws=%u)",
                    (unsigned long long)gws, lws);
    if (gws % lws != 0)
        return fail(e, ECL_ERR_SIZE, "work_items: gws %llu is not a multiple of lws %u",
                    (unsigned long long)gws, lws);
    e->gws = gws;
    e->lws = lws;
    return ECL_OK;
}

ecl_status ecl_scheduler(ecl_engine *e, ecl_sched_kind kind, const double *params, int nparams)
{
    if (!e) return ECL_ERR_ARG;
    if ((int)kind < 0 || (int)kind > (int)ECL_MONOLITHIC)
        return fail(e, ECL_ERR_SCHED, "unknown scheduler kind %d", (int)kind);
    if (nparams < 0 || (nparams > 0 && !params))
        return fail(e, ECL_ERR_SCHED, "scheduler: bad parameter array");
    e->kind = kind;
    e->params.assign(params, params + nparams);
    return ECL_OK;
}

ecl_status ecl_workers(ecl_engine *e, int devices, int ctas_per_device)
{
    if (!e) return ECL_ERR_ARG;
    if (devices < 0 || ctas_per_device < 0)
        return fail(e, ECL_ERR_ARG, "workers: counts must be >= 0");
    e->D = devices;
    e->C = ctas_per_device;
    return ECL_OK;
}

ecl_status ecl_engine_program(ecl_engine *e, ecl_program *p)
{
    if (!e || !p) return ECL_ERR_ARG;
    if (p->owned) return fail(e, ECL_ERR_STATE, "program already belongs to an engine");
    if (e->prog && e->prog != p) {
        e->prog->owned = false;
        ecl_program_destroy(e->prog);
    }
    p->owned = true;
    e->prog = p;
    return ECL_OK;
}

ecl_status ecl_set_coverage(ecl_engine *e, uint32_t *counts, uint64_t n)
{
    if (!e) return ECL_ERR_ARG;
    e->coverage = counts;
    e->coverage_n = counts ? n : 0;
    return ECL_OK;
}

ecl_status ecl_debug(ecl_engine *e, int kind, int64_t value)
{
    if (!e) return ECL_ERR_ARG;
    if (value < 0) return fail(e, ECL_ERR_ARG, "ecl_debug: negative value");
    if (kind == ECL_DEBUG_SPIN_LIMIT) {
        e->spin_limit = value == 0 ? 20000000u : (uint32_t)std::min<int64_t>(value, 0xffffffffll);
    } else if (kind == ECL_DEBUG_WITHHOLD) {
        e->withhold = value ? 1u : 0u;
    } else {
        return fail(e, ECL_ERR_ARG, "ecl_debug: unknown kind %d", kind);
    }
    return ECL_OK;
}

const char *ecl_last_error(const ecl_engine *e)
{
    if (!e) return "NULL engine";
    return e->last_error.c_str();
}

int ecl_error_count(const ecl_engine *e) { return e ? e->nerrors : 0; }

void ecl_clear_errors(ecl_engine *e)
{
    if (!e) return;
    e->nerrors = 0;
    e->last_error.clear();
}

ecl_status ecl_plan_info(const ecl_engine *e, uint64_t *G, uint64_t *packages, uint32_t *devices,
                         uint32_t *ctas_per_device, uint32_t *ctas)
{
    if (!e) return ECL_ERR_ARG;
    if (G) *G = e->last_G;
    if (packages) *packages = e->last_npkg;
    if (devices) *devices = e->last_D;
    if (ctas_per_device) *ctas_per_device = e->last_C;
    if (ctas) *ctas = e->last_grid;
    return ECL_OK;
}

ecl_status ecl_kernel_occupancy(int device_ordinal, const char *kernel_name, int *sms, int *ctas_per_sm)
{
    const KernelDesc *k = kernel_name ? find_kernel(kernel_name) : nullptr;
    if (!k) return ECL_ERR_KERNEL;
    if (cudaSetDevice(device_ordinal) != cudaSuccess) {
        cudaGetLastError();
        return ECL_ERR_CUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device_ordinal) != cudaSuccess) {
        cudaGetLastError();
        return ECL_ERR_CUDA;
    }
    if (sms) *sms = n;
    if (ctas_per_sm) *ctas_per_sm = k->ctas_per_sm();
    return ECL_OK;
}

// ------------------------------------------------------------------ program
ecl_status ecl_program_create(ecl_program **out, const char *kernel_name)
{
    if (!out || !kernel_name) return ECL_ERR_ARG;
    *out = nullptr;
    const KernelDesc *k = find_kernel(kernel_name);
    if (!k) return ECL_ERR_KERNEL;
    ecl_program *p = new (std::nothrow) ecl_program();
    if (!p) return ECL_ERR_ARG;
    p->k = k;
    *out = p;
    return ECL_OK;
}

void ecl_program_destroy(ecl_program *p)
{
    if (!p || p->owned) return;
    for (Buf &b : p->bufs)
        if (b.mirror) cudaFree(b.mirror);
    delete p;
}

static ecl_status add_buf(ecl_program *p, void *ptr, size_t bytes, bool in)
{
    if (!p || !ptr || bytes == 0) return ECL_ERR_ARG;
    for (Buf &b : p->bufs)
        if (b.ptr == ptr) {  // re-registration updates size and direction
            if (b.mirror && b.bytes < bytes) {
                cudaFree(b.mirror);
                b.mirror = nullptr;
            }
            b.bytes = bytes;
            b.in = in;
            return ECL_OK;
        }
    Buf b;
    b.ptr = ptr;
    b.bytes = bytes;
    b.in = in;
    b.host = is_host_pointer(ptr);
    b.mirror = nullptr;
    p->bufs.push_back(b);
    return ECL_OK;
}

ecl_status ecl_program_in(ecl_program *p, void *ptr, size_t bytes) { return add_buf(p, ptr, bytes, true); }
ecl_status ecl_program_out(ecl_program *p, void *ptr, size_t bytes) { return add_buf(p, ptr, bytes, false); }

ecl_status ecl_program_out_pattern(ecl_program *p, uint32_t outs, uint32_t work_items)
{
    if (!p || outs == 0 || work_items == 0) return ECL_ERR_ARG;
    p->out_outs = outs;
    p->out_wis = work_items;
    return ECL_OK;
}

ecl_status ecl_program_arg(ecl_program *p, int index, const void *value, size_t bytes)
{
    if (!p || !value) return ECL_ERR_ARG;
    if (index < 0) index = p->next_arg;
    if (index >= p->k->nargs) return ECL_ERR_ARG;
    const ArgKind kind = p->k->args[index].kind;
    size_t want = (kind == A_BUF_IN || kind == A_BUF_OUT || kind == A_BUF_OUT_OPT) ? sizeof(void *)
                  : (kind == A_I64) ? 8 : 4;
    if (bytes != want) return ECL_ERR_ARG;
    ArgVal &a = p->args[index];
    a.set = true;
    a.bytes = bytes;
    a.raw = 0;
    memcpy(&a.raw, value, bytes);
    p->next_arg = index + 1;
    return ECL_OK;
}

ecl_status ecl_program_local(ecl_program *p, int index, size_t bytes)
{
    (void)index;
    (void)bytes;
    if (!p) return ECL_ERR_ARG;
    return ECL_ERR_ARG;  // no built-in kernel declares a local-memory argument
}

// ------------------------------------------------------------------ run
ecl_status ecl_run(ecl_engine *e)
{
    if (!e) return ECL_ERR_ARG;
    ecl_program *p = e->prog;
    if (!p) return fail(e, ECL_ERR_STATE, "run: no program (call ecl_engine_program first)");
    if (!e->gws) return fail(e, ECL_ERR_STATE, "run: work items not set");
    const KernelDesc *k = p->k;
    CUDA_OR_FAIL(e, cudaSetDevice(e->device));

    // resolve arguments (the Buffer proxy: host buffers get device mirrors)
    KArgs a;
    a.n = k->nargs;
    std::vector<Buf *> host_in, host_out;
    for (int i = 0; i < k->nargs; ++i) {
        const ArgVal &v = p->args[i];
        const ArgKind kind = k->args[i].kind;
        if (!v.set) return fail(e, ECL_ERR_ARG, "%s: argument %d (%s) not set", k->name, i, k->args[i].name);
        if (kind == A_BUF_IN || kind == A_BUF_OUT || kind == A_BUF_OUT_OPT) {
            void *ptr = nullptr;
            memcpy(&ptr, &v.raw, sizeof(void *));
            if (!ptr) {
                if (kind != A_BUF_OUT_OPT)
                    return fail(e, ECL_ERR_BUFFER, "%s: argument %d (%s) is NULL", k->name, i, k->args[i].name);
                continue;
            }
            Buf *hit = nullptr;
            for (Buf &b : p->bufs)
                if ((char *)ptr >= (char *)b.ptr && (char *)ptr < (char *)b.ptr + b.bytes) hit = &b;
            if (!hit)
                return fail(e, ECL_ERR_BUFFER, "%s: argument %d (%s) is not a registered buffer", k->name, i,
                            k->args[i].name);
            if ((kind == A_BUF_IN) != hit->in)
                return fail(e, ECL_ERR_BUFFER, "%s: argument %d (%s) registered with the wrong direction",
                            k->name, i, k->args[i].name);
            const size_t offb = (size_t)((char *)ptr - (char *)hit->ptr);
            a.bytes[i] = hit->bytes - offb;
            if (hit->host) {
                if (!hit->mirror) CUDA_OR_FAIL(e, cudaMalloc(&hit->mirror, hit->bytes));
                a.ptr[i] = (char *)hit->mirror + offb;
                std::vector<Buf *> &lst = hit->in ? host_in : host_out;
                if (std::find(lst.begin(), lst.end(), hit) == lst.end()) lst.push_back(hit);
            } else {
                a.ptr[i] = ptr;
            }
        } else {
            a.raw[i] = v.raw;
        }
    }
    std::string err;
    ecl_status st = k->validate(a, e->gws, e->lws, err);
    if (st != ECL_OK) return fail(e, st, "%s: %s", k->name, err.c_str());
    {  // output pattern (Sec. 4.2): must agree with the kernel's own
        const uint32_t ko = k->out_outs, kw = k->out_wis ? k->out_wis : e->lws;
        if (p->out_outs && (uint64_t)p->out_outs * kw != (uint64_t)ko * p->out_wis)
            return fail(e, ECL_ERR_ARG, "%s: out pattern %u:%u differs from the kernel's %u:%u", k->name,
                        p->out_outs, p->out_wis, ko, kw);
    }

    const uint64_t G = e->gws / e->lws;
    const uint64_t grain = k->grain(a, e->gws, e->lws);
    const int per_sm = k->ctas_per_sm();
    if (per_sm < 1) return fail(e, ECL_ERR_CUDA, "%s: kernel cannot be resident (occupancy 0)", k->name);
    const uint32_t resident = (uint32_t)(per_sm * e->sms);
    uint32_t D = (uint32_t)e->D, C = (uint32_t)e->C;
    if (D == 0 && C == 0) {
        if (k->default_D > 0) {
            D = std::min<uint32_t>((uint32_t)k->default_D, resident);
            C = std::max<uint32_t>(1, resident / D);
        } else {
            D = resident;
            C = 1;
        }
    } else if (D == 0) {
        D = std::max<uint32_t>(1, resident / C);
    } else if (C == 0) {
        C = std::max<uint32_t>(1, resident / D);
    }
    if ((uint64_t)D * C > (uint64_t)resident * 64)
        return fail(e, ECL_ERR_SIZE, "workers: %u x %u CTAs is far beyond the %u resident", D, C, resident);

    Plan pl;
    st = make_plan(e->kind, e->params, G, grain, D, pl, err);
    if (st != ECL_OK) return fail(e, st, "%s", err.c_str());
    SchedArgs s{};
    s.G = G;
    s.grain = grain;
    s.units = pl.units;
    s.mode = pl.mode;
    s.D = D;
    s.C = C;
    s.spin_limit = e->spin_limit;
    s.withhold = e->withhold;
    s.coverage = e->coverage;
    if (e->coverage && e->coverage_n < G)
        return fail(e, ECL_ERR_BUFFER, "coverage array has %llu entries, G = %llu",
                    (unsigned long long)e->coverage_n, (unsigned long long)G);
    uint32_t grid;
    bool grid_static = false;
    if (pl.mode == MODE_MONO) {
        const uint64_t nch = k->nchunks(a, e->gws, e->lws, 0, G);
        if (nch == 0 || nch > 0x7fffffffull)
            return fail(e, ECL_ERR_SIZE, "%s: monolithic grid of %llu CTAs", k->name, (unsigned long long)nch);
        s.mono_nchunks = (uint32_t)nch;
        grid = (uint32_t)nch;
        D = C = 0;
        s.D = s.C = 0;
    } else {
        grid = D * C;
        for (Pkg &pk : pl.table) {
            const uint64_t nch = k->nchunks(a, e->gws, e->lws, pk.off, pk.len);
            if (nch > 0x7fffffffull) return fail(e, ECL_ERR_SIZE, "%s: package of %llu chunks", k->name,
                                                 (unsigned long long)nch);
            pk.nchunks = (uint32_t)nch;
        }
        // Static over one device leaves nothing to decide at run time: the
        // device's single package [0, G) runs as one grid, CTA b = chunk b
        // (as the paper's runtime enqueues one kernel per device package),
        // with its package and worker records kept.  Kernels with their own
        // claim loop stay on the queue.
        grid_static = pl.mode == MODE_STATIC && D == 1 && pl.table.size() == 1 && !k->own_claims &&
                      pl.table[0].off == 0 && pl.table[0].len == G && pl.table[0].nchunks > 0;
        if (grid_static) grid = pl.table[0].nchunks;
        const size_t cap_need = pl.mode == MODE_HGUIDED ? (size_t)std::max<uint64_t>(pl.units, 1)
                                                        : std::max<size_t>(pl.table.size(), 1);
        if (cap_need > 0xffffffffull) return fail(e, ECL_ERR_SIZE, "too many packages");
        size_t tcap = e->table_cap;
        if (tcap < cap_need) {
            CUDA_OR_FAIL(e, cudaStreamSynchronize(e->stream));
            st = grow(e, (void **)&e->table, &tcap, cap_need, sizeof(Pkg));
            if (st != ECL_OK) return st;
            size_t rcap = 0;
            if (e->rec) cudaFree(e->rec);
            e->rec = nullptr;
            st = grow(e, (void **)&e->rec, &rcap, tcap, sizeof(PkgRec));
            if (st != ECL_OK) return st;
            e->table_cap = tcap;
            e->uploaded.clear();
            e->uploaded_mode = 0xffffffffu;
        }
        if (e->dev_cap < D) {
            CUDA_OR_FAIL(e, cudaStreamSynchronize(e->stream));
            st = grow(e, (void **)&e->dev, &e->dev_cap, D, sizeof(DevState));
            if (st != ECL_OK) return st;
        }
        if (e->wst_cap < grid) {
            CUDA_OR_FAIL(e, cudaStreamSynchronize(e->stream));
            st = grow(e, (void **)&e->wst, &e->wst_cap, grid, sizeof(ecl_worker_stat));
            if (st != ECL_OK) return st;
        }
        if (pl.mode != MODE_HGUIDED &&
            (e->uploaded_mode == MODE_HGUIDED || !same_table(pl.table, e->uploaded))) {
            if (e->stage_cap < pl.table.size()) {
                CUDA_OR_FAIL(e, cudaStreamSynchronize(e->stream));
                cudaFreeHost(e->stage);
                e->stage = nullptr;
                e->stage_cap = 0;
                CUDA_OR_FAIL(e, cudaMallocHost((void **)&e->stage, pl.table.size() * sizeof(Pkg)));
                e->stage_cap = pl.table.size();
            } else {
                CUDA_OR_FAIL(e, cudaStreamSynchronize(e->stream));  // staging may be in flight
            }
            memcpy(e->stage, pl.table.data(), pl.table.size() * sizeof(Pkg));
            if (!pl.table.empty())
                CUDA_OR_FAIL(e, cudaMemcpyAsync(e->table, e->stage, pl.table.size() * sizeof(Pkg),
                                                cudaMemcpyHostToDevice, e->stream));
            e->uploaded = pl.table;
        }
        e->uploaded_mode = pl.mode;
        if (pl.mode == MODE_HGUIDED) {
            e->uploaded.clear();
            if (e->hg_cap < D) {
                CUDA_OR_FAIL(e, cudaStreamSynchronize(e->stream));
                cudaFree(e->hg_p);
                cudaFree(e->hg_min);
                e->hg_p = nullptr;
                e->hg_min = nullptr;
                e->hg_cap = 0;
                CUDA_OR_FAIL(e, cudaMalloc((void **)&e->hg_p, D * sizeof(double)));
                CUDA_OR_FAIL(e, cudaMalloc((void **)&e->hg_min, D * sizeof(uint32_t)));
                e->hg_cap = D;
                e->hg_uploaded_p.clear();
            }
            if (pl.hg_p != e->hg_uploaded_p || pl.hg_min != e->hg_uploaded_min) {
                CUDA_OR_FAIL(e, cudaMemcpy(e->hg_p, pl.hg_p.data(), D * sizeof(double), cudaMemcpyHostToDevice));
                CUDA_OR_FAIL(e, cudaMemcpy(e->hg_min, pl.hg_min.data(), D * sizeof(uint32_t),
                                           cudaMemcpyHostToDevice));
                e->hg_uploaded_p = pl.hg_p;
                e->hg_uploaded_min = pl.hg_min;
            }
            s.hg_k = pl.hg_k;
            s.hg_sum_p = pl.hg_sum_p;
            s.hg_p = e->hg_p;
            s.hg_min = e->hg_min;
        }
        s.table = e->table;
        s.rec = e->rec;
        s.table_cap = e->table_cap;
        s.npkg = (uint32_t)pl.table.size();
        s.dev = e->dev;
        s.wst = e->wst;
        if (grid_static) {
            s.mode = MODE_MONO;
            s.records = 1;
            s.mono_nchunks = grid;
            C = grid;
        }
    }
    s.q = e->q;

    const bool copies = e->copies_set && (!host_in.empty() || !host_out.empty());
    cudaStream_t h2d = e->h2d ? e->h2d : e->stream, d2h = e->d2h ? e->d2h : e->stream;
    if (copies && e->ev_pending) {
        // the previous run's kernel reads the input mirrors and its output
        // copies read the output mirrors: new copies in wait for the kernel,
        // the new kernel waits for the copies out
        CUDA_OR_FAIL(e, cudaStreamWaitEvent(h2d, e->ev_done, 0));
        CUDA_OR_FAIL(e, cudaStreamWaitEvent(e->stream, e->ev_out, 0));
    }
    if (copies && !host_in.empty()) {
        for (Buf *b : host_in)
            CUDA_OR_FAIL(e, cudaMemcpyAsync(b->mirror, b->ptr, b->bytes, cudaMemcpyHostToDevice, h2d));
        CUDA_OR_FAIL(e, cudaEventRecord(e->ev_in, h2d));
        CUDA_OR_FAIL(e, cudaStreamWaitEvent(e->stream, e->ev_in, 0));
    } else {
        for (Buf *b : host_in)
            CUDA_OR_FAIL(e, cudaMemcpyAsync(b->mirror, b->ptr, b->bytes, cudaMemcpyHostToDevice, e->stream));
    }
    LaunchCtx lc;
    lc.stream = e->stream;
    lc.lws = e->lws;
    lc.gws = e->gws;
    lc.grid = grid;
    lc.ws = &e->ws;
    bool marked = false;
    if (e->kev_begin) {
        CUDA_OR_FAIL(e, cudaEventRecord(e->kev_begin, e->stream));
        lc.mark_begin = e->kev_begin;
        lc.mark_end = e->kev_end;
        lc.marked = &marked;
    }
    st = k->launch(a, s, lc, err);
    if (st != ECL_OK) return fail(e, st, "%s: %s", k->name, err.c_str());
    if (e->kev_end && !marked) CUDA_OR_FAIL(e, cudaEventRecord(e->kev_end, e->stream));
    e->last_G = G;
    e->last_npkg = pl.mode == MODE_HGUIDED ? 0 : pl.table.size();
    e->last_D = D;
    e->last_C = C;
    e->last_grid = grid;
    e->last_mode = pl.mode;
    e->ran = true;
    if (copies) {
        CUDA_OR_FAIL(e, cudaEventRecord(e->ev_done, e->stream));
        CUDA_OR_FAIL(e, cudaStreamWaitEvent(d2h, e->ev_done, 0));
        for (Buf *b : host_out)
            CUDA_OR_FAIL(e, cudaMemcpyAsync(b->ptr, b->mirror, b->bytes, cudaMemcpyDeviceToHost, d2h));
        CUDA_OR_FAIL(e, cudaEventRecord(e->ev_out, d2h));
        e->ev_pending = true;
        return e->host_async ? ECL_OK : check_device_error(e);
    }
    if (!host_out.empty() || !host_in.empty()) {
        for (Buf *b : host_out)
            CUDA_OR_FAIL(e, cudaMemcpyAsync(b->ptr, b->mirror, b->bytes, cudaMemcpyDeviceToHost, e->stream));
        return check_device_error(e);
    }
    return ECL_OK;
}

ecl_status ecl_plan(ecl_sched_kind kind, const double *params, int nparams, uint64_t G, uint64_t grain,
                    uint32_t devices, uint64_t *off, uint64_t *len, uint32_t *device, size_t cap, size_t *n,
                    char *errbuf, size_t errlen)
{
    if (!n || (cap && (!off || !len)) || grain == 0 || devices == 0 || nparams < 0 || (nparams && !params))
        return ECL_ERR_ARG;
    *n = 0;
    std::vector<double> pr(params, params + nparams);
    Plan pl;
    std::string err;
    ecl_status st = make_plan(kind, pr, G, grain, devices, pl, err);
    if (st == ECL_OK && pl.mode == MODE_MONO) {
        st = ECL_ERR_SCHED;
        err = "the monolithic launch has no packages";
    }
    if (st != ECL_OK) {
        if (errbuf && errlen) snprintf(errbuf, errlen, "%s", err.c_str());
        return st;
    }
    std::vector<uint32_t> who;
    if (pl.mode == MODE_HGUIDED) {  // device-cut sizes: simulate requests in device order 0..D-1, cyclic
        uint64_t used = 0;
        uint32_t d = 0;
        while (used < pl.units) {
            const uint64_t gr = pl.units - used;
            const double q = ((double)gr * pl.hg_p[d]) / ((pl.hg_k * (double)devices) * pl.hg_sum_p);
            uint64_t sz = (uint64_t)floor(q);
            sz = std::max<uint64_t>(sz, pl.hg_min[d]);
            sz = std::min(sz, gr);
            push_units(pl, G, grain, used, sz);
            who.push_back(d);
            used += sz;
            d = (d + 1) % devices;
        }
    } else {
        for (size_t i = 0; i < pl.table.size(); ++i)
            who.push_back(pl.mode == MODE_STATIC ? (uint32_t)i : 0xffffffffu);
    }
    const size_t m = std::min(cap, pl.table.size());
    for (size_t i = 0; i < m; ++i) {
        off[i] = pl.table[i].off;
        len[i] = pl.table[i].len;
        if (device) device[i] = who[i];
    }
    *n = pl.table.size();
    return m < pl.table.size() ? ECL_ERR_SIZE : ECL_OK;
}

ecl_status ecl_synchronize(ecl_engine *e)
{
    if (!e) return ECL_ERR_ARG;
    CUDA_OR_FAIL(e, cudaSetDevice(e->device));
    return check_device_error(e);
}

ecl_status ecl_stats(ecl_engine *e, ecl_pkg_stat *out, size_t cap, size_t *n)
{
    if (!e || !n || (cap && !out)) return ECL_ERR_ARG;
    *n = 0;
    ecl_status st = ecl_synchronize(e);
    if (st != ECL_OK) return st;
    if (!e->ran || e->last_mode == MODE_MONO) return ECL_OK;
    uint64_t np = e->last_npkg;
    if (e->last_mode == MODE_HGUIDED) {
        np = e->q_host->last_npkg;  // read by ecl_synchronize
        e->last_npkg = np;
    }
    const size_t m = (size_t)std::min<uint64_t>(np, cap);
    if (m) {
        std::vector<PkgRec> tmp(m);
        CUDA_OR_FAIL(e, cudaMemcpy(tmp.data(), e->rec, m * sizeof(PkgRec), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < m; ++i) {
            out[i].off_wg = tmp[i].off;
            out[i].len_wg = tmp[i].len;
            out[i].t0_ns = tmp[i].t0;
            out[i].t1_ns = tmp[i].t1 ? tmp[i].t1 : tmp[i].t0;
            out[i].pkg = tmp[i].pkg;
            out[i].device = tmp[i].device;
            out[i].cta = tmp[i].cta;
            out[i].smid = tmp[i].smid;
        }
    }
    *n = m;
    return ECL_OK;
}

ecl_status ecl_worker_stats(ecl_engine *e, ecl_worker_stat *out, size_t cap, size_t *n)
{
    if (!e || !n || (cap && !out)) return ECL_ERR_ARG;
    *n = 0;
    ecl_status st = ecl_synchronize(e);
    if (st != ECL_OK) return st;
    if (!e->ran || e->last_mode == MODE_MONO) return ECL_OK;
    const size_t m = std::min<size_t>(e->last_grid, cap);
    if (m) CUDA_OR_FAIL(e, cudaMemcpy(out, e->wst, m * sizeof(ecl_worker_stat), cudaMemcpyDeviceToHost));
    *n = m;
    return ECL_OK;
}

}  // extern "C"

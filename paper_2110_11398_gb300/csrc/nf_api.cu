// nf_api.cu -- the C ABI of libnf (declared in include/nf.h): context
// lifetime, argument checks, CUDA-graph replay of the compute phase, the
// launch-shape autotuner, statistics and the host-buffer end-to-end call.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/nf.h"
#include "nf_ctx.h"
#include "nf_internal.cuh"

using nf::Ctx;

namespace {

thread_local std::string g_init_err;

int fail(Ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    else g_init_err = msg;
    return code;
}

int cuda_fail(Ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
    return fail(c, NF_ECUDA, m);
}

#define NF_CK(ctx, call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (size_t)count);
}

bool is_pow2(double L) {
    int ex;
    const double m = std::frexp(L, &ex);
    return m == 0.5;
}

void release(Ctx *c) {
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    void *bufs[] = {c->boxes_d, c->poff_d, c->keys_a, c->keys_b, c->vals_a, c->vals_b,
                    c->count, c->cell_start, c->scan_tmp, c->sort_status, c->bin_state, c->sorted,
                    c->sorted_d, c->w_sorted, c->nsrc_cell, c->items, c->pencils, c->pencil_ok, c->decomp_d,
                    c->state, c->mom_partial, c->mom_result, c->st_pos, c->st_mass, c->st_acc,
                    c->step_bits};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (c->state_h) cudaFreeHost(c->state_h);
    if (c->mom_h) cudaFreeHost(c->mom_h);
    if (c->step_bits_h) cudaFreeHost(c->step_bits_h);
    if (c->pin_i32) cudaFreeHost(c->pin_i32);
    if (c->g_fwd.exec) cudaGraphExecDestroy(c->g_fwd.exec);
    if (c->g_vjp.exec) cudaGraphExecDestroy(c->g_vjp.exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaStream_t cs : c->cp_streams)
        if (cs) cudaStreamDestroy(cs);
    for (cudaEvent_t ev : c->cp_events)
        if (ev) cudaEventDestroy(ev);
    far_release(c);
    cudaEvent_t evs[] = {c->ev_bin0, c->ev_bin1, c->ev_pair0, c->ev_pair1,
                         c->ev_far[0], c->ev_far[1], c->ev_far[2], c->ev_far[3]};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bool valid_tuning(const nf_tuning &t) {
    const int k = t.sinks_per_lane, w = t.warps_per_block, kv = t.vjp_sinks_per_lane, st = t.source_tile;
    return (k == 1 || k == 2 || k == 4) && (w == 2 || w == 4 || w == 8 || w == 16) &&
           t.blocks_per_sm >= 0 && t.blocks_per_sm <= 32 && (kv == 0 || kv == 1 || kv == 2 || kv == 4) &&
           (st == 0 || st == 64 || st == 128 || st == 256) && (t.use_pencils == 0 || t.use_pencils == 1) &&
           (t.small_items == 0 || t.small_items == 1);
}

int decomp_slot(int K) { return K == 1 ? 0 : (K == 2 ? 1 : 2); }

// Selects the item decomposition for K sinks per lane. Each K has its own
// table (uploaded once, synchronously, so that graphs captured afterwards
// see it), so the forward and adjoint kernels can alternate without copies.
int ensure_decomp(Ctx *c, int K, cudaStream_t s) {
    const int slot = decomp_slot(K);
    if (!(c->decomp_built & (1 << slot))) {
        nf::Decomp h;
        nf::make_decomp(K, &h);
        NF_CK(c, cudaStreamSynchronize(s));
        NF_CK(c, cudaMemcpy(c->decomp_d + slot, &h, sizeof(h), cudaMemcpyHostToDevice));
        c->decomp_built |= 1 << slot;
    }
    c->decomp_k = K;
    return NF_OK;
}

// Sinks per lane of the adjoint kernel.
int vjp_k(const Ctx *c) {
    if (c->precision == NF_PREC_FP64_REF) return 1;
    return c->tune.vjp_sinks_per_lane ? c->tune.vjp_sinks_per_lane : c->tune.sinks_per_lane;
}

// Event record that stays a real (timed) record when `s` is being captured
// into a graph: there it must be an "external" record node, while a stream
// that is not capturing takes the plain form.
cudaError_t record_timing(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e) return e;
    if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    return cudaEventRecord(ev, s);
}

// One host<->device copy of `bytes`, split into four parts on the context's
// copy streams (each part can take its own copy engine), ordered after the
// work already on `s` and before the work enqueued on `s` next.
cudaError_t split_copy(Ctx *c, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
                       cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (!c->cp_streams[0]) {
        for (cudaStream_t &cs : c->cp_streams)
            if (!e) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (cudaEvent_t &ev : c->cp_events)
            if (!e) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e) return e;
    }
    if ((e = cudaEventRecord(c->cp_events[4], s))) return e;
    const size_t part = ((bytes / 4) + 255) & ~size_t(255);
    for (int i = 0; i < 4; ++i) {
        const size_t off = part * i;
        const size_t len = off >= bytes ? 0 : std::min(part, bytes - off);
        if ((e = cudaStreamWaitEvent(c->cp_streams[i], c->cp_events[4], 0))) return e;
        if (len && (e = cudaMemcpyAsync(static_cast<char *>(dst) + off, static_cast<const char *>(src) + off,
                                        len, kind, c->cp_streams[i])))
            return e;
        if ((e = cudaEventRecord(c->cp_events[i], c->cp_streams[i]))) return e;
    }
    for (int i = 0; i < 4; ++i)
        if ((e = cudaStreamWaitEvent(s, c->cp_events[i], 0))) return e;
    return cudaSuccess;
}

// The device address of page-locked host memory (cudaHostAlloc, or
// cudaHostRegister'ed) that the current device can load from and store to,
// else nullptr (pageable memory, device memory, unknown pointers).
void *host_mapped(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return at.devicePointer;
}

// The compute phase: work list, pair kernel, momentum diagnostic and the
// copy of the counters to pinned host memory.
cudaError_t enqueue_forward(Ctx *c, void *acc, int f64, cudaStream_t s, float *dens = nullptr) {
    cudaError_t e;
    if ((e = nf::launch_worklist(c, s, nf::pencils_active(c, c->tune, !dens && !f64),
                                 nf::small_active(c, c->tune, !dens && !f64))))
        return e;
    if ((e = record_timing(c->ev_pair0, s))) return e;
    if ((e = nf::launch_pairs(c, acc, f64, c->tune, s, dens))) return e;
    if ((e = record_timing(c->ev_pair1, s))) return e;
    if ((e = nf::launch_momentum(c, acc, f64, s))) return e;
    if ((e = cudaMemcpyAsync(c->state_h, c->state, sizeof(nf::DevState), cudaMemcpyDeviceToHost, s)))
        return e;
    return cudaMemcpyAsync(c->mom_h, c->mom_result, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
}

cudaError_t enqueue_vjp(Ctx *c, const float *w, float *grad, cudaStream_t s) {
    cudaError_t e;
    if ((e = nf::launch_worklist(c, s))) return e;
    if ((e = record_timing(c->ev_pair0, s))) return e;
    nf_tuning t = c->tune;
    t.sinks_per_lane = vjp_k(c);
    if ((e = nf::launch_vjp(c, w, grad, t, s))) return e;
    if ((e = record_timing(c->ev_pair1, s))) return e;
    return cudaMemcpyAsync(c->state_h, c->state, sizeof(nf::DevState), cudaMemcpyDeviceToHost, s);
}

// Replay `enqueue` from a CUDA graph captured on the private stream; the
// graph is re-captured (and updated in place when possible) whenever `key`
// changes. Captures are thread-local so other threads' work is unaffected.
template <typename F>
cudaError_t run_graph(Ctx *c, nf::GraphSlot &slot, const std::vector<uint64_t> &key, F enqueue,
                      cudaStream_t s) {
    cudaError_t e;
    if (!slot.exec || slot.key != key) {
        if ((e = cudaStreamSynchronize(s))) return e;
        cudaGraph_t g = nullptr;
        const int64_t before = c->launches;
        if ((e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal))) return e;
        cudaError_t ee = enqueue(c->cap_stream);
        e = cudaStreamEndCapture(c->cap_stream, &g);
        slot.n_kernels = c->launches - before;   // captured, not yet run
        c->launches = before;
        if (ee) { if (g) cudaGraphDestroy(g); return ee; }
        if (e) return e;
        bool updated = false;
        if (slot.exec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(slot.exec, g, &info) == cudaSuccess) updated = true;
            else {
                cudaGetLastError();
                cudaGraphExecDestroy(slot.exec);
                slot.exec = nullptr;
            }
        }
        if (!updated) {
            e = cudaGraphInstantiate(&slot.exec, g, 0);
            if (e) { cudaGraphDestroy(g); slot.exec = nullptr; return e; }
        }
        cudaGraphDestroy(g);
        slot.key = key;
    }
    c->launches += slot.n_kernels;
    return cudaGraphLaunch(slot.exec, s);
}

int compute_forward(Ctx *c, void *acc, int f64, cudaStream_t s, float *dens = nullptr) {
    if (!c->binned) return fail(c, NF_ESTATE, "nf_compute_accel: no binned particles (call nf_bin_particles first)");
    if (c->slab && !c->ghosts_ready)
        return fail(c, NF_ESTATE, "nf_compute_accel: slab context without ghosts (call nf_slab_import after binning)");
    if (!acc && c->n > 0) return fail(c, NF_EINVAL, "nf_compute_accel: acc is NULL");
    int rc = ensure_decomp(c, c->precision == NF_PREC_FP64_REF ? 1 : c->tune.sinks_per_lane, s);
    if (rc) return rc;
    cudaError_t e;
    if (c->tune.use_graph) {
        std::vector<uint64_t> key = {(uint64_t)(uintptr_t)acc, (uint64_t)f64, (uint64_t)c->n,
                                     (uint64_t)c->tune.sinks_per_lane, (uint64_t)c->tune.warps_per_block,
                                     (uint64_t)c->tune.blocks_per_sm, (uint64_t)(uintptr_t)c->perm,
                                     (uint64_t)c->equal_mass, (uint64_t)(uintptr_t)dens,
                                     (uint64_t)c->tune.source_tile, (uint64_t)c->tune.use_pencils,
                                     (uint64_t)c->tune.small_items};
        e = run_graph(c, c->g_fwd, key,
                      [&](cudaStream_t cs) { return enqueue_forward(c, acc, f64, cs, dens); }, s);
    } else {
        e = enqueue_forward(c, acc, f64, s, dens);
    }
    if (e) return cuda_fail(c, e, "nf_compute_accel");
    c->have_momentum = 1;
    c->have_pair_time = 1;
    c->last_stream = s;
    return NF_OK;
}

}  // namespace

namespace nf {
// Message of a failing call that has no context (read by nf_last_error(NULL)).
void set_thread_error(const char *msg) { g_init_err = msg ? msg : ""; }
}  // namespace nf

extern "C" {

const char *nf_status_string(int status) {
    switch (status) {
        case NF_OK: return "NF_OK";
        case NF_EINVAL: return "NF_EINVAL";
        case NF_ERANGE: return "NF_ERANGE";
        case NF_ENOMEM: return "NF_ENOMEM";
        case NF_ECUDA: return "NF_ECUDA";
        case NF_ESTATE: return "NF_ESTATE";
        case NF_ETIMEOUT: return "NF_ETIMEOUT";
        default: return "NF_UNKNOWN";
    }
}

const char *nf_last_error(const nf_ctx *ctx) {
    if (!ctx) return g_init_err.c_str();
    return reinterpret_cast<const Ctx *>(ctx)->err.c_str();
}

}  // extern "C"

namespace {

// Context creation for nf_init (slab_nx = 0) and nf_init_slab (one box,
// owned x slabs [slab_x0, slab_x0 + slab_nx) plus R ghost slabs a side).
int init_impl(nf_ctx **out, int device, int n_boxes, const double *box_size, const int *cpd,
              int radius, const double *eps, int softening, int precision, int64_t capacity,
              int slab_x0, int slab_nx) {
    if (!out) return fail(nullptr, NF_EINVAL, "nf_init: out is NULL");
    *out = nullptr;
    if (n_boxes < 1 || n_boxes > (1 << 20))
        return fail(nullptr, NF_EINVAL, "nf_init: n_boxes must be in [1, 2^20]");
    if (!box_size || !cpd || !eps) return fail(nullptr, NF_EINVAL, "nf_init: box_size, cpd and eps are required");
    if (radius < 1 || radius > nf::kMaxRadius)
        return fail(nullptr, NF_EINVAL, "nf_init: radius must be 1, 2 or 3");
    if (softening != NF_SOFT_PLUMMER && softening != NF_SOFT_SPLINE)
        return fail(nullptr, NF_EINVAL, "nf_init: unsupported softening");
    if (precision < NF_PREC_FP32 || precision > NF_PREC_FP32_COMP_PAIR)
        return fail(nullptr, NF_EINVAL, "nf_init: unknown precision");
    if (softening == NF_SOFT_SPLINE && precision != NF_PREC_FP32)
        return fail(nullptr, NF_EINVAL, "nf_init: the spline softening is implemented for NF_PREC_FP32");
    if (capacity < 0 || capacity >= ((int64_t)1 << 31) - 1)
        return fail(nullptr, NF_EINVAL, "nf_init: capacity must be in [0, 2^31 - 1)");
    int64_t n_cells = 0;
    for (int b = 0; b < n_boxes; ++b) {
        if (!(box_size[b] > 0.0) || !std::isfinite(box_size[b]))
            return fail(nullptr, NF_EINVAL, "nf_init: box_size must be finite and > 0");
        if (cpd[b] < 2 * radius + 1 || cpd[b] > 1024)
            return fail(nullptr, NF_EINVAL, "nf_init: cpd must satisfy 2R+1 <= cpd <= 1024");
        if (!(eps[b] > 0.0) || !std::isfinite(eps[b]))
            return fail(nullptr, NF_EINVAL, "nf_init: eps must be finite and > 0");
        n_cells += (int64_t)cpd[b] * cpd[b] * cpd[b];
    }
    if (n_cells >= ((int64_t)1 << 30))
        return fail(nullptr, NF_EINVAL, "nf_init: total cells must stay below 2^30");
    int64_t n_sink_cells = n_cells;
    if (slab_nx > 0) {
        // owned slabs and R ghost slabs on each side; owned cells come first
        n_sink_cells = (int64_t)slab_nx * cpd[0] * cpd[0];
        n_cells = (int64_t)(slab_nx + 2 * radius) * cpd[0] * cpd[0];
    }

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, NF_ECUDA, "nf_init: no such CUDA device");
    }
    Ctx *c = new (std::nothrow) Ctx();
    if (!c) return fail(nullptr, NF_ENOMEM, "nf_init: out of host memory");
    DeviceGuard guard(device);
    c->device = device;
    c->n_boxes = n_boxes;
    c->R = radius;
    c->precision = precision;
    c->softening = softening;
    c->capacity = capacity;
    c->n_cells = n_cells;
    c->n_sink_cells = n_sink_cells;
    c->slab = slab_nx > 0 ? 1 : 0;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    c->pow2_all = 1;
    int64_t off = 0;
    for (int b = 0; b < n_boxes; ++b) {
        nf::BoxDev B{};
        const double L = box_size[b], h = L / cpd[b];
        B.L = L;
        B.cpd_d = (double)cpd[b];
        B.cpd = cpd[b];
        B.cell_off = (int)off;
        B.eps2_d = (eps[b] / h) * (eps[b] / h);
        B.inv_h2_d = 1.0 / (h * h);
        B.inv_h3_d = 1.0 / (h * h * h);
        B.eps2 = (float)B.eps2_d;
        B.inv_h2 = (float)B.inv_h2_d;
        B.inv_h3 = (float)B.inv_h3_d;
        B.Lf = (float)L;
        B.inv_Lf = (float)(1.0 / L);
        B.slab_x0 = slab_x0;
        B.slab_nx = slab_nx;
        if (slab_nx > 0) {
            B.x_lo_add = slab_nx + radius;
            B.x_hi = slab_nx;
            B.x_hi_add = radius;
        } else {
            B.x_lo_add = cpd[b];
            B.x_hi = cpd[b];
            B.x_hi_add = -cpd[b];
        }
        if (softening == NF_SOFT_SPLINE) {
            // pair factor inside eps_s: (10 - 15 u + 6 u^2) / eps_s^3, u = r / eps_s,
            // as c0 + c1 r + c2 r^2 in cell units; s gets a 1e-30 floor instead of eps^2
            const double e = eps[b] / h;
            B.sp_c0 = (float)(10.0 / (e * e * e));
            B.sp_c1 = (float)(-15.0 / (e * e * e * e));
            B.sp_c2 = (float)(6.0 / (e * e * e * e * e));
            B.sp_eps = (float)e;
            B.eps2_d = 0.0;
            B.eps2 = 1e-30f;
        }
        c->boxes_h.push_back(B);
        if (!is_pow2(L)) c->pow2_all = 0;
        off += (int64_t)cpd[b] * cpd[b] * cpd[b];
    }
    const int64_t cap = capacity > 0 ? capacity : 1;
    const int64_t tiles = nf::sort_tiles(cap);
    c->max_tiles = tiles;
    cudaError_t e = cudaSuccess;
#define NF_AL(p, cnt) if (!e) e = dalloc(&(p), (cnt))
    NF_AL(c->boxes_d, n_boxes);
    NF_AL(c->poff_d, n_boxes + 1);
    NF_AL(c->keys_a, cap);
    NF_AL(c->keys_b, cap);
    NF_AL(c->vals_a, cap);
    NF_AL(c->vals_b, cap);
    NF_AL(c->count, n_cells);
    NF_AL(c->cell_start, n_cells + 1);
    NF_AL(c->scan_tmp, nf::scan_tmp_ints(n_cells));
    NF_AL(c->sort_status, tiles * 256);
    NF_AL(c->bin_state, 1);
    NF_AL(c->sorted, cap);
    if (precision == NF_PREC_FP64_REF) NF_AL(c->sorted_d, cap);
    NF_AL(c->w_sorted, cap);
    NF_AL(c->nsrc_cell, n_cells);
    NF_AL(c->items, cap);
    NF_AL(c->pencils, n_cells / nf::kPencil + 1);
    NF_AL(c->pencil_ok, n_cells);
    NF_AL(c->decomp_d, 3);
    NF_AL(c->state, 1);
    NF_AL(c->mom_partial, (int64_t)nf::kMomBlocks * 4);
    NF_AL(c->mom_result, 4);
    NF_AL(c->step_bits, 1);
#undef NF_AL
    if (!e) e = cudaMallocHost(reinterpret_cast<void **>(&c->state_h), sizeof(nf::DevState));
    if (!e) e = cudaMallocHost(reinterpret_cast<void **>(&c->mom_h), 4 * sizeof(double));
    if (!e) e = cudaMallocHost(reinterpret_cast<void **>(&c->step_bits_h), sizeof(unsigned));
    if (!e) e = cudaMallocHost(reinterpret_cast<void **>(&c->pin_i32), 4 * sizeof(int32_t));
    if (!e) e = cudaMemcpy(c->boxes_d, c->boxes_h.data(), sizeof(nf::BoxDev) * n_boxes, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(c->state, 0, sizeof(nf::DevState));
    if (!e) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreate(&c->ev_bin0);
    if (!e) e = cudaEventCreate(&c->ev_bin1);
    if (!e) e = cudaEventCreate(&c->ev_pair0);
    if (!e) e = cudaEventCreate(&c->ev_pair1);
    if (e) {
        const bool oom = e == cudaErrorMemoryAllocation;
        std::string m = std::string("nf_init: ") + cudaGetErrorString(e);
        cudaGetLastError();
        release(c);
        return fail(nullptr, oom ? NF_ENOMEM : NF_ECUDA, m);
    }
    memset(c->state_h, 0, sizeof(nf::DevState));
    // default launch shape: 4 sinks per lane, 4 warps per block (FP32);
    // the compensated variant keeps 2 sinks per lane to stay clear of spills
    c->tune = nf_tuning{4, 4, 0, 1, 2, 0, 1, 1};
    if (precision == NF_PREC_FP32_COMP || precision == NF_PREC_FP32_COMP_PAIR) c->tune.sinks_per_lane = 2;
    if (precision == NF_PREC_FP64_REF) c->tune.sinks_per_lane = 1, c->tune.vjp_sinks_per_lane = 1;
    *out = reinterpret_cast<nf_ctx *>(c);
    return NF_OK;
}

}  // namespace

extern "C" {

int nf_init(nf_ctx **out, int device, int n_boxes, const double *box_size, const int *cpd,
            int radius, const double *eps, int softening, int precision, int64_t capacity) {
    return init_impl(out, device, n_boxes, box_size, cpd, radius, eps, softening, precision, capacity, 0, 0);
}

int nf_init_slab(nf_ctx **out, int device, double box_size, int cpd, int radius, double eps,
                 int softening, int precision, int64_t capacity, int x_begin, int x_count) {
    if (out) *out = nullptr;
    if (radius < 1 || radius > nf::kMaxRadius)
        return fail(nullptr, NF_EINVAL, "nf_init_slab: radius must be 1, 2 or 3");
    if (cpd < 2 * radius + 1 || cpd > 1024)
        return fail(nullptr, NF_EINVAL, "nf_init_slab: cpd must satisfy 2R+1 <= cpd <= 1024");
    if (x_begin < 0 || x_begin >= cpd || x_count < radius || x_count > cpd)
        return fail(nullptr, NF_EINVAL, "nf_init_slab: need 0 <= x_begin < cpd and R <= x_count <= cpd");
    if (precision == NF_PREC_FP64_REF)
        return fail(nullptr, NF_EINVAL, "nf_init_slab: FP32 precisions only (ghost records are FP32)");
    return init_impl(out, device, 1, &box_size, &cpd, radius, &eps, softening, precision, capacity,
                     x_begin, x_count);
}

void nf_free(nf_ctx *ctx) { release(reinterpret_cast<Ctx *>(ctx)); }

namespace {
// nf_bin_particles; with pos_copy (device [n x 3]) the positions may be
// page-locked host memory: the key kernel reads them once and writes the
// device copy that the rest of the binning reads.
int bin_particles(Ctx *c, const float *pos, float *pos_copy, const float *mass, double mass_if_null,
                  int64_t n, const int64_t *box_offsets, cudaStream_t s) {
    c->binned = 0;
    if (n < 0 || n > c->capacity) return fail(c, NF_EINVAL, "nf_bin_particles: n must be in [0, capacity]");
    if (n > 0 && !pos) return fail(c, NF_EINVAL, "nf_bin_particles: pos is NULL");
    if (!mass && c->box_gm.empty() && !(std::isfinite(mass_if_null)))
        return fail(c, NF_EINVAL, "nf_bin_particles: mass_if_null must be finite");
    std::vector<int64_t> poff(c->n_boxes + 1);
    if (c->n_boxes == 1) {
        if (box_offsets && (box_offsets[0] != 0 || box_offsets[1] != n))
            return fail(c, NF_EINVAL, "nf_bin_particles: box_offsets must be {0, n}");
        poff[0] = 0;
        poff[1] = n;
    } else {
        if (!box_offsets) return fail(c, NF_EINVAL, "nf_bin_particles: box_offsets required for n_boxes > 1");
        if (box_offsets[0] != 0 || box_offsets[c->n_boxes] != n)
            return fail(c, NF_EINVAL, "nf_bin_particles: box_offsets must start at 0 and end at n");
        for (int b = 0; b < c->n_boxes; ++b) {
            if (box_offsets[b + 1] < box_offsets[b])
                return fail(c, NF_EINVAL, "nf_bin_particles: box_offsets must be non-decreasing");
            poff[b] = box_offsets[b];
        }
        poff[c->n_boxes] = n;
    }
    if (poff != c->poff_h) {
        NF_CK(c, cudaStreamSynchronize(s));
        NF_CK(c, cudaMemcpy(c->poff_d, poff.data(), sizeof(int64_t) * poff.size(), cudaMemcpyHostToDevice));
        c->poff_h = poff;
    }
    c->equal_mass = mass ? 0 : 1;
    c->m0 = (float)mass_if_null;
    if (!mass) {
        // equal masses: one G m per box (nf_set_box_masses), else mass_if_null
        bool changed = false;
        for (int b = 0; b < c->n_boxes; ++b) {
            const double g = c->box_gm.empty() ? mass_if_null : c->box_gm[b];
            nf::BoxDev &B = c->boxes_h[b];
            if (B.gm_d != (double)(float)g || B.gm != (float)g) {
                B.gm = (float)g;
                B.gm_d = (double)B.gm;
                changed = true;
            }
        }
        if (changed) {
            NF_CK(c, cudaStreamSynchronize(s));
            NF_CK(c, cudaMemcpy(c->boxes_d, c->boxes_h.data(), sizeof(nf::BoxDev) * c->n_boxes,
                                cudaMemcpyHostToDevice));
        }
    }
    NF_CK(c, cudaEventRecord(c->ev_bin0, s));
    cudaError_t e = nf::launch_bin(c, pos, mass, c->m0, n, s, pos_copy);
    if (e) return cuda_fail(c, e, "nf_bin_particles");
    NF_CK(c, cudaEventRecord(c->ev_bin1, s));
    c->have_bin_time = 1;
    NF_CK(c, cudaMemcpyAsync(&c->state_h->error, &c->state->error, sizeof(int), cudaMemcpyDeviceToHost, s));
    NF_CK(c, cudaStreamSynchronize(s));
    c->n = n;
    c->last_stream = s;
    if (c->state_h->error & 2)
        return fail(c, NF_ETIMEOUT, "nf_bin_particles: the cell sort's look-back gave up waiting");
    if (c->state_h->error) {
        return fail(c, NF_ERANGE, "nf_bin_particles: a position component is not finite or outside [0, L)");
    }
    c->binned = 1;
    c->have_momentum = 0;
    c->ghosts_ready = 0;
    c->n_ghost = 0;
    return NF_OK;
}
}  // namespace

int nf_bin_particles(nf_ctx *ctx, const float *pos, const float *mass, double mass_if_null,
                     int64_t n, const int64_t *box_offsets, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_bin_particles: ctx is NULL");
    DeviceGuard guard(c->device);
    return bin_particles(c, pos, nullptr, mass, mass_if_null, n, box_offsets,
                         reinterpret_cast<cudaStream_t>(stream));
}

int nf_set_box_masses(nf_ctx *ctx, const double *gm) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_set_box_masses: ctx is NULL");
    if (!gm) {
        c->box_gm.clear();
        return NF_OK;
    }
    for (int b = 0; b < c->n_boxes; ++b)
        if (!std::isfinite(gm[b])) return fail(c, NF_EINVAL, "nf_set_box_masses: masses must be finite");
    c->box_gm.assign(gm, gm + c->n_boxes);
    return NF_OK;
}

int nf_compute_accel(nf_ctx *ctx, float *acc, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_compute_accel: ctx is NULL");
    DeviceGuard guard(c->device);
    return compute_forward(c, acc, 0, reinterpret_cast<cudaStream_t>(stream));
}

int nf_compute_accel_f64(nf_ctx *ctx, double *acc, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_compute_accel_f64: ctx is NULL");
    DeviceGuard guard(c->device);
    return compute_forward(c, acc, 1, reinterpret_cast<cudaStream_t>(stream));
}

int nf_compute_accel_density(nf_ctx *ctx, float *acc, float *density, const double *kde_b,
                             void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_compute_accel_density: ctx is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (c->precision != NF_PREC_FP32)
        return fail(c, NF_EINVAL, "nf_compute_accel_density: NF_PREC_FP32 contexts only");
    if (!kde_b) return fail(c, NF_EINVAL, "nf_compute_accel_density: kde_b is required");
    if (!c->binned) return fail(c, NF_ESTATE, "nf_compute_accel_density: no binned particles");
    if (c->n > 0 && !density) return fail(c, NF_EINVAL, "nf_compute_accel_density: density is NULL");
    bool changed = false;
    for (int b = 0; b < c->n_boxes; ++b) {
        nf::BoxDev &B = c->boxes_h[b];
        const double h = B.L / B.cpd;
        if (!(kde_b[b] > 0.0) || !(kde_b[b] <= c->R * h))
            return fail(c, NF_EINVAL, "nf_compute_accel_density: kde_b must satisfy 0 < b <= R L / CPD");
        // 1 - r^2/b^2 = kb0 + kb1 s with s = r^2 + eps2 (cell units)
        const double bc2 = (kde_b[b] / h) * (kde_b[b] / h);
        const float kb1 = (float)(-1.0 / bc2);
        const float kb0 = (float)(1.0 + (double)B.eps2 / bc2);
        if (B.kb0 != kb0 || B.kb1 != kb1) { B.kb0 = kb0; B.kb1 = kb1; changed = true; }
    }
    if (changed) {
        NF_CK(c, cudaStreamSynchronize(s));
        NF_CK(c, cudaMemcpy(c->boxes_d, c->boxes_h.data(), sizeof(nf::BoxDev) * c->n_boxes,
                            cudaMemcpyHostToDevice));
    }
    return compute_forward(c, acc, 0, s, density);
}

int nf_compute_accel_vjp(nf_ctx *ctx, const float *w, float *grad_pos, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_compute_accel_vjp: ctx is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!c->binned) return fail(c, NF_ESTATE, "nf_compute_accel_vjp: no binned particles");
    if (c->slab) return fail(c, NF_EINVAL, "nf_compute_accel_vjp: not available on slab contexts");
    if (c->n > 0 && (!w || !grad_pos)) return fail(c, NF_EINVAL, "nf_compute_accel_vjp: w and grad_pos are required");
    const int K = vjp_k(c);
    int rc = ensure_decomp(c, K, s);
    if (rc) return rc;
    cudaError_t e;
    if (c->tune.use_graph) {
        std::vector<uint64_t> key = {(uint64_t)(uintptr_t)w, (uint64_t)(uintptr_t)grad_pos, (uint64_t)c->n,
                                     (uint64_t)K, (uint64_t)c->tune.warps_per_block,
                                     (uint64_t)c->tune.blocks_per_sm, (uint64_t)(uintptr_t)c->perm,
                                     (uint64_t)c->equal_mass};
        e = run_graph(c, c->g_vjp, key, [&](cudaStream_t cs) { return enqueue_vjp(c, w, grad_pos, cs); }, s);
    } else {
        e = enqueue_vjp(c, w, grad_pos, s);
    }
    if (e) return cuda_fail(c, e, "nf_compute_accel_vjp");
    c->have_pair_time = 1;
    c->last_stream = s;
    return NF_OK;
}

int nf_far_init(nf_ctx *ctx, int order, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_far_init: ctx is NULL");
    if (order < 1 || order > 8) return fail(c, NF_EINVAL, "nf_far_init: order must be in [1, 8]");
    if (c->slab) return fail(c, NF_EINVAL, "nf_far_init: not available on slab contexts");
    for (const nf::BoxDev &B : c->boxes_h)
        if (B.cpd > 192) return fail(c, NF_EINVAL, "nf_far_init: CPD above 192 is not supported");
    DeviceGuard guard(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::string err;
    const int rc = far_setup(c, order, s, err);
    if (rc) return fail(c, rc, err);
    return NF_OK;
}

int nf_compute_far(nf_ctx *ctx, float *acc, int accumulate, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_compute_far: ctx is NULL");
    if (!c->far) return fail(c, NF_ESTATE, "nf_compute_far: call nf_far_init first");
    if (!c->binned) return fail(c, NF_ESTATE, "nf_compute_far: no binned particles");
    if (c->n > 0 && !acc) return fail(c, NF_EINVAL, "nf_compute_far: acc is required");
    DeviceGuard guard(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (c->n == 0) return NF_OK;
    for (cudaEvent_t &ev : c->ev_far)
        if (!ev) NF_CK(c, cudaEventCreate(&ev));
    std::string fft_fail;
    cudaError_t e = far_compute(c, acc, accumulate ? 1 : 0, s, fft_fail);
    if (!fft_fail.empty()) return fail(c, NF_ECUDA, "nf_compute_far: " + fft_fail);
    if (e) return cuda_fail(c, e, "nf_compute_far");
    c->have_far_time = 1;
    c->last_stream = s;
    return NF_OK;
}

int nf_kick(nf_ctx *ctx, float *vel, const float *acc, double dt, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_kick: ctx is NULL");
    DeviceGuard guard(c->device);
    if (!c->binned) return fail(c, NF_ESTATE, "nf_kick: no binned particles");
    if (c->n > 0 && (!vel || !acc)) return fail(c, NF_EINVAL, "nf_kick: vel and acc are required");
    if (!std::isfinite(dt)) return fail(c, NF_EINVAL, "nf_kick: dt must be finite");
    cudaError_t e = nf::launch_kick(c, vel, acc, dt, reinterpret_cast<cudaStream_t>(stream));
    return e ? cuda_fail(c, e, "nf_kick") : NF_OK;
}

int nf_drift(nf_ctx *ctx, float *pos, const float *vel, double dt, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_drift: ctx is NULL");
    DeviceGuard guard(c->device);
    if (!c->binned) return fail(c, NF_ESTATE, "nf_drift: no binned particles");
    if (c->n > 0 && (!pos || !vel)) return fail(c, NF_EINVAL, "nf_drift: pos and vel are required");
    if (!std::isfinite(dt)) return fail(c, NF_EINVAL, "nf_drift: dt must be finite");
    cudaError_t e = nf::launch_drift(c, pos, vel, dt, reinterpret_cast<cudaStream_t>(stream));
    return e ? cuda_fail(c, e, "nf_drift") : NF_OK;
}

int nf_timestep(nf_ctx *ctx, const float *vel, const float *acc, double eta, double *dt_out,
                void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_timestep: ctx is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!c->binned) return fail(c, NF_ESTATE, "nf_timestep: no binned particles");
    if (!dt_out || (c->n > 0 && (!vel || !acc)))
        return fail(c, NF_EINVAL, "nf_timestep: vel, acc and dt_out are required");
    if (!(eta > 0.0)) return fail(c, NF_EINVAL, "nf_timestep: eta must be > 0");
    cudaError_t e = nf::launch_cell_timestep(c, vel, acc, c->step_bits, s);
    if (!e) e = cudaMemcpyAsync(c->step_bits_h, c->step_bits, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(c, e, "nf_timestep");
    float r;
    memcpy(&r, c->step_bits_h, sizeof(float));
    *dt_out = r >= 3.0e38f ? INFINITY : eta * (double)r;
    c->last_stream = s;
    return NF_OK;
}

int nf_kdk_step(nf_ctx *ctx, float *pos, float *vel, float *acc, const float *mass,
                double mass_if_null, double dt, const int64_t *box_offsets, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_kdk_step: ctx is NULL");
    DeviceGuard guard(c->device);
    if (!c->binned) return fail(c, NF_ESTATE, "nf_kdk_step: bin the positions and compute acc first");
    if (c->slab)
        return fail(c, NF_EINVAL, "nf_kdk_step: slab contexts exchange ghosts between binning and force; "
                                  "use nf_kick, nf_drift, nf_bin_particles, nf_slab_import, nf_compute_accel");
    const int64_t n = c->n;
    int rc;
    if ((rc = nf_kick(ctx, vel, acc, 0.5 * dt, stream))) return rc;
    if ((rc = nf_drift(ctx, pos, vel, dt, stream))) return rc;
    if ((rc = nf_bin_particles(ctx, pos, mass, mass_if_null, n, box_offsets, stream))) return rc;
    if ((rc = nf_compute_accel(ctx, acc, stream))) return rc;
    if (c->far && (rc = nf_compute_far(ctx, acc, 1, stream))) return rc;   // total force
    return nf_kick(ctx, vel, acc, 0.5 * dt, stream);
}

int nf_accel_host(nf_ctx *ctx, const float *pos_host, const float *mass_host, double mass_if_null,
                  int64_t n, const int64_t *box_offsets, float *acc_host, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_accel_host: ctx is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n < 0 || n > c->capacity) return fail(c, NF_EINVAL, "nf_accel_host: n must be in [0, capacity]");
    if (c->slab) return fail(c, NF_EINVAL, "nf_accel_host: not available on slab contexts");
    if (n > 0 && (!pos_host || !acc_host)) return fail(c, NF_EINVAL, "nf_accel_host: pos_host and acc_host are required");
    if (n > c->st_cap || (mass_host && !c->st_mass)) {
        NF_CK(c, cudaStreamSynchronize(s));
        cudaFree(c->st_pos); cudaFree(c->st_acc); cudaFree(c->st_mass);
        c->st_pos = c->st_acc = c->st_mass = nullptr;
        c->st_cap = 0;
        const int64_t m = n > 0 ? n : 1;
        cudaError_t e = dalloc(&c->st_pos, 3 * m);
        if (!e) e = dalloc(&c->st_acc, 3 * m);
        if (!e) e = dalloc(&c->st_mass, m);
        if (e) { cudaGetLastError(); return fail(c, NF_ENOMEM, "nf_accel_host: staging allocation failed"); }
        c->st_cap = m;
    }
    // Page-locked host buffers that the device can address are read and
    // written by the kernels themselves: the binning's key kernel loads the
    // positions once (and keeps a device copy for the sort's gather), and the
    // pair kernels store each sink's acceleration into acc_host as the pass
    // goes. Other host memory goes through device buffers and copies.
    const float *pos_dev = n > 0 ? static_cast<const float *>(host_mapped(pos_host)) : nullptr;
    float *acc_dev = n > 0 ? static_cast<float *>(host_mapped(acc_host)) : nullptr;
    if (n > 0) {
        if (!pos_dev)
            NF_CK(c, split_copy(c, c->st_pos, pos_host, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
        if (mass_host)
            NF_CK(c, cudaMemcpyAsync(c->st_mass, mass_host, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    }
    int rc = bin_particles(c, pos_dev ? pos_dev : c->st_pos, pos_dev ? c->st_pos : nullptr,
                           mass_host ? c->st_mass : nullptr, mass_if_null, n, box_offsets, s);
    if (rc) return rc;
    rc = nf_compute_accel(ctx, acc_dev ? acc_dev : c->st_acc, stream);
    if (rc) return rc;
    if (n > 0 && !acc_dev)
        NF_CK(c, split_copy(c, acc_host, c->st_acc, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
    NF_CK(c, cudaStreamSynchronize(s));
    return NF_OK;
}

int nf_copy_binning(nf_ctx *ctx, int32_t *cell_start, int32_t *perm, float *sorted, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_copy_binning: ctx is NULL");
    if (!c->binned) return fail(c, NF_ESTATE, "nf_copy_binning: no binned particles");
    DeviceGuard guard(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cell_start)
        NF_CK(c, cudaMemcpyAsync(cell_start, c->cell_start, sizeof(int) * (c->n_cells + 1),
                                 cudaMemcpyDeviceToDevice, s));
    if (c->n > 0 && perm)
        NF_CK(c, cudaMemcpyAsync(perm, c->perm, sizeof(int) * c->n, cudaMemcpyDeviceToDevice, s));
    if (c->n > 0 && sorted)
        NF_CK(c, cudaMemcpyAsync(sorted, c->sorted, sizeof(float4) * c->n, cudaMemcpyDeviceToDevice, s));
    c->last_stream = s;
    return NF_OK;
}

int nf_get_stats(nf_ctx *ctx, nf_stats *out) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !out) return fail(c, NF_EINVAL, "nf_get_stats: ctx and out are required");
    DeviceGuard guard(c->device);
    NF_CK(c, cudaStreamSynchronize(c->last_stream));
    out->n_particles = c->binned ? c->n : 0;
    out->n_cells = c->n_cells;
    out->interactions = (int64_t)c->state_h->interactions;
    out->max_occupancy = c->state_h->max_occ;
    out->n_items = c->state_h->n_items;
    out->n_pencils = c->state_h->n_pencils;
    out->n_small = c->state_h->n_items - c->state_h->n_main;
    for (int a = 0; a < 3; ++a) out->momentum[a] = c->have_momentum ? c->mom_h[a] : 0.0;
    out->abs_momentum = c->have_momentum ? c->mom_h[3] : 0.0;
    float ms = 0.f;
    out->bin_ms = (c->have_bin_time && cudaEventElapsedTime(&ms, c->ev_bin0, c->ev_bin1) == cudaSuccess) ? ms : 0.0;
    ms = 0.f;
    out->pair_ms = (c->have_pair_time && cudaEventElapsedTime(&ms, c->ev_pair0, c->ev_pair1) == cudaSuccess) ? ms : 0.0;
    cudaGetLastError();
    out->kernel_launches = c->launches;
    out->far_ms = out->far_conv_ms = 0.0;
    if (c->have_far_time) {
        if (cudaEventElapsedTime(&ms, c->ev_far[0], c->ev_far[1]) == cudaSuccess) out->far_ms = ms;
        if (cudaEventElapsedTime(&ms, c->ev_far[2], c->ev_far[3]) == cudaSuccess) out->far_conv_ms = ms;
        cudaGetLastError();
    }
    return NF_OK;
}

int nf_set_tuning(nf_ctx *ctx, const nf_tuning *t) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !t) return fail(c, NF_EINVAL, "nf_set_tuning: ctx and t are required");
    if (!valid_tuning(*t)) return fail(c, NF_EINVAL, "nf_set_tuning: sinks_per_lane in {1,2,4}, warps_per_block in {2,4,8,16}, blocks_per_sm in [0,32], vjp_sinks_per_lane in {0,1,2,4}, source_tile in {0,64,128,256}, use_pencils in {0,1}, small_items in {0,1}");
    if (c->precision == NF_PREC_FP64_REF && (t->sinks_per_lane != 1 || t->vjp_sinks_per_lane > 1))
        return fail(c, NF_EINVAL, "nf_set_tuning: FP64 reference contexts use one sink per lane");
    c->tune = *t;
    return NF_OK;
}

int nf_get_tuning(const nf_ctx *ctx, nf_tuning *t) {
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c || !t) return NF_EINVAL;
    *t = c->tune;
    return NF_OK;
}

int nf_autotune(nf_ctx *ctx, int reps, nf_tuning *best, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_autotune: ctx is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!c->binned) return fail(c, NF_ESTATE, "nf_autotune: no binned particles");
    if (c->slab && !c->ghosts_ready) return fail(c, NF_ESTATE, "nf_autotune: slab context without ghosts");
    if (reps < 1) reps = 1;
    std::vector<nf_tuning> cands;
    const int ks[] = {1, 2, 4};
    const int ws[] = {4, 8};
    const bool tiles = c->precision != NF_PREC_FP64_REF && c->softening == NF_SOFT_PLUMMER;
    const int ts[] = {64, 128, 256};
    for (int k : ks) {
        if (c->precision == NF_PREC_FP64_REF && k != 1) continue;
        for (int w : ws)
            for (int st : ts) {
                if (!tiles && st != 128) continue;
                for (int pen = 0; pen < 2; ++pen) {
                    nf_tuning t{k, w, 0, c->tune.use_graph, c->tune.vjp_sinks_per_lane, st, pen,
                                c->tune.small_items};
                    if (pen && !nf::pencils_active(c, t, true)) continue;
                    cands.push_back(t);
                }
            }
    }
    float *acc = nullptr;
    NF_CK(c, dalloc(&acc, 3 * (c->n > 0 ? c->n : 1)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const nf_tuning saved = c->tune;
    float best_ms = 1e30f;
    nf_tuning best_t = saved;
    int rc = NF_OK;
    for (const nf_tuning &t : cands) {
        c->tune = t;
        c->tune.use_graph = 0;
        if ((rc = ensure_decomp(c, t.sinks_per_lane, s))) break;
        const bool pen = nf::pencils_active(c, t, true), sm = nf::small_active(c, t, true);
        cudaError_t e = nf::launch_worklist(c, s, pen, sm);
        if (!e) e = nf::launch_pairs(c, acc, 0, c->tune, s);   // warm-up
        if (e) { rc = cuda_fail(c, e, "nf_autotune"); break; }
        float tot = 0.f;
        for (int r = 0; r < reps && !e; ++r) {
            e = nf::launch_worklist(c, s, pen, sm);
            if (!e) e = cudaEventRecord(e0, s);
            if (!e) e = nf::launch_pairs(c, acc, 0, c->tune, s);
            if (!e) e = cudaEventRecord(e1, s);
            if (!e) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
            tot += ms;
        }
        if (e) { rc = cuda_fail(c, e, "nf_autotune"); break; }
        if (tot < best_ms) { best_ms = tot; best_t = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(acc);
    best_t.use_graph = saved.use_graph;
    c->tune = rc ? saved : best_t;
    if (!rc && best) *best = best_t;
    c->last_stream = s;
    return rc;
}

int nf_slab_export(nf_ctx *ctx, int side, int32_t *counts, float *records, int64_t records_cap,
                   int64_t *n_records, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_slab_export: ctx is NULL");
    if (!c->slab) return fail(c, NF_EINVAL, "nf_slab_export: not a slab context");
    if (side != 0 && side != 1) return fail(c, NF_EINVAL, "nf_slab_export: side must be 0 or 1");
    if (!n_records) return fail(c, NF_EINVAL, "nf_slab_export: n_records is required");
    if (!c->binned) return fail(c, NF_ESTATE, "nf_slab_export: no binned particles");
    DeviceGuard guard(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const nf::BoxDev &B = c->boxes_h[0];
    const int64_t plane = (int64_t)B.cpd * B.cpd, ncell = (int64_t)c->R * plane;
    // owned cells [c0, c0 + ncell): the first R owned slabs (side 0) or the last R (side 1)
    const int64_t c0 = side == 0 ? 0 : (int64_t)(B.slab_nx - c->R) * plane;
    int32_t *h = c->pin_i32;                   // pinned scratch for the two bounds
    NF_CK(c, cudaMemcpyAsync(h, c->cell_start + c0, sizeof(int), cudaMemcpyDeviceToHost, s));
    NF_CK(c, cudaMemcpyAsync(h + 1, c->cell_start + c0 + ncell, sizeof(int), cudaMemcpyDeviceToHost, s));
    NF_CK(c, cudaStreamSynchronize(s));
    const int64_t first = h[0], n = (int64_t)h[1] - h[0];
    *n_records = n;
    if (counts)
        NF_CK(c, cudaMemcpyAsync(counts, c->count + c0, sizeof(int) * ncell, cudaMemcpyDeviceToDevice, s));
    if (records && n > 0) {
        if (n > records_cap) return fail(c, NF_EINVAL, "nf_slab_export: records_cap is below n_records");
        NF_CK(c, cudaMemcpyAsync(records, c->sorted + first, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
    }
    c->last_stream = s;
    return NF_OK;
}

int nf_slab_import(nf_ctx *ctx, const int32_t *left_counts, const float *left_records, int64_t n_left,
                   const int32_t *right_counts, const float *right_records, int64_t n_right, void *stream) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, NF_EINVAL, "nf_slab_import: ctx is NULL");
    if (!c->slab) return fail(c, NF_EINVAL, "nf_slab_import: not a slab context");
    if (!c->binned) return fail(c, NF_ESTATE, "nf_slab_import: bin the owned particles first");
    if (!left_counts || !right_counts || n_left < 0 || n_right < 0 ||
        (n_left > 0 && !left_records) || (n_right > 0 && !right_records))
        return fail(c, NF_EINVAL, "nf_slab_import: both sides' counts, and their records when non-empty, are required");
    if (c->n + n_left + n_right > c->capacity)
        return fail(c, NF_EINVAL, "nf_slab_import: owned plus ghost particles exceed the capacity");
    DeviceGuard guard(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    c->ghosts_ready = 0;
    const nf::BoxDev &B = c->boxes_h[0];
    const int64_t plane = (int64_t)B.cpd * B.cpd, ncell = (int64_t)c->R * plane;
    const int64_t g0 = c->n_sink_cells;        // left ghost cells, then the right ones
    NF_CK(c, cudaMemcpyAsync(c->count + g0, left_counts, sizeof(int) * ncell, cudaMemcpyDeviceToDevice, s));
    NF_CK(c, cudaMemcpyAsync(c->count + g0 + ncell, right_counts, sizeof(int) * ncell,
                             cudaMemcpyDeviceToDevice, s));
    if (n_left > 0)
        NF_CK(c, cudaMemcpyAsync(c->sorted + c->n, left_records, sizeof(float4) * n_left,
                                 cudaMemcpyDeviceToDevice, s));
    if (n_right > 0)
        NF_CK(c, cudaMemcpyAsync(c->sorted + c->n + n_left, right_records, sizeof(float4) * n_right,
                                 cudaMemcpyDeviceToDevice, s));
    NF_CK(c, cudaMemsetAsync(&c->state->error, 0, sizeof(int), s));
    NF_CK(c, nf::launch_check_counts(c->count + g0, 2 * ncell, &c->state->error, s));
    NF_CK(c, nf::scan_exclusive(c->count, c->cell_start, c->n_cells, c->scan_tmp, s, &c->launches));
    // the ghost counts must be non-negative and add up to the records given
    int32_t *h = c->pin_i32;
    NF_CK(c, cudaMemcpyAsync(h, c->cell_start + g0 + ncell, sizeof(int), cudaMemcpyDeviceToHost, s));
    NF_CK(c, cudaMemcpyAsync(h + 1, c->cell_start + c->n_cells, sizeof(int), cudaMemcpyDeviceToHost, s));
    NF_CK(c, cudaMemcpyAsync(&c->state_h->error, &c->state->error, sizeof(int), cudaMemcpyDeviceToHost, s));
    NF_CK(c, cudaStreamSynchronize(s));
    if (c->state_h->error & 4)
        return fail(c, NF_EINVAL, "nf_slab_import: a ghost count is negative");
    if ((int64_t)h[0] != c->n + n_left || (int64_t)h[1] != c->n + n_left + n_right)
        return fail(c, NF_EINVAL, "nf_slab_import: the ghost counts do not add up to n_left and n_right");
    c->n_ghost = n_left + n_right;
    c->ghosts_ready = 1;
    c->last_stream = s;
    return NF_OK;
}

int nf_slab_of(const float *pos, int64_t n, double box_size, int cpd, int32_t *slab, void *stream) {
    if (n < 0 || (n > 0 && (!pos || !slab)))
        return fail(nullptr, NF_EINVAL, "nf_slab_of: pos and slab are required for n > 0");
    if (!(box_size > 0.0) || !std::isfinite(box_size) || cpd < 1 || cpd > 1024)
        return fail(nullptr, NF_EINVAL, "nf_slab_of: box_size must be finite and > 0, 1 <= cpd <= 1024");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, NF_ECUDA, "nf_slab_of: no usable current CUDA device");
    }
    nf::BoxDev B{};
    B.L = box_size;
    B.cpd_d = (double)cpd;
    B.cpd = cpd;
    B.Lf = (float)box_size;
    B.inv_Lf = (float)(1.0 / box_size);
    cudaError_t e = nf::launch_slab_of(pos, n, B, is_pow2(box_size) ? 1 : 0, sms, slab,
                                       reinterpret_cast<cudaStream_t>(stream));
    if (e) {
        cudaGetLastError();
        return fail(nullptr, NF_ECUDA, std::string("nf_slab_of: ") + cudaGetErrorString(e));
    }
    return NF_OK;
}

}  // extern "C"

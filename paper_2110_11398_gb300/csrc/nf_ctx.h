// nf_ctx.h -- host-side context of libnf (one per nf_init).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nf_internal.cuh"

namespace nf {

struct FarState;   // far-field state (nf_far.cu)

// A captured phase of work replayed as a CUDA graph; `key` holds the
// arguments baked into the capture.
struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    std::vector<uint64_t> key;
    int64_t n_kernels = 0;        // kernels per replay
};

struct Ctx {
    int device = 0;
    int n_boxes = 0;
    int R = 2;
    int precision = NF_PREC_FP32;
    int softening = NF_SOFT_PLUMMER;
    int64_t capacity = 0;
    int64_t n_cells = 0;          // total over boxes (a slab context: owned and ghost cells)
    int64_t n_sink_cells = 0;     // cells whose particles are sinks (all but a slab context's ghosts)
    int slab = 0;                 // 1: a slab context (one box, owned x slabs + R ghost slabs a side)
    int ghosts_ready = 0;         // slab context: ghosts imported since the last binning
    int64_t n_ghost = 0;          // slab context: ghost records behind the owned ones
    int sm_count = 0;
    int pow2_all = 0;             // every box side is a power of two

    std::vector<BoxDev> boxes_h;
    BoxDev *boxes_d = nullptr;
    int64_t *poff_d = nullptr;    // particle offsets per box [n_boxes+1]
    std::vector<int64_t> poff_h;

    // binning
    int *keys_a = nullptr, *keys_b = nullptr;     // [capacity]
    int *vals_a = nullptr, *vals_b = nullptr;     // [capacity]
    int *perm = nullptr;                           // alias of the final values buffer
    int *count = nullptr;                          // [n_cells]
    int *cell_start = nullptr;                     // [n_cells + 1]
    int *scan_tmp = nullptr;                       // block sums of the scans
    unsigned long long *sort_status = nullptr;     // [256 * max_tiles] look-back words of the sort
    BinState *bin_state = nullptr;                 // digit histograms and tile counters
    unsigned bin_epoch = 0;                        // tag of the next sort pass (0: words not yet cleared)
    int64_t max_tiles = 0;
    float4 *sorted = nullptr;                      // [capacity] (rx, ry, rz, m)
    dbl4 *sorted_d = nullptr;                   // [capacity] FP64 copy (FP64_REF only)
    float4 *w_sorted = nullptr;                    // [capacity] VJP cotangent, sorted

    // work list
    int *nsrc_cell = nullptr;                      // [n_cells]
    WorkItem *items = nullptr;                     // [capacity]
    int *pencils = nullptr;                        // [n_cells / kPencil + 1] first cell of each pencil item
    unsigned char *pencil_ok = nullptr;            // [n_cells] at a pencil's first cell: served as a pencil
    Decomp *decomp_d = nullptr;                    // [3]: tables for K = 1, 2, 4
    int decomp_built = 0;                          // bit i: table i uploaded
    int decomp_k = 0;                              // K of the next work list
    DevState *state = nullptr;
    DevState *state_h = nullptr;                   // pinned mirror

    // momentum diagnostic
    double *mom_partial = nullptr;                 // [kMomBlocks * 4]
    double *mom_result = nullptr;                  // [4]
    double *mom_h = nullptr;                       // pinned [4]
    unsigned *step_bits = nullptr;                 // [1] timestep criterion (float bits)
    unsigned *step_bits_h = nullptr;               // pinned mirror
    int32_t *pin_i32 = nullptr;                    // pinned [4]: small reads of cell_start

    // last binning
    int64_t n = 0;
    int binned = 0;
    int equal_mass = 1;
    float m0 = 0.f;
    std::vector<double> box_gm;                    // per-box G m (nf_set_box_masses), empty = unset
    int have_momentum = 0;

    nf_tuning tune{4, 4, 0, 1, 2};
    cudaStream_t cap_stream = nullptr;             // private capture stream
    GraphSlot g_fwd, g_vjp;
    cudaStream_t last_stream = nullptr;

    // host-buffer staging for nf_accel_host
    float *st_pos = nullptr, *st_mass = nullptr, *st_acc = nullptr;
    int64_t st_cap = 0;
    cudaStream_t cp_streams[4] = {nullptr, nullptr, nullptr, nullptr};   // split host copies
    cudaEvent_t cp_events[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

    // timing of the last binning / pair kernel, and the launch counter
    cudaEvent_t ev_bin0 = nullptr, ev_bin1 = nullptr, ev_pair0 = nullptr, ev_pair1 = nullptr;
    cudaEvent_t ev_far[4] = {nullptr, nullptr, nullptr, nullptr};   // far step, convolution (start, end)
    int have_far_time = 0;
    int64_t launches = 0;
    int have_bin_time = 0, have_pair_time = 0;

    FarState *far = nullptr;                       // far field (nf_far_init), one-box contexts

    std::string err;
};

// far field (nf_far.cu)
int far_setup(Ctx *c, int order, cudaStream_t s, std::string &err);
cudaError_t far_compute(Ctx *c, float *acc, int accumulate, cudaStream_t s, std::string &fft_fail);
void far_release(Ctx *c);

constexpr int kMomBlocks = 512;

}  // namespace nf

// nf_internal.cuh -- device-side structures and helpers shared by the libnf
// translation units (binning, work list, pair kernels, C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nf.h"

namespace nf {

// Largest supported near-field radius (neighbourhood of (2R+1)^3 cells).
constexpr int kMaxRadius = 3;
constexpr int kMaxNbr = (2 * kMaxRadius + 1) * (2 * kMaxRadius + 1) * (2 * kMaxRadius + 1);
// Sources staged per warp tile.
constexpr int kTile = 128;
// Pencils (k_pencils): kPencil z-consecutive cells of one (x, y) row served
// by one block of kPencil warps that share every staged column of sources;
// each warp takes the first kPencilSinks sinks of its cell (the rest make
// ordinary items), and a column (the pencil's cells plus R on either side in
// z, at one (dx, dy)) holds at most kColMax sources (odd counts padded to
// even).
constexpr int kPencil = 4;
constexpr int kPencilSinks = 64;
constexpr int kColMax = 768;
// Number of cost buckets of the work list (heaviest items are served first).
constexpr int kBuckets = 64;
// Items whose lanes split the sources at least 1 << kSmallLog2S ways (at most
// 8 sinks with 4 sinks per lane) over at most kSmallMaxSrc sources go to the
// small-item kernel when it is on. Heavier ones (the last sinks of dense
// cells) stay with the tiled kernel, whose cost order starts them early; run
// after it, one of them would be a serial tail.
constexpr int kSmallLog2S = 4;
constexpr int kSmallMaxSrc = 32768;
// Max items one remainder of a cell can be cut into (see make_decomp()).
constexpr int kDecompMax = 8;

// Cell sort (nf_bin.cu): threads per tile, keys per thread, keys per tile,
// and the most 8-bit digit passes a cell id can need (ids stay below 2^31).
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kMaxSortPasses = 4;

// Device counters of one binning: the digit histogram of every radix pass
// (counted with the cell ids) and each pass's dynamic tile counter.
struct BinState {
    int hist[kMaxSortPasses][256];
    int tile_ctr[kMaxSortPasses];
};

// Four doubles, 32-byte aligned (cell-sorted FP64 record x, y, z, m).
struct __align__(32) dbl4 {
    double x, y, z, w;
};
__host__ __device__ __forceinline__ dbl4 dbl4_make(double x, double y, double z, double w) {
    dbl4 r;
    r.x = x; r.y = y; r.z = z; r.w = w;
    return r;
}

// Per-box constants. Coordinates inside the library are in cell units
// (h = L / CPD = 1); the epilogue scales back to the caller's units.
struct BoxDev {
    double L;          // box side (caller units)
    double cpd_d;      // CPD as double (binning arithmetic)
    double eps2_d;     // (eps / h)^2
    double inv_h2_d;   // 1 / h^2
    double inv_h3_d;   // 1 / h^3
    int cpd;           // cells per dimension
    int cell_off;      // global id of this box's first cell
    float eps2;        // (eps / h)^2, FP32 (spline law: a 1e-30 floor, see k_pairs)
    float inv_h2;      // 1 / h^2, FP32
    float inv_h3;      // 1 / h^3, FP32
    float sp_c0, sp_c1, sp_c2;   // spline law inside eps_s: f = c0 + c1 r + c2 r^2 (cell units)
    float sp_eps;                // eps_s in cell units (branch test of the spline adjoint)
    float kb0, kb1;    // density weight 1 - r^2/b^2 written as kb0 + kb1 s
    float gm;          // G m of every particle of this box when no mass array is given
    float Lf;          // L as float (exact when L is a power of two)
    float inv_Lf;      // 1 / L as float (exact when L is a power of two)
    double gm_d;       // same G m, double
    int slab_x0;       // slab contexts: first owned x slab (global index)
    int slab_nx;       // slab contexts: owned x slabs; 0 for a whole periodic box
    // x index map of neighbour rows (xwrap): t + (t < 0 ? x_lo_add : 0) +
    // (t >= x_hi ? x_hi_add : 0). A whole box wraps periodically (CPD, CPD,
    // -CPD). A slab context keeps its owned slabs at local x 0..nx-1, then the
    // R ghost slabs on its left (global x0-R..x0-1) at nx..nx+R-1 and the R on
    // its right (global x0+nx..x0+nx+R-1) at nx+R..nx+2R-1 (nx+R, nx, R), so
    // an owned sink's neighbours never wrap.
    int x_lo_add, x_hi, x_hi_add;
};

// Local x index of the cell row at x offset t (owned/sink x plus dx).
__device__ __forceinline__ int xwrap(const BoxDev &B, int t) {
    return t + (t < 0 ? B.x_lo_add : 0) + (t >= B.x_hi ? B.x_hi_add : 0);
}

// One unit of pair work: `n` consecutive cell-sorted sinks of one cell,
// processed by one warp whose lanes are split `1 << log2s` ways over sources.
struct __align__(16) WorkItem {
    int cell;      // global cell id of the sinks
    int first;     // first sorted slot of the sinks
    int n;         // number of sinks (<= 32 * K >> log2s)
    int box_s;     // (box << 8) | log2s
};

// Device-resident counters of one context.
struct DevState {
    int error;                   // bit 0: a position outside [0, L) or not finite;
                                 // bit 1: the cell sort's look-back gave up waiting
    int n_items;                 // items written by the last work-list build
    int queue_head;              // persistent-kernel work counter
    int max_occ;                 // largest cell population
    unsigned long long interactions;
    int n_pencils;               // pencil items of the last work-list build
    int pencil_head;             // pencil kernel work counter
    int n_main;                  // items [0, n_main) for the tiled kernels, the rest small items
    int small_head;              // small-item kernel work counter
    int bucket_count[2 * kBuckets];   // cost buckets; the upper half holds the small items
    int bucket_cursor[2 * kBuckets];
};

// Decomposition of a cell's remainder of sinks into items: entry r lists
// (count, log2s) pairs; see make_decomp() in nf_pairs.cu.
struct Decomp {
    int n_entries[128];
    int entry[128][kDecompMax];  // (count << 8) | log2s
};

// ------------------------------------------------------------ packed FP32
// Blackwell executes two FP32 lanes per instruction with the .f32x2 forms
// (PTX ISA 8.6+, sm_100a family). A packed value is a 64-bit register pair
// {lo, hi}.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// Hardware reciprocal square root (MUFU), flush-to-zero: the PTX
// rsqrt.approx.ftz.f32 instruction.
__device__ __forceinline__ float rsqrt_hw(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ f2_t f2_min(f2_t a, f2_t b) {
    float a0, a1, b0, b1;
    f2_unpack(a, a0, a1);
    f2_unpack(b, b0, b1);
    return f2_pack(fminf(a0, b0), fminf(a1, b1));
}
__device__ __forceinline__ f2_t f2_max0(f2_t a) {
    float a0, a1;
    f2_unpack(a, a0, a1);
    return f2_pack(fmaxf(a0, 0.f), fmaxf(a1, 0.f));
}
__device__ __forceinline__ f2_t f2_rsqrt(f2_t v) {
    float a, b;
    f2_unpack(v, a, b);
    return f2_pack(rsqrt_hw(a), rsqrt_hw(b));
}

// The box of input particle i: the last b with poff[b] <= i.
__device__ __forceinline__ int box_of_particle(const int64_t *poff, int n_boxes, int64_t i) {
    int lo = 0, hi = n_boxes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (poff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int box_of_cell(const BoxDev *boxes, int n_boxes, int cell) {
    int lo = 0, hi = n_boxes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].cell_off <= cell) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace nf

// Host-side entry points of each translation unit (C++ linkage, internal).
namespace nf {
struct Ctx;
// pos_copy (optional, device [n x 3]): the key kernel also writes the positions
// there as it reads them (pos may then be page-locked host memory), and the
// sort's gather reads the copy.
cudaError_t launch_bin(Ctx *c, const float *pos, const float *mass, float m0, int64_t n,
                       cudaStream_t s, float *pos_copy = nullptr);
cudaError_t launch_worklist(Ctx *c, cudaStream_t s, bool pencils = false, bool small = false);
bool pencils_active(const Ctx *c, const nf_tuning &t, bool density);
bool small_active(const Ctx *c, const nf_tuning &t, bool plain_out);
cudaError_t launch_pairs(Ctx *c, void *acc, int out_f64, const nf_tuning &t, cudaStream_t s,
                         float *dens = nullptr);
cudaError_t launch_vjp(Ctx *c, const float *w, float *grad, const nf_tuning &t, cudaStream_t s);
cudaError_t launch_momentum(Ctx *c, const void *acc, int acc_f64, cudaStream_t s);
cudaError_t launch_slab_of(const float *pos, int64_t n, const BoxDev &B, int pow2, int sm_count,
                           int32_t *slab, cudaStream_t s);
cudaError_t launch_check_counts(const int *count, int64_t n, int *error_word, cudaStream_t s);
void make_decomp(int k, Decomp *d);
cudaError_t launch_kick(Ctx *c, float *vel, const float *acc, double h, cudaStream_t s);
cudaError_t launch_drift(Ctx *c, float *pos, const float *vel, double dt, cudaStream_t s);
cudaError_t launch_cell_timestep(Ctx *c, const float *vel, const float *acc, unsigned *best_bits,
                                 cudaStream_t s);
cudaError_t scan_exclusive(const int *in, int *out, int64_t n, int *tmp, cudaStream_t s,
                           int64_t *launches);
int64_t scan_tmp_ints(int64_t n);
int64_t sort_tiles(int64_t n);
int sort_passes(int64_t n_cells);
}  // namespace nf

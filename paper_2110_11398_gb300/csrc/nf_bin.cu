// nf_bin.cu -- cell binning (the cubic cell lattice of Maksimova et al. 2021,
// Sec. 3.1): per-particle cell id, stable sort by cell and the cell-sorted
// float4 records of cell-relative coordinates, then per-cell counts and the
// exclusive prefix scan cell_start.
//
// Cell arithmetic, identical on every device and host: u = (x * CPD) / L in
// IEEE double with no contraction, cell = floor(u) (CPD rounds down to
// CPD-1), relative coordinate float32(u - (cell + 0.5)) in cell units.
//
// The sort is a least-significant-digit radix sort on the cell id with
// 8-bit digits, one kernel per digit ("one sweep"): a tile of 4096 keys ranks
// its keys by digit in input order (match_any within a warp, warps in
// order), learns where each digit's run starts in the output from the tiles
// before it by a decoupled look-back over per-tile digit counts, and writes
// its keys digit-run by digit-run through shared memory, so the stores are
// coalesced. The digit histograms of every pass are counted once, in the
// kernel that computes the cell ids. The last pass writes the cell-sorted
// records (reading each particle's position at its input index) instead of
// the sort values, so no separate gather pass is needed, and counts each
// cell's particles from the runs of equal keys in its tile.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>

#include "nf_ctx.h"
#include "nf_internal.cuh"

namespace nf {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;                       // per thread
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kDigits = 256;
static_assert(kSortThreads == kDigits, "one thread per digit in the per-digit steps");
// Look-back spin limit: a tile waits for a predecessor's count at most this
// many polls (with a short sleep between polls), then flags an error and
// goes on; the host turns the flag into NF_ETIMEOUT.
constexpr unsigned kSpinLimit = 1u << 22;

// u = (x * CPD) / L. When L is a power of two the division is exact and
// equals multiplication by 1/L, which avoids the FP64 divide.
__device__ __forceinline__ double cell_unit(double x, const BoxDev &B, bool pow2) {
    double p = __dmul_rn(x, B.cpd_d);
    return pow2 ? __dmul_rn(p, (double)B.inv_Lf) : __ddiv_rn(p, B.L);
}

__device__ __forceinline__ int cell_index(double u, int cpd) {
    int c = (int)floor(u);
    return c >= cpd ? cpd - 1 : c;
}

// The same cell and cell-relative coordinate in FP32 when L is a power of
// two (FP64 is slow on this GPU). x*CPD = p + e exactly (e from an fma), and
// scaling by 1/L = 2^-k is exact, so u = p + e. floor(u) is floor(p), less
// one when p is an integer and e < 0. Then p - (c + 1/2) is exact (Sterbenz:
// both within a factor of two) when c >= 1 or p >= 1/4, and adding e rounds
// once: the result equals float32(u - (c + 1/2)) formed in double. Returns
// false (the caller then uses the FP64 path) outside those conditions; they
// also keep p >= 1/4, so e is never subnormal.
__device__ __forceinline__ bool cell_rel_pow2(float x, float cpd_f, float inv_L, int cpd, int &c,
                                              float &r) {
    float p = x * cpd_f;
    float e = fmaf(x, cpd_f, -p);
    p *= inv_L;
    e *= inv_L;
    float fl = floorf(p);
    int ci = (int)fl;
    if (fl == p && e < 0.f) ci -= 1;
    if (ci >= cpd) return false;
    if (!(ci >= 1 || p >= 0.25f)) return false;
    c = ci;
    r = __fadd_rn(__fsub_rn(p, (float)ci + 0.5f), e);
    return true;
}

// a1: the global cell id of a particle with coordinates x[3] in box B; ok is
// false for a component outside [0, L) or not finite (false for NaN), and
// such a particle goes to the box's first cell.
__device__ __forceinline__ int particle_cell(const float x[3], const BoxDev &B, int pow2, bool &ok) {
    int c3[3];
    ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xf = x[a];
        // for a power-of-two L, L is a float and the test is exact in FP32
        const bool in = pow2 ? (xf >= 0.f && xf < B.Lf) : ((double)xf >= 0.0 && (double)xf < B.L);
        ok = ok && in;
        int cc = 0;
        float rr;
        if (in && !(pow2 && cell_rel_pow2(xf, (float)B.cpd, B.inv_Lf, B.cpd, cc, rr)))
            cc = cell_index(cell_unit((double)xf, B, pow2 != 0), B.cpd);
        c3[a] = cc;
    }
    if (B.slab_nx > 0) {           // slab context: local x slab; other slabs are not owned
        int lx = c3[0] - B.slab_x0;
        if (lx < 0) lx += B.cpd;
        if (lx >= B.slab_nx) {
            ok = false;
            lx = 0;
        }
        c3[0] = lx;
    }
    return B.cell_off + (c3[0] * B.cpd + c3[1]) * B.cpd + c3[2];
}

// a5: cell-relative coordinates of a particle (cell units) as float, and as
// double for the FP64 reference records.
__device__ __forceinline__ void particle_rel(const float x[3], const BoxDev &B, int pow2, bool want_d,
                                             float rf[3], double rd[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xf = x[a];
        const double xd = (double)xf;
        const bool in = pow2 ? (xf >= 0.f && xf < B.Lf) : (xd >= 0.0 && xd < B.L);
        int c;
        float r32;
        if (in && !want_d && pow2 && cell_rel_pow2(xf, (float)B.cpd, B.inv_Lf, B.cpd, c, r32)) {
            rf[a] = r32;
            rd[a] = (double)r32;
        } else {
            const double u = in ? cell_unit(xd, B, pow2 != 0) : 0.5;
            c = in ? cell_index(u, B.cpd) : 0;
            rd[a] = __dsub_rn(u, (double)c + 0.5);
            rf[a] = __double2float_rn(rd[a]);
        }
    }
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// ------------------------------------------------------------ scan
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ int block_excl_scan(int v, int &excl) {
    __shared__ int warp_tot[32];
    __shared__ int block_tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? warp_tot[lane] : 0;
        int ti = warp_incl_scan(t);
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == 31) block_tot = ti;     // lane 31 holds the inclusive total
    }
    __syncthreads();
    excl = warp_tot[warp] + inc - v;
    int total = block_tot;
    __syncthreads();
    return total;
}

__global__ void k_scan_reduce(const int *__restrict__ in, int64_t n, int *__restrict__ block_sum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    int excl;
    int tot = block_excl_scan(s, excl);
    if (threadIdx.x == 0) block_sum[blockIdx.x] = tot;
}

// One block scans up to kScanThreads * 8 block sums in place; writes the
// grand total to *total.
__global__ void k_scan_blocks(int *__restrict__ block_sum, int nb, int *__restrict__ total) {
    constexpr int P = 8;
    int v[P];
    int s = 0;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        int idx = threadIdx.x * P + k;
        v[k] = idx < nb ? block_sum[idx] : 0;
        s += v[k];
    }
    int excl;
    int tot = block_excl_scan(s, excl);
#pragma unroll
    for (int k = 0; k < P; ++k) {
        int idx = threadIdx.x * P + k;
        if (idx < nb) block_sum[idx] = excl;
        excl += v[k];
    }
    if (threadIdx.x == 0) *total = tot;
}

__global__ void k_scan_apply(const int *__restrict__ in, int64_t n,
                             const int *__restrict__ block_off, int *__restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int excl;
    block_excl_scan(s, excl);
    excl += block_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = excl;
        excl += v[k];
    }
}

// ------------------------------------------------------------ cell ids + digit counts
constexpr int kKeyThreads = 256;
constexpr int kKeyPer = 4;                              // particles per thread per chunk
constexpr int kKeyChunk = kKeyThreads * kKeyPer;        // 1024 particles, 12 KB of positions

// a1 for every particle (cell id into cid, range check), and the 8-bit digit
// histograms of all `passes` radix passes (block-private in shared memory,
// then added to the global counts). A block copies a chunk of 1024
// positions into shared memory with coalesced 16-byte loads, then each
// thread takes four particles from there.
template <bool COPY>
__global__ void __launch_bounds__(kKeyThreads) k_cell_keys(const float *__restrict__ pos, int64_t n,
                                                           const int64_t *__restrict__ poff, int n_boxes,
                                                           const BoxDev *__restrict__ boxes, int pow2,
                                                           int passes, int *__restrict__ cid, BinState *bs,
                                                           DevState *st, float *__restrict__ pos_copy) {
    __shared__ __align__(16) float sp[3 * kKeyChunk];
    __shared__ int h[kMaxSortPasses][kDigits];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int t = tid; t < kMaxSortPasses * kDigits; t += kKeyThreads) (&h[0][0])[t] = 0;
    bool bad = false;
    for (int64_t c0 = (int64_t)blockIdx.x * kKeyChunk; c0 < n; c0 += (int64_t)gridDim.x * kKeyChunk) {
        const int cnt = (int)min((int64_t)kKeyChunk, n - c0);
        const float *src = pos + 3 * c0;
        __syncthreads();                       // previous chunk consumed
        float *dst = COPY ? pos_copy + 3 * c0 : nullptr;        // the device copy
        if (cnt == kKeyChunk && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
            const float4 *s4 = reinterpret_cast<const float4 *>(src);
            float4 *d4 = reinterpret_cast<float4 *>(sp);
            float4 *c4 = reinterpret_cast<float4 *>(dst);
            for (int t = tid; t < 3 * kKeyChunk / 4; t += kKeyThreads) {
                const float4 v = s4[t];
                d4[t] = v;
                if (COPY) c4[t] = v;
            }
        } else {
            for (int t = tid; t < 3 * cnt; t += kKeyThreads) {
                const float v = src[t];
                sp[t] = v;
                if (COPY) dst[t] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kKeyPer; ++u) {
            const int j = tid + u * kKeyThreads;
            const bool live = j < cnt;
            int cell = 0;
            if (live) {
                const int64_t i = c0 + j;
                const int b = n_boxes == 1 ? 0 : box_of_particle(poff, n_boxes, i);
                const float x[3] = {sp[3 * j], sp[3 * j + 1], sp[3 * j + 2]};
                bool ok;
                cell = particle_cell(x, boxes[b], pow2, ok);
                bad = bad || !ok;
                cid[i] = cell;
            }
            // the digit histograms of every pass: the lanes of one digit are
            // counted by one add
            const unsigned live_mask = __ballot_sync(0xffffffffu, live);
            if (live_mask) {
                for (int p = 0; p < passes; ++p) {
                    const int d = (cell >> (8 * p)) & 0xff;
                    if (live) {
                        const unsigned peers = __match_any_sync(live_mask, d);
                        if (lane == __ffs(peers) - 1) atomicAdd(&h[p][d], __popc(peers));
                    }
                }
            }
        }
    }
    if (bad) atomicOr(&st->error, 1);
    __syncthreads();
    for (int t = tid; t < passes * kDigits; t += kKeyThreads) {
        const int v = (&h[0][0])[t];
        if (v) atomicAdd(&bs->hist[t / kDigits][t % kDigits], v);
    }
}

// ------------------------------------------------------------ one radix pass
struct SortArgs {
    const int *keys_in;
    const int *vals_in;            // nullptr: values are the input indices (first pass)
    int *keys_out;
    int *vals_out;                 // last pass: the permutation (sorted slot -> input index)
    int64_t n;
    int shift;
    int pass;
    unsigned epoch;                // tags this pass's look-back words (unique per pass)
    unsigned long long *status;    // [tiles][kDigits] look-back words
    BinState *bs;
    DevState *st;
    // last pass: the cell-sorted records
    const float *pos;
    const float *mass;             // nullptr: per-box G m
    const int64_t *poff;
    int n_boxes;
    const BoxDev *boxes;
    int pow2;
    float4 *sorted;
    dbl4 *sorted_d;                // FP64 copy (FP64 reference contexts) or nullptr
    int *count;                    // per-cell counts, zero on entry to the last pass
};

// Look-back word of (tile, digit): high 32 bits 2 * epoch (the tile's own
// count of that digit is published) or 2 * epoch + 1 (the inclusive count of
// all tiles up to it is published), low 32 bits the count. Words of an
// earlier pass carry another epoch and read as "not yet published".
template <bool LAST>
__global__ void __launch_bounds__(kSortThreads, 3) k_sort_pass(SortArgs a) {
    __shared__ int s_key[kSortTile];
    __shared__ int s_val[kSortTile];
    __shared__ int s_wcnt[kSortWarps][kDigits];
    __shared__ int s_dstart[kDigits];
    __shared__ int s_gbase[kDigits];
    __shared__ int s_tile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&a.bs->tile_ctr[a.pass], 1);
    for (int t = tid; t < kSortWarps * kDigits; t += kSortThreads) (&s_wcnt[0][0])[t] = 0;
    // global start of each digit's output run: exclusive scan of the pass's
    // digit histogram
    int goff;
    block_excl_scan(a.bs->hist[a.pass][tid], goff);
    const int64_t tile = s_tile;
    const int64_t t0 = tile * kSortTile;
    const int64_t base = t0 + warp * (32 * kSortItems);
    int key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
    for (int c = 0; c < kSortItems; ++c) {
        const int64_t idx = base + c * 32 + lane;
        const bool live = idx < a.n;
        key[c] = live ? a.keys_in[idx] : 0;
        val[c] = live ? (a.vals_in ? a.vals_in[idx] : (int)idx) : 0;
    }
    // rank of each key among the warp's keys of the same digit, in input order
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int c = 0; c < kSortItems; ++c) {
        const bool live = base + c * 32 + lane < a.n;
        const int d = live ? ((key[c] >> a.shift) & 0xff) : (0x100 + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        int r = 0;
        if (live) r = s_wcnt[warp][d] + __popc(peers & lt);
        __syncwarp();
        if (live && lane == __ffs(peers) - 1) s_wcnt[warp][d] += __popc(peers);
        __syncwarp();
        rank[c] = r;
    }
    __syncthreads();
    // thread tid = digit: warps' exclusive prefix of that digit and the tile's count
    int cnt = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        const int t = s_wcnt[w][tid];
        s_wcnt[w][tid] = cnt;
        cnt += t;
    }
    int dstart;
    block_excl_scan(cnt, dstart);
    s_dstart[tid] = dstart;
    // publish this tile's count of digit tid, then look back over the
    // predecessors until one publishes an inclusive count
    const unsigned hiA = 2u * a.epoch, hiP = 2u * a.epoch + 1u;
    unsigned long long *mine = a.status + tile * kDigits + tid;
    unsigned excl = 0;
    if (tile == 0) {
        st_relaxed(mine, ((unsigned long long)hiP << 32) | (unsigned)cnt);
    } else {
        st_relaxed(mine, ((unsigned long long)hiA << 32) | (unsigned)cnt);
        int64_t p = tile - 1;
        while (true) {
            const unsigned long long *w = a.status + p * kDigits + tid;
            unsigned long long v = ld_relaxed(w);
            unsigned hi = (unsigned)(v >> 32);
            unsigned spins = 0;
            while (hi != hiA && hi != hiP) {
                if (++spins >= kSpinLimit) break;
                if (spins > 16) __nanosleep(100);
                v = ld_relaxed(w);
                hi = (unsigned)(v >> 32);
            }
            if (hi != hiA && hi != hiP) {       // gave up: flag it and go on
                atomicOr(&a.st->error, 2);
                break;
            }
            excl += (unsigned)v;
            if (hi == hiP || p == 0) break;
            --p;
        }
        st_relaxed(mine, ((unsigned long long)hiP << 32) | (excl + (unsigned)cnt));
    }
    s_gbase[tid] = goff + (int)excl - dstart;
    __syncthreads();
    // keys into shared memory in digit order (stable)
#pragma unroll
    for (int c = 0; c < kSortItems; ++c) {
        if (base + c * 32 + lane < a.n) {
            const int d = (key[c] >> a.shift) & 0xff;
            const int slot = s_dstart[d] + s_wcnt[warp][d] + rank[c];
            s_key[slot] = key[c];
            s_val[slot] = val[c];
        }
    }
    __syncthreads();
    const int tile_n = (int)min((int64_t)kSortTile, a.n - t0);
    if (!LAST) {
        for (int j = tid; j < tile_n; j += kSortThreads) {
            const int k = s_key[j];
            const int dest = s_gbase[(k >> a.shift) & 0xff] + j;
            a.keys_out[dest] = k;
            a.vals_out[dest] = s_val[j];
        }
        return;
    }
    // last pass: the records. Positions are read at the input index, four
    // slots per thread at a time so that the scattered loads overlap.
    constexpr int U = 4;
    for (int j0 = tid; j0 < tile_n; j0 += U * kSortThreads) {
        float x[U][3];
        int ii[U], kk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u * kSortThreads;
            ii[u] = 0;
            kk[u] = 0;
            if (j < tile_n) {
                ii[u] = s_val[j];
                kk[u] = s_key[j];
                const float *p = a.pos + 3 * (int64_t)ii[u];
                x[u][0] = p[0];
                x[u][1] = p[1];
                x[u][2] = p[2];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u * kSortThreads;
            if (j >= tile_n) continue;
            const int i = ii[u];
            const int b = a.n_boxes == 1 ? 0 : box_of_particle(a.poff, a.n_boxes, i);
            const BoxDev &B = a.boxes[b];
            float rf[3];
            double rd[3];
            particle_rel(x[u], B, a.pow2, a.sorted_d != nullptr, rf, rd);
            const float m = a.mass ? a.mass[i] : B.gm;
            const int dest = s_gbase[(kk[u] >> a.shift) & 0xff] + j;
            a.sorted[dest] = make_float4(rf[0], rf[1], rf[2], m);
            if (a.sorted_d) a.sorted_d[dest] = dbl4_make(rd[0], rd[1], rd[2], (double)m);
            a.vals_out[dest] = i;
            // per-cell counts: the tile's keys are in full key order here, so
            // a cell's slots form one run; its last slot adds the run's end,
            // its first subtracts the run's start (runs that continue in
            // another tile add up across tiles)
            const bool first = j == 0 || s_key[j - 1] != kk[u];
            const bool last = j == tile_n - 1 || s_key[j + 1] != kk[u];
            if (first && last) atomicAdd(&a.count[kk[u]], 1);
            else if (first) atomicAdd(&a.count[kk[u]], -j);
            else if (last) atomicAdd(&a.count[kk[u]], j + 1);
        }
    }
}

// The global x slab of every particle (the x part of a1), or -1 for a
// particle whose x is outside [0, L) or not finite.
__global__ void k_slab_of(const float *__restrict__ pos, int64_t n, BoxDev B, int pow2,
                          int32_t *__restrict__ slab) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float xf = pos[3 * i];
        const bool in = pow2 ? (xf >= 0.f && xf < B.Lf) : ((double)xf >= 0.0 && (double)xf < B.L);
        int c = -1;
        float r;
        if (in && !(pow2 && cell_rel_pow2(xf, (float)B.cpd, B.inv_Lf, B.cpd, c, r)))
            c = cell_index(cell_unit((double)xf, B, pow2 != 0), B.cpd);
        slab[i] = in ? c : -1;
    }
}

// Sets bit 2 of *error_word if any of n counts is negative.
__global__ void k_check_counts(const int *__restrict__ count, int64_t n, int *error_word) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        bad = bad || count[i] < 0;
    if (bad) atomicOr(error_word, 4);
}

int grid_for(int64_t n, int threads, int sm_count, int per_sm = 8) {
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count * per_sm;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

// Exclusive scan of in[0..n) into out[0..n], out[n] = total (in == out is
// allowed). Block sums of 4096-element tiles go to tmp; up to 8192 of them
// are scanned by one block, more by scanning the block sums recursively
// (tmp holds scan_tmp_ints(n) ints).
cudaError_t scan_exclusive(const int *in, int *out, int64_t n, int *tmp, cudaStream_t s,
                           int64_t *launches) {
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int), s);
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
    if (launches) *launches += 2;
    if (nb <= kScanThreads * 8) {
        k_scan_blocks<<<1, kScanThreads, 0, s>>>(tmp, (int)nb, out + n);
        if (launches) *launches += 1;
    } else {
        // tmp[0..nb) scanned in place; its total lands in tmp[nb]
        cudaError_t e = scan_exclusive(tmp, tmp, nb, tmp + nb + 1, s, launches);
        if (e) return e;
        e = cudaMemcpyAsync(out + n, tmp + nb, sizeof(int), cudaMemcpyDeviceToDevice, s);
        if (e) return e;
    }
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp, out);
    return cudaGetLastError();
}

int64_t scan_tmp_ints(int64_t n) {
    int64_t total = 0;
    while (true) {
        const int64_t nb = (n + kScanTile - 1) / kScanTile;
        total += nb + 1;
        if (nb <= kScanThreads * 8) break;
        n = nb;
    }
    return total;
}

int64_t sort_tiles(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

cudaError_t launch_slab_of(const float *pos, int64_t n, const BoxDev &B, int pow2, int sm_count,
                           int32_t *slab, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_slab_of<<<grid_for(n, 256, sm_count), 256, 0, s>>>(pos, n, B, pow2, slab);
    return cudaGetLastError();
}

cudaError_t launch_check_counts(const int *count, int64_t n, int *error_word, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_check_counts<<<grid_for(n, 256, 152), 256, 0, s>>>(count, n, error_word);
    return cudaGetLastError();
}

int sort_passes(int64_t n_cells) {
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < n_cells) ++bits;
    const int p = (bits + 7) / 8;
    return p < 1 ? 1 : p;
}

cudaError_t launch_bin(Ctx *c, const float *pos, const float *mass, float m0, int64_t n,
                       cudaStream_t s, float *pos_copy) {
    (void)m0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->count, 0, sizeof(int) * c->n_cells, s))) return e;
    if ((e = cudaMemsetAsync(&c->state->error, 0, sizeof(int), s))) return e;
    if (n == 0) {
        c->perm = c->vals_a;
        return scan_exclusive(c->count, c->cell_start, c->n_cells, c->scan_tmp, s, &c->launches);
    }
    const int passes = sort_passes(c->n_cells);
    if ((e = cudaMemsetAsync(c->bin_state, 0, sizeof(BinState), s))) return e;
    if (pos_copy)
        k_cell_keys<true><<<grid_for(n, kKeyChunk, c->sm_count), kKeyThreads, 0, s>>>(
            pos, n, c->poff_d, c->n_boxes, c->boxes_d, c->pow2_all, passes, c->keys_a, c->bin_state,
            c->state, pos_copy);
    else
        k_cell_keys<false><<<grid_for(n, kKeyChunk, c->sm_count), kKeyThreads, 0, s>>>(
            pos, n, c->poff_d, c->n_boxes, c->boxes_d, c->pow2_all, passes, c->keys_a, c->bin_state,
            c->state, nullptr);
    if ((e = cudaGetLastError())) return e;
    c->launches += 1;
    // look-back words are told apart by an epoch per pass; when the counter
    // would wrap, the words are cleared and the count restarts
    if (c->bin_epoch + (unsigned)passes >= 0x7ffffff0u || c->bin_epoch == 0) {
        if ((e = cudaMemsetAsync(c->sort_status, 0,
                                 sizeof(unsigned long long) * kDigits * c->max_tiles, s)))
            return e;
        c->bin_epoch = 1;
    }
    const int64_t nt = sort_tiles(n);
    SortArgs a{};
    a.n = n;
    a.status = c->sort_status;
    a.bs = c->bin_state;
    a.st = c->state;
    a.pos = pos_copy ? pos_copy : pos;       // the last pass gathers from device memory
    a.mass = mass;
    a.poff = c->poff_d;
    a.n_boxes = c->n_boxes;
    a.boxes = c->boxes_d;
    a.pow2 = c->pow2_all;
    a.sorted = c->sorted;
    a.sorted_d = c->precision == NF_PREC_FP64_REF ? c->sorted_d : nullptr;
    a.count = c->count;
    for (int p = 0; p < passes; ++p) {
        const bool even = (p & 1) == 0;
        a.keys_in = even ? c->keys_a : c->keys_b;
        a.vals_in = p == 0 ? nullptr : (even ? c->vals_a : c->vals_b);
        a.keys_out = even ? c->keys_b : c->keys_a;
        a.vals_out = even ? c->vals_b : c->vals_a;
        a.shift = 8 * p;
        a.pass = p;
        a.epoch = c->bin_epoch++;
        if (p == passes - 1)
            k_sort_pass<true><<<(unsigned)nt, kSortThreads, 0, s>>>(a);
        else
            k_sort_pass<false><<<(unsigned)nt, kSortThreads, 0, s>>>(a);
        if ((e = cudaGetLastError())) return e;
        c->launches += 1;
    }
    c->perm = a.vals_out;
    return scan_exclusive(c->count, c->cell_start, c->n_cells, c->scan_tmp, s, &c->launches);
}

}  // namespace nf

// ---------------------------------------------------------------- no-alloc binning
// nf_bin_cells_noalloc: the binning above for one box, with every scratch
// buffer carved out of one file-scope device array instead of cudaMalloc.
// It serves callers that must not allocate device memory themselves or
// through a library, e.g. a host program whose own pool already reserves the
// GPU's memory (a further cudaMalloc would fail or fragment it), or a
// latency-critical loop that cannot pay cudaMalloc's implicit device-wide
// synchronisation. The paper has no counterpart to this call.
namespace nf {
void set_thread_error(const char *msg);
}

namespace {

constexpr int64_t kNoAllocMaxParticles = int64_t(1) << 20;   // 1,048,576
constexpr int64_t kNoAllocMaxCells = int64_t(1) << 18;       // CPD^3 <= 262,144
constexpr int64_t kNoAllocTiles = (kNoAllocMaxParticles + nf::kSortTile - 1) / nf::kSortTile;
constexpr int64_t kNoAllocScanInts = 256;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffKeysA = 0;
constexpr size_t kOffKeysB = kOffKeysA + align256(4 * kNoAllocMaxParticles);
constexpr size_t kOffValsA = kOffKeysB + align256(4 * kNoAllocMaxParticles);
constexpr size_t kOffValsB = kOffValsA + align256(4 * kNoAllocMaxParticles);
constexpr size_t kOffCount = kOffValsB + align256(4 * kNoAllocMaxParticles);
constexpr size_t kOffStatus = kOffCount + align256(4 * kNoAllocMaxCells);
constexpr size_t kOffBinState = kOffStatus + align256(8 * 256 * kNoAllocTiles);
constexpr size_t kOffScan = kOffBinState + align256(sizeof(nf::BinState));
constexpr size_t kOffState = kOffScan + align256(4 * kNoAllocScanInts);
constexpr size_t kOffBox = kOffState + align256(sizeof(nf::DevState));
constexpr size_t kOffPoff = kOffBox + align256(sizeof(nf::BoxDev));
constexpr size_t kNoAllocBytes = kOffPoff + align256(2 * sizeof(int64_t));   // about 17.3 MB
static_assert(kNoAllocScanInts >= (kNoAllocMaxCells + 4095) / 4096 + 1, "scan scratch");

// Shared by every call on a device and kept (with the last call's contents)
// until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_base[kNoAllocMaxDevices] = {};
int g_noalloc_sms[kNoAllocMaxDevices] = {};
unsigned g_noalloc_epoch[kNoAllocMaxDevices] = {};

// Device address of the array on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up
// once per device with that device current.
int noalloc_setup(int dev, unsigned char **base, int *sms, unsigned **epoch) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return NF_ECUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return NF_ECUDA;
        }
        g_noalloc_base[dev] = static_cast<unsigned char *>(p);
        g_noalloc_sms[dev] = n;
    }
    *base = g_noalloc_base[dev];
    *sms = g_noalloc_sms[dev];
    *epoch = &g_noalloc_epoch[dev];
    return NF_OK;
}

}  // namespace

extern "C" NF_API int nf_bin_cells_noalloc(const float *pos, const float *mass, double mass_if_null,
                                           int64_t n, double box_size, int cpd,
                                           int32_t *cell_start, int32_t *perm, float *sorted,
                                           void *stream) {
    using namespace nf;
    const int64_t ncell = (int64_t)cpd * cpd * cpd;
    if (n < 0 || n > kNoAllocMaxParticles) {
        set_thread_error("nf_bin_cells_noalloc: n must be in [0, 1048576]");
        return NF_EINVAL;
    }
    if (cpd < 1 || ncell > kNoAllocMaxCells) {
        set_thread_error("nf_bin_cells_noalloc: cpd must be in [1, 64] (CPD^3 <= 262144)");
        return NF_EINVAL;
    }
    if (!(box_size > 0.0) || !(box_size < 1e300)) {
        set_thread_error("nf_bin_cells_noalloc: box_size must be finite and > 0");
        return NF_EINVAL;
    }
    if (!cell_start || (n > 0 && (!pos || !perm || !sorted))) {
        set_thread_error("nf_bin_cells_noalloc: pos, cell_start, perm and sorted are required");
        return NF_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(sorted) % 16 != 0) {
        set_thread_error("nf_bin_cells_noalloc: sorted must be 16-byte aligned");
        return NF_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        set_thread_error("nf_bin_cells_noalloc: no usable current CUDA device");
        return NF_ECUDA;
    }
    unsigned char *base = nullptr;
    int sms = 0;
    unsigned *epoch = nullptr;
    if (noalloc_setup(dev, &base, &sms, &epoch) != NF_OK) {
        set_thread_error("nf_bin_cells_noalloc: cudaGetSymbolAddress of the scratch array failed");
        return NF_ECUDA;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    // A context on the stack whose buffers are views of the static array and
    // of the caller's outputs; the existing binning launcher runs on it.
    Ctx c;
    c.device = dev;
    c.n_boxes = 1;
    c.precision = NF_PREC_FP32;
    c.capacity = kNoAllocMaxParticles;
    c.n_cells = ncell;
    c.sm_count = sms;
    c.keys_a = reinterpret_cast<int *>(base + kOffKeysA);
    c.keys_b = reinterpret_cast<int *>(base + kOffKeysB);
    c.vals_a = reinterpret_cast<int *>(base + kOffValsA);
    c.vals_b = reinterpret_cast<int *>(base + kOffValsB);
    c.count = reinterpret_cast<int *>(base + kOffCount);
    c.sort_status = reinterpret_cast<unsigned long long *>(base + kOffStatus);
    c.max_tiles = kNoAllocTiles;
    c.bin_state = reinterpret_cast<BinState *>(base + kOffBinState);
    c.bin_epoch = *epoch;
    c.scan_tmp = reinterpret_cast<int *>(base + kOffScan);
    c.state = reinterpret_cast<DevState *>(base + kOffState);
    c.boxes_d = reinterpret_cast<BoxDev *>(base + kOffBox);
    c.poff_d = reinterpret_cast<int64_t *>(base + kOffPoff);
    c.cell_start = cell_start;
    c.sorted = reinterpret_cast<float4 *>(sorted);

    BoxDev B{};
    const double h = box_size / cpd;
    B.L = box_size;
    B.cpd_d = (double)cpd;
    B.cpd = cpd;
    B.cell_off = 0;
    B.inv_h2_d = 1.0 / (h * h);
    B.inv_h3_d = 1.0 / (h * h * h);
    B.gm = (float)mass_if_null;
    B.gm_d = (double)B.gm;
    B.Lf = (float)box_size;
    B.inv_Lf = (float)(1.0 / box_size);
    int ex = 0;
    c.pow2_all = std::frexp(box_size, &ex) == 0.5 ? 1 : 0;
    const int64_t poff[2] = {0, n};
    cudaError_t e = cudaMemcpyAsync(c.boxes_d, &B, sizeof(B), cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(c.poff_d, poff, sizeof(poff), cudaMemcpyHostToDevice, s);
    if (!e) e = launch_bin(&c, pos, mass, (float)mass_if_null, n, s);
    *epoch = c.bin_epoch;
    if (!e && n > 0) e = cudaMemcpyAsync(perm, c.perm, sizeof(int) * n, cudaMemcpyDeviceToDevice, s);
    int err_word = 0;
    if (!e) e = cudaMemcpyAsync(&err_word, &c.state->error, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        cudaGetLastError();
        set_thread_error(cudaGetErrorString(e));
        return NF_ECUDA;
    }
    if (err_word & 2) {
        set_thread_error("nf_bin_cells_noalloc: the sort's look-back gave up waiting");
        return NF_ETIMEOUT;
    }
    if (err_word) {
        set_thread_error("nf_bin_cells_noalloc: a position component is not finite or outside [0, L)");
        return NF_ERANGE;
    }
    return NF_OK;
}

// nf_pairs.cu -- work list and pair kernels of the near-field direct sum
// (Maksimova et al. 2021, Sec. 3.1: every sink sums the particles of the
// (2R+1)^3 cells around its own cell; Sec. 4.3/4.5: the GPU works through
// queued units of sink x source cells).
//
// Work decomposition. A work item is a run of consecutive cell-sorted sinks
// of one cell, served to one warp. The warp's lanes are split S ways over the
// sources (lane = g * S + s; lane g holds K sinks g, g + 32/S, ...), so a cell
// of n sinks costs ceil-ish(n / (32K/S)) items with little idle lane time.
// Items are placed in cost buckets, heaviest first, and a persistent grid of
// warps pulls them from an atomic counter.
//
// Pair loop. Coordinates are cell-relative in cell units. A source of
// neighbour cell offset d is staged in shared memory already shifted into the
// sink cell's frame (r_j + d), so one pair costs the 20 algorithmic flops of
// the Plummer law: 3 sub, 3 fma (s = |D|^2 + eps^2), rsqrt, 2 mul (s^-3/2),
// 3 fma (accumulate); masses are applied once per sink for equal-mass sets.
// Two sources are processed per instruction with the packed .f32x2 forms.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nf_ctx.h"
#include "nf_internal.cuh"

namespace nf {

namespace {

constexpr float kFarAway = 1.0e18f;   // padding source: contributes exactly 0

__device__ __forceinline__ int wrapc(int t, int cpd) {
    t = t < 0 ? t + cpd : t;
    return t >= cpd ? t - cpd : t;
}

__device__ __forceinline__ int cell_nsrc(const BoxDev &B, int local, const int *__restrict__ count,
                                         int R) {
    const int cpd = B.cpd;
    const int cx = local / (cpd * cpd), cy = (local / cpd) % cpd, cz = local % cpd;
    int s = 0;
    for (int dx = -R; dx <= R; ++dx) {
        const int x = xwrap(B, cx + dx);
        for (int dy = -R; dy <= R; ++dy) {
            const int row = B.cell_off + (x * cpd + wrapc(cy + dy, cpd)) * cpd;
            for (int dz = -R; dz <= R; ++dz) s += count[row + wrapc(cz + dz, cpd)];
        }
    }
    return s;
}

// Item cost model: each lane handles K sinks over n_src / S sources at ~11
// packed-lane instructions per sink-source, plus staging; the bucket is the
// number of leading zeros so that heavier items get smaller bucket indices.
__device__ __forceinline__ int cost_bucket(int nsrc, int K, int log2s) {
    unsigned long long cost = (unsigned long long)nsrc * (unsigned long long)((22 * K) >> log2s) +
                              (unsigned long long)nsrc;
    return __clzll(cost | 1ull);
}

// Bucket of an item with 2^log2s lanes per sink: small items (when the
// small-item kernel is on) take the upper half, after every other item.
__device__ __forceinline__ int item_bucket(int nsrc, int K, int log2s, int small_on) {
    const bool small = small_on && log2s >= kSmallLog2S && nsrc <= kSmallMaxSrc;
    return cost_bucket(nsrc, K, log2s) + (small ? kBuckets : 0);
}

struct WLArgs {
    const BoxDev *boxes;
    int n_boxes;
    int R;
    int K;
    int64_t n_cells;           // cells that hold sinks (a slab context's owned cells come first)
    const int *count;
    const int *cell_start;
    int *nsrc_cell;
    const Decomp *decomp;
    DevState *st;
    WorkItem *items;
    int pencils_on;            // serve eligible pencils with k_pencils
    int small_on;              // items of >= 2^kSmallLog2S lane splits go to k_pairs_small
    unsigned char *pencil_ok;  // [n_cells]: at a pencil's first cell, 1 if it is served as a pencil
    int *pencils;              // pencil items: first cell of each
};

// Cell c's pencil is served by k_pencils (its cells make no other items).
__device__ __forceinline__ bool cell_in_pencil(const WLArgs &a, const BoxDev &B, int64_t c) {
    if (!a.pencils_on) return false;
    const int cz = ((int)c - B.cell_off) % B.cpd;
    if (cz >= (B.cpd / kPencil) * kPencil) return false;
    return a.pencil_ok[c - cz % kPencil] != 0;
}

// Pencil items: a thread per pencil's first cell decides whether the pencil
// is served by k_pencils (every staged column fits kColMax, at least one
// cell is not empty) and, if so, appends it to the pencil list. k_pencils
// takes the first kPencilSinks sinks of each of the pencil's cells; the
// rest of a fuller cell makes ordinary items.
__global__ void __launch_bounds__(256) k_wl_pencils(WLArgs a) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.n_cells) return;
    const int box = a.n_boxes == 1 ? 0 : box_of_cell(a.boxes, a.n_boxes, (int)c);
    const BoxDev &B = a.boxes[box];
    const int cpd = B.cpd, R = a.R, W = 2 * R + 1;
    const int local = (int)c - B.cell_off;
    const int cx = local / (cpd * cpd), cy = (local / cpd) % cpd, cz = local % cpd;
    if (cz % kPencil != 0 || cz >= (cpd / kPencil) * kPencil) return;
    bool ok = true, any = false;
    for (int j = 0; j < kPencil; ++j) any = any || a.count[c + j] > 0;
    for (int ix = 0; ix < W && ok; ++ix) {
        const int x = xwrap(B, cx + ix - R);
        for (int iy = 0; iy < W && ok; ++iy) {
            const int row = B.cell_off + (x * cpd + wrapc(cy + iy - R, cpd)) * cpd;
            int tot = 0;
            for (int k = 0; k < kPencil + 2 * R; ++k) {
                const int n = a.count[row + wrapc(cz - R + k, cpd)];
                tot += n + (n & 1);
            }
            ok = tot <= kColMax;
        }
    }
    ok = ok && any;
    a.pencil_ok[c] = ok ? 1 : 0;
    if (ok) a.pencils[atomicAdd(&a.st->n_pencils, 1)] = (int)c;
}

__global__ void __launch_bounds__(256) k_wl_count(WLArgs a) {
    __shared__ int hist[2 * kBuckets];
    __shared__ unsigned long long s_inter;
    __shared__ int s_max;
    for (int b = threadIdx.x; b < 2 * kBuckets; b += blockDim.x) hist[b] = 0;
    if (threadIdx.x == 0) { s_inter = 0; s_max = 0; }
    __syncthreads();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long inter = 0;
    int mx = 0;
    if (c < a.n_cells) {
        const int n = a.count[c];
        if (n > 0) {
            const int box = a.n_boxes == 1 ? 0 : box_of_cell(a.boxes, a.n_boxes, (int)c);
            const BoxDev B = a.boxes[box];
            const int ns = cell_nsrc(B, (int)c - B.cell_off, a.count, a.R);
            a.nsrc_cell[c] = ns;
            inter = (unsigned long long)n * (unsigned long long)ns;
            mx = n;
            // sinks beyond the first kPencilSinks of a pencil cell make items
            const int ni = cell_in_pencil(a, B, c) ? max(0, n - kPencilSinks) : n;
            if (ni > 0) {
                const int full = 32 * a.K;
                const int q = ni / full, r = ni % full;
                if (q) atomicAdd(&hist[cost_bucket(ns, a.K, 0)], q);
                for (int e = 0; e < a.decomp->n_entries[r]; ++e) {
                    const int ent = a.decomp->entry[r][e];
                    atomicAdd(&hist[item_bucket(ns, a.K, ent & 0xff, a.small_on)], 1);
                }
            }
        }
    }
    // block reductions
    for (int o = 16; o > 0; o >>= 1) {
        inter += __shfl_xor_sync(0xffffffffu, inter, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (inter) atomicAdd(&s_inter, inter);
        if (mx) atomicMax(&s_max, mx);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 2 * kBuckets; b += blockDim.x)
        if (hist[b]) atomicAdd(&a.st->bucket_count[b], hist[b]);
    if (threadIdx.x == 0) {
        if (s_inter) atomicAdd(&a.st->interactions, s_inter);
        if (s_max) atomicMax(&a.st->max_occ, s_max);
    }
}

__global__ void k_wl_scan(DevState *st) {
    // one warp: exclusive scan of the bucket counts; the small items' buckets
    // (upper half) start at n_main
    const int lane = threadIdx.x;
    int run = 0;
    for (int b0 = 0; b0 < 2 * kBuckets; b0 += 32) {
        if (b0 == kBuckets && lane == 0) st->n_main = run;
        const int v = st->bucket_count[b0 + lane];
        int inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        st->bucket_cursor[b0 + lane] = run + inc - v;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) {
        st->n_items = run;
        st->queue_head = 0;
        st->small_head = 0;
    }
}

__global__ void __launch_bounds__(256) k_wl_write(WLArgs a) {
    __shared__ int cnt[2 * kBuckets];
    __shared__ int base[2 * kBuckets];
    for (int b = threadIdx.x; b < 2 * kBuckets; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int n = 0, ns = 0, box = 0;
    int skip = 0;                       // leading sinks served by k_pencils
    if (c < a.n_cells) {
        n = a.count[c];
        if (n > 0) {
            box = a.n_boxes == 1 ? 0 : box_of_cell(a.boxes, a.n_boxes, (int)c);
            ns = a.nsrc_cell[c];
            if (cell_in_pencil(a, a.boxes[box], c)) {
                skip = min(n, kPencilSinks);
                n -= skip;
            }
        }
    }
    const int full = 32 * a.K;
    const int q = n / full, r = n % full;
    if (n > 0) {
        if (q) atomicAdd(&cnt[cost_bucket(ns, a.K, 0)], q);
        for (int e = 0; e < a.decomp->n_entries[r]; ++e)
            atomicAdd(&cnt[item_bucket(ns, a.K, a.decomp->entry[r][e] & 0xff, a.small_on)], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 2 * kBuckets; b += blockDim.x) {
        base[b] = cnt[b] ? atomicAdd(&a.st->bucket_cursor[b], cnt[b]) : 0;
        cnt[b] = 0;
    }
    __syncthreads();
    if (n > 0) {
        const int first = a.cell_start[c] + skip;
        if (q) {
            const int b = cost_bucket(ns, a.K, 0);
            const int p = base[b] + atomicAdd(&cnt[b], q);
            for (int j = 0; j < q; ++j) {
                WorkItem w;
                w.cell = (int)c;
                w.first = first + j * full;
                w.n = full;
                w.box_s = box << 8;
                a.items[p + j] = w;
            }
        }
        int off = first + q * full;
        for (int e = 0; e < a.decomp->n_entries[r]; ++e) {
            const int ent = a.decomp->entry[r][e];
            const int b = item_bucket(ns, a.K, ent & 0xff, a.small_on);
            const int p = base[b] + atomicAdd(&cnt[b], 1);
            WorkItem w;
            w.cell = (int)c;
            w.first = off;
            w.n = ent >> 8;
            w.box_s = (box << 8) | (ent & 0xff);
            a.items[p] = w;
            off += ent >> 8;
        }
    }
}

// ------------------------------------------------------------ pair kernels
struct PairArgs {
    const float4 *sorted;      // cell-sorted (rx, ry, rz, m)
    const dbl4 *sorted_d;   // FP64 copy (FP64 kernel only)
    const float4 *w_sorted;    // cell-sorted cotangent (VJP only)
    const int *cell_start;
    const int *perm;
    const BoxDev *boxes;
    const WorkItem *items;
    DevState *st;
    void *out;                 // N x 3, input order
    int out_f64;
    int R;
    int nbr;                   // (2R+1)^3
    int tbl;                   // per-warp table stride (ints), >= nbr + 1
    float *dens;               // N, input order: kernel density estimate (KDE kernels)
    int n_boxes;
};

// Per-warp neighbourhood table: pfx[ci] = exclusive prefix of the source
// counts in cell order, dlt[ci] = cell_start - pfx (so source q of cell ci
// sits at sorted slot q + dlt[ci]), ofs[ci] = packed cell offset d + R.
// Returns the number of sources.
__device__ __forceinline__ int build_table(const PairArgs &a, const BoxDev &B, int cell,
                                           int *pfx, int *dlt, int *ofs) {
    const int lane = threadIdx.x & 31;
    const int cpd = B.cpd, R = a.R, W = 2 * R + 1;
    const int local = cell - B.cell_off;
    const int cx = local / (cpd * cpd), cy = (local / cpd) % cpd, cz = local % cpd;
    int run = 0;
    for (int b0 = 0; b0 < a.nbr; b0 += 32) {
        const int ci = b0 + lane;
        int cnt = 0, st = 0, code = 0;
        if (ci < a.nbr) {
            const int ix = ci / (W * W), iy = (ci / W) % W, iz = ci % W;
            const int g = B.cell_off +
                          (xwrap(B, cx + ix - R) * cpd + wrapc(cy + iy - R, cpd)) * cpd +
                          wrapc(cz + iz - R, cpd);
            st = a.cell_start[g];
            cnt = a.cell_start[g + 1] - st;
            code = ix | (iy << 8) | (iz << 16);
        }
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (ci < a.nbr) {
            const int p = run + inc - cnt;
            pfx[ci] = p;
            dlt[ci] = st - p;
            ofs[ci] = code;
        }
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) pfx[a.nbr] = run;
    __syncwarp();
    return run;
}

// Source q of the item -> (sorted slot, offset code); `ci` is the lane's
// running cell index (q only grows within an item).
__device__ __forceinline__ int locate(const int *pfx, int nbr, int q, int &ci) {
    while (ci + 1 < nbr && pfx[ci + 1] <= q) ++ci;
    return ci;
}

__device__ __forceinline__ void two_sum(f2_t a, f2_t b, f2_t &s, f2_t &e) {
    s = f2_add(a, b);
    const f2_t bb = f2_sub(s, a);
    e = f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb));
}

__device__ __forceinline__ void two_sum1(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Forward pair kernel. K sinks per lane; EQ: all masses equal (applied in
// the epilogue); COMP: 0 plain FP32 sums; 1 the per-tile FP32 partial sums
// are folded into a compensated (hi, lo) running total by TwoSum (three per
// sink and tile; the pair loop is the plain one); 2 every pair term is added
// by TwoSum (the most accurate and the slowest form).
// LAW 0: Plummer, f = s^-3/2 with s = r^2 + eps^2.
// LAW 1: spline, f = min(c0 + c1 r + c2 r^2, r^-3): the polynomial is the
//   law inside eps_s and r^-3 outside, and the two cross only at r = eps_s
//   (u^3 (10 - 15u + 6u^2) - 1 has derivative 30 u^2 (u-1)^2 >= 0), so the
//   minimum selects the right branch without a divergent test. s carries a
//   1e-30 floor so that the self pair gives a finite f times a zero offset.
// KDE: also accumulate the density sum_j m_j max(0, 1 - r^2/b^2)
//   (Sec. 3.3), with 1 - r^2/b^2 = kb0 + kb1 s.
// TILE: sources staged per tile (64, 128 or 256).
template <int K, bool EQ, int COMP, int LAW = 0, bool KDE = false, int TILE = kTile>
__global__ void __launch_bounds__(512) k_pairs(PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    constexpr int NF = EQ ? 3 : 4;
    float *sbase = reinterpret_cast<float *>(smem_raw) + wib * (NF * TILE + 3 * a.tbl);
    float *sx = sbase, *sy = sbase + TILE, *sz = sbase + 2 * TILE, *sm = sbase + 3 * TILE;
    int *pfx = reinterpret_cast<int *>(sbase + NF * TILE);
    int *dlt = pfx + a.tbl, *ofs = dlt + a.tbl;
    const int n_items = a.st->n_main;            // the small items, if split off, come after

    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&a.st->queue_head, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const WorkItem w = a.items[it];
        const int box = w.box_s >> 8, log2s = w.box_s & 0xff;
        const int S = 1 << log2s, G = 32 >> log2s;
        const int g = lane >> log2s, sp = lane & (S - 1);
        // box constants are read where they are used (not kept in registers
        // across the tile loop)
        const BoxDev *Bp = a.boxes + box;
        const int nsrc = build_table(a, *Bp, w.cell, pfx, dlt, ofs);
        const f2_t eps2 = f2_pack(Bp->eps2, Bp->eps2);
        f2_t c0 = 0ull, c1 = 0ull, c2 = 0ull, kb0 = 0ull, kb1 = 0ull;
        if (LAW == 1) {
            c0 = f2_pack(Bp->sp_c0, Bp->sp_c0);
            c1 = f2_pack(Bp->sp_c1, Bp->sp_c1);
            c2 = f2_pack(Bp->sp_c2, Bp->sp_c2);
        }
        if (KDE) {
            kb0 = f2_pack(Bp->kb0, Bp->kb0);
            kb1 = f2_pack(Bp->kb1, Bp->kb1);
        }

        f2_t xi[K], yi[K], zi[K], ax[K], ay[K], az[K];
        f2_t lx[K], ly[K], lz[K], rho[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int si = g + G * k;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            if (si < w.n) p = a.sorted[w.first + si];
            xi[k] = f2_pack(p.x, p.x);
            yi[k] = f2_pack(p.y, p.y);
            zi[k] = f2_pack(p.z, p.z);
            ax[k] = ay[k] = az[k] = 0ull;
            lx[k] = ly[k] = lz[k] = 0ull;
            rho[k] = 0ull;
        }
        int ci = 0, co = 0;   // cell stream: current neighbour cell, sources taken from it
        for (int q0 = 0; q0 < nsrc; q0 += TILE) {
            const int cntT = min(TILE, nsrc - q0);
            const int npair = (cntT + 1) >> 1;
            // fill the tile cell by cell: each cell's sources are contiguous in
            // the sorted array and share one offset d, so the lanes copy
            // coalesced runs and add a warp-uniform shift
            int filled = 0;
            while (filled < cntT && ci < a.nbr) {
                const int p0 = pfx[ci];
                const int left = pfx[ci + 1] - p0 - co;
                if (left <= 0) { ++ci; co = 0; continue; }
                const int take = min(left, cntT - filled);
                const int base = p0 + dlt[ci] + co;
                const int code = ofs[ci];
                const float ox = (float)((code & 0xff) - a.R);
                const float oy = (float)(((code >> 8) & 0xff) - a.R);
                const float oz = (float)((code >> 16) - a.R);
                for (int t = lane; t < take; t += 32) {
                    const float4 p = a.sorted[base + t];
                    sx[filled + t] = p.x + ox;
                    sy[filled + t] = p.y + oy;
                    sz[filled + t] = p.z + oz;
                    if (!EQ) sm[filled + t] = p.w;
                }
                filled += take;
                co += take;
                if (take == left) { ++ci; co = 0; }
            }
            if ((cntT & 1) && lane == 0) {   // odd tile: pad with a source that adds 0
                sx[cntT] = kFarAway;
                sy[cntT] = 0.f;
                sz[cntT] = 0.f;
                if (!EQ) sm[cntT] = 0.f;
            }
            __syncwarp();
            const f2_t *px = reinterpret_cast<const f2_t *>(sx);
            const f2_t *py = reinterpret_cast<const f2_t *>(sy);
            const f2_t *pz = reinterpret_cast<const f2_t *>(sz);
            const f2_t *pm = reinterpret_cast<const f2_t *>(sm);
            // per-tile partial sums (plain FP32): each tile's <= 64/S terms per
            // accumulator are summed afresh and then folded into the running
            // total, which keeps the rounding random walk short
            f2_t tx[K], ty[K], tz[K], tr[K];
#pragma unroll
            for (int k = 0; k < K; ++k) tx[k] = ty[k] = tz[k] = tr[k] = 0ull;
            // lane split sp takes source pairs sp, sp + S, ...; a counted
            // loop (trip count known on entry) unrolls cleanly
            const int n_it = (npair - sp + S - 1) >> log2s;
#pragma unroll 2
            for (int it = 0; it < n_it; ++it) {
                const int pp = sp + (it << log2s);
                const f2_t x2 = px[pp], y2 = py[pp], z2 = pz[pp];
                f2_t m2 = 0ull;
                if (!EQ) m2 = pm[pp];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const f2_t dx = f2_sub(x2, xi[k]);
                    const f2_t dy = f2_sub(y2, yi[k]);
                    const f2_t dz = f2_sub(z2, zi[k]);
                    f2_t s = f2_fma(dx, dx, eps2);
                    s = f2_fma(dy, dy, s);
                    s = f2_fma(dz, dz, s);
                    const f2_t r = f2_rsqrt(s);
                    f2_t f = f2_mul(f2_mul(r, r), r);
                    if (LAW == 1) {
                        const f2_t rr = f2_mul(s, r);
                        f = f2_min(f2_fma(f2_fma(c2, rr, c1), rr, c0), f);
                    }
                    if (KDE) {
                        const f2_t t = f2_max0(f2_fma(s, kb1, kb0));
                        tr[k] = EQ ? f2_add(tr[k], t) : f2_fma(t, m2, tr[k]);
                    }
                    if (!EQ) f = f2_mul(f, m2);
                    if (COMP != 2) {
                        tx[k] = f2_fma(f, dx, tx[k]);
                        ty[k] = f2_fma(f, dy, ty[k]);
                        tz[k] = f2_fma(f, dz, tz[k]);
                    } else {
                        f2_t e;
                        two_sum(ax[k], f2_mul(f, dx), ax[k], e); lx[k] = f2_add(lx[k], e);
                        two_sum(ay[k], f2_mul(f, dy), ay[k], e); ly[k] = f2_add(ly[k], e);
                        two_sum(az[k], f2_mul(f, dz), az[k], e); lz[k] = f2_add(lz[k], e);
                    }
                }
            }
            if (COMP == 0) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    ax[k] = f2_add(ax[k], tx[k]);
                    ay[k] = f2_add(ay[k], ty[k]);
                    az[k] = f2_add(az[k], tz[k]);
                }
            } else if (COMP == 1) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    f2_t e;
                    two_sum(ax[k], tx[k], ax[k], e); lx[k] = f2_add(lx[k], e);
                    two_sum(ay[k], ty[k], ay[k], e); ly[k] = f2_add(ly[k], e);
                    two_sum(az[k], tz[k], az[k], e); lz[k] = f2_add(lz[k], e);
                }
            }
            if (KDE) {
#pragma unroll
                for (int k = 0; k < K; ++k) rho[k] = f2_add(rho[k], tr[k]);
            }
            __syncwarp();
        }
        // epilogue: fold the two packed halves, reduce over the S lanes of
        // each sink group (xor tree, fixed order), scale and un-permute
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float v[3];
            const f2_t hs[3] = {ax[k], ay[k], az[k]};
            const f2_t ls[3] = {lx[k], ly[k], lz[k]};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float h0, h1;
                f2_unpack(hs[c], h0, h1);
                if (COMP == 0) {
                    float s = h0 + h1;
                    for (int o = 1; o < S; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    v[c] = s;
                } else {
                    float l0, l1, h, e;
                    f2_unpack(ls[c], l0, l1);
                    two_sum1(h0, h1, h, e);
                    float l = __fadd_rn(__fadd_rn(l0, l1), e);
                    for (int o = 1; o < S; o <<= 1) {
                        const float ho = __shfl_xor_sync(0xffffffffu, h, o);
                        const float lo = __shfl_xor_sync(0xffffffffu, l, o);
                        two_sum1(h, ho, h, e);
                        l = __fadd_rn(__fadd_rn(l, lo), e);
                    }
                    v[c] = __fadd_rn(h, l);
                }
            }
            float dv = 0.f;
            if (KDE) {
                float r0, r1;
                f2_unpack(rho[k], r0, r1);
                dv = r0 + r1;
                for (int o = 1; o < S; o <<= 1) dv += __shfl_xor_sync(0xffffffffu, dv, o);
            }
            const int si = g + G * k;
            if (sp == 0 && si < w.n) {
                const int i = a.perm[w.first + si];
                if (KDE) a.dens[i] = EQ ? dv * __ldg(&Bp->gm) : dv;
                if (a.out_f64) {
                    const double sc = EQ ? __ldg(&Bp->gm_d) * __ldg(&Bp->inv_h2_d) : __ldg(&Bp->inv_h2_d);
                    double *o = reinterpret_cast<double *>(a.out) + 3 * (int64_t)i;
                    o[0] = (double)v[0] * sc;
                    o[1] = (double)v[1] * sc;
                    o[2] = (double)v[2] * sc;
                } else {
                    const float sc = EQ ? __ldg(&Bp->gm) * __ldg(&Bp->inv_h2) : __ldg(&Bp->inv_h2);
                    float *o = reinterpret_cast<float *>(a.out) + 3 * (int64_t)i;
                    o[0] = v[0] * sc;
                    o[1] = v[1] * sc;
                    o[2] = v[2] * sc;
                }
            }
        }
    }
}

// ------------------------------------------------------------ small items
// Per-warp pair table of an item's neighbourhood, for the small-item kernel:
// ppf[ci] = exclusive prefix over the cells of their source pairs
// ceil(n/2), sst[ci] = the cell's first sorted slot, scn[ci] = its source
// count, sof[ci] = packed offset d + R. Returns the number of pairs.
__device__ __forceinline__ int build_pair_table(const PairArgs &a, const BoxDev &B, int cell, int *ppf,
                                                int *sst, int *scn, int *sof) {
    const int lane = threadIdx.x & 31;
    const int cpd = B.cpd, R = a.R, W = 2 * R + 1;
    const int local = cell - B.cell_off;
    const int cx = local / (cpd * cpd), cy = (local / cpd) % cpd, cz = local % cpd;
    int run = 0;
    for (int b0 = 0; b0 < a.nbr; b0 += 32) {
        const int ci = b0 + lane;
        int cnt = 0, st = 0, code = 0;
        if (ci < a.nbr) {
            const int ix = ci / (W * W), iy = (ci / W) % W, iz = ci % W;
            const int gc = B.cell_off +
                           (xwrap(B, cx + ix - R) * cpd + wrapc(cy + iy - R, cpd)) * cpd +
                           wrapc(cz + iz - R, cpd);
            st = a.cell_start[gc];
            cnt = a.cell_start[gc + 1] - st;
            code = ix | (iy << 8) | (iz << 16);
        }
        const int np = (cnt + 1) >> 1;
        int inc = np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (ci < a.nbr) {
            ppf[ci] = run + inc - np;
            sst[ci] = st;
            scn[ci] = cnt;
            sof[ci] = code;
        }
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) ppf[a.nbr] = run;
    __syncwarp();
    return run;
}

// One source pair of a small item: pair P of the neighbourhood, shifted into
// the sink cell's frame (an odd cell's last pair is padded with a source
// that adds 0, as in the tiled kernel).
struct SrcPair {
    f2_t x, y, z, m;
};

template <bool EQ>
__device__ __forceinline__ SrcPair load_pair(const PairArgs &a, const int *ppf, const int *sst,
                                             const int *scn, const int *sof, int nbr, int P, int &ci) {
    while (ci + 1 < nbr && ppf[ci + 1] <= P) ++ci;
    const int j = 2 * (P - ppf[ci]);
    const int st = sst[ci], cnt = scn[ci], code = sof[ci];
    const float ox = (float)((code & 0xff) - a.R);
    const float oy = (float)(((code >> 8) & 0xff) - a.R);
    const float oz = (float)((code >> 16) - a.R);
    const float4 p0 = a.sorted[st + j];
    float4 p1 = make_float4(kFarAway, 0.f, 0.f, 0.f);
    if (j + 1 < cnt) {
        p1 = a.sorted[st + j + 1];
        p1.x += ox;
        p1.y += oy;
        p1.z += oz;
    }
    SrcPair q;
    q.x = f2_pack(p0.x + ox, p1.x);
    q.y = f2_pack(p0.y + oy, p1.y);
    q.z = f2_pack(p0.z + oz, p1.z);
    q.m = EQ ? 0ull : f2_pack(p0.w, p1.w);
    return q;
}

// Forward kernel for small items (plain FP32, Plummer, K = 4 sinks per lane):
// the items of at most 8 sinks whose lanes split the sources 16 or 32 ways,
// over at most kSmallMaxSrc sources, mostly the sinks of a cell left over
// after its full groups. They cost the
// tiled kernel a whole neighbourhood of staging for a few sinks; here each
// lane reads its own source pairs straight from the records (P = sp, sp + S,
// ..., two pairs in flight), with no shared-memory tile and no warp
// barrier. Same sink mapping, pair arithmetic and epilogue as k_pairs; the
// lane sums are folded into the running totals every 8 pairs.
template <bool EQ>
__global__ void __launch_bounds__(128, 4) k_pairs_small(PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int K = 4;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *ppf = reinterpret_cast<int *>(smem_raw) + wib * 4 * a.tbl;
    int *sst = ppf + a.tbl, *scn = sst + a.tbl, *sof = scn + a.tbl;
    const int n_items = a.st->n_items, n_main = a.st->n_main;
    for (;;) {
        int it = 0;
        if (lane == 0) it = n_main + atomicAdd(&a.st->small_head, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const WorkItem w = a.items[it];
        const int box = w.box_s >> 8, log2s = w.box_s & 0xff;
        const int S = 1 << log2s, G = 32 >> log2s;
        const int g = lane >> log2s, sp = lane & (S - 1);
        const BoxDev *Bp = a.boxes + box;
        const int npairs = build_pair_table(a, *Bp, w.cell, ppf, sst, scn, sof);
        const f2_t eps2 = f2_pack(Bp->eps2, Bp->eps2);
        f2_t xi[K], yi[K], zi[K], ax[K], ay[K], az[K], tx[K], ty[K], tz[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int si = g + G * k;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            if (si < w.n) p = a.sorted[w.first + si];
            xi[k] = f2_pack(p.x, p.x);
            yi[k] = f2_pack(p.y, p.y);
            zi[k] = f2_pack(p.z, p.z);
            ax[k] = ay[k] = az[k] = tx[k] = ty[k] = tz[k] = 0ull;
        }
        const int n_it = (npairs - sp + S - 1) >> log2s;
        int ci = 0;
        for (int i = 0; i < n_it; i += 2) {
            SrcPair q[2];
            q[0] = load_pair<EQ>(a, ppf, sst, scn, sof, a.nbr, sp + (i << log2s), ci);
            const bool two = i + 1 < n_it;
            if (two) q[1] = load_pair<EQ>(a, ppf, sst, scn, sof, a.nbr, sp + ((i + 1) << log2s), ci);
            else q[1] = SrcPair{f2_pack(kFarAway, kFarAway), 0ull, 0ull, 0ull};
#pragma unroll
            for (int u = 0; u < 2; ++u) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const f2_t dx = f2_sub(q[u].x, xi[k]);
                    const f2_t dy = f2_sub(q[u].y, yi[k]);
                    const f2_t dz = f2_sub(q[u].z, zi[k]);
                    f2_t s2 = f2_fma(dx, dx, eps2);
                    s2 = f2_fma(dy, dy, s2);
                    s2 = f2_fma(dz, dz, s2);
                    const f2_t r = f2_rsqrt(s2);
                    f2_t f = f2_mul(f2_mul(r, r), r);
                    if (!EQ) f = f2_mul(f, q[u].m);
                    tx[k] = f2_fma(f, dx, tx[k]);
                    ty[k] = f2_fma(f, dy, ty[k]);
                    tz[k] = f2_fma(f, dz, tz[k]);
                }
            }
            if ((i & 7) == 6 || i + 2 >= n_it) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    ax[k] = f2_add(ax[k], tx[k]);
                    ay[k] = f2_add(ay[k], ty[k]);
                    az[k] = f2_add(az[k], tz[k]);
                    tx[k] = ty[k] = tz[k] = 0ull;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float v[3];
            const f2_t hs[3] = {ax[k], ay[k], az[k]};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float h0, h1;
                f2_unpack(hs[c], h0, h1);
                float sum = h0 + h1;
                for (int o = 1; o < S; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                v[c] = sum;
            }
            const int si = g + G * k;
            if (sp == 0 && si < w.n) {
                const int i = a.perm[w.first + si];
                const float sc = EQ ? __ldg(&Bp->gm) * __ldg(&Bp->inv_h2) : __ldg(&Bp->inv_h2);
                float *o = reinterpret_cast<float *>(a.out) + 3 * (int64_t)i;
                o[0] = v[0] * sc;
                o[1] = v[1] * sc;
                o[2] = v[2] * sc;
            }
        }
    }
}

// ------------------------------------------------------------ pencil kernel
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Forward pair kernel for pencils (plain FP32, Plummer, K = 4 sinks per
// lane, two lanes per sink): one block of kPencil warps takes kPencil
// z-consecutive cells cz0..cz0+3 of one (x, y) row, warp w the first
// kPencilSinks sinks of cell cz0 + w. The block stages, for each of the (2R+1)^2 (dx, dy) columns, the
// column's kPencil + 2R cells (z from cz0 - R) once; warp w sums over the
// 2R+1 of them around its own cell, a contiguous range of the staged
// column. Columns are copied with cp.async one ahead of the one being summed.
// Each source is staged in its sinks' cell frame as in k_pairs: x and y
// shifted by (dx, dy), shared by the warps, and z once per warp, shifted by
// that warp's cell offset k - R - w, so the pair arithmetic is k_pairs'
// exactly. Each cell's staged run is padded to an even length with a far
// source (adds 0), so every warp's range starts on a packed pair. The
// per-column sums are folded into the running totals.
template <bool EQ>
__global__ void __launch_bounds__(32 * kPencil) k_pencils(PairArgs a, const int *__restrict__ pencils) {
    constexpr int K = 4;
    constexpr int MAXC = kPencil + 4;           // cells per column for R <= 2
    constexpr int MAXCOL = 25;                  // (2R + 1)^2 for R <= 2
    __shared__ __align__(16) float4 raw[2][kColMax];
    __shared__ __align__(16) float sxy[2][kColMax];
    __shared__ __align__(16) float szw[kPencil][kColMax];     // z in warp w's frame
    __shared__ __align__(16) float sms[EQ ? 1 : kColMax];
    __shared__ int t_start[MAXCOL][MAXC];
    __shared__ int t_cnt[MAXCOL][MAXC];
    __shared__ int t_pfx[MAXCOL][MAXC + 1];
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int R = a.R, W = 2 * R + 1, ncol = W * W, ncell = kPencil + 2 * R;
    const int g = lane >> 1, sp = lane & 1;
    const int n_pen = a.st->n_pencils;
    const f2_t *px = reinterpret_cast<const f2_t *>(sxy[0]);
    const f2_t *py = reinterpret_cast<const f2_t *>(sxy[1]);
    const f2_t *pz = reinterpret_cast<const f2_t *>(szw[w]);
    const f2_t *pm = reinterpret_cast<const f2_t *>(sms);
    for (;;) {
        __syncthreads();                        // the previous pencil is done with shared memory
        if (tid == 0) s_item = atomicAdd(&a.st->pencil_head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_pen) break;
        const int c0 = pencils[it];
        const BoxDev *Bp = a.boxes + (a.n_boxes == 1 ? 0 : box_of_cell(a.boxes, a.n_boxes, c0));
        const int cpd = Bp->cpd;
        const int local = c0 - Bp->cell_off;
        const int cx = local / (cpd * cpd), cy = (local / cpd) % cpd, cz0 = local % cpd;
        // the staged columns: start and count of each cell
        for (int e = tid; e < ncol * ncell; e += 32 * kPencil) {
            const int col = e / ncell, k = e % ncell;
            const int gc = Bp->cell_off +
                           (xwrap(*Bp, cx + col / W - R) * cpd + wrapc(cy + col % W - R, cpd)) * cpd +
                           wrapc(cz0 - R + k, cpd);
            const int st = a.cell_start[gc];
            t_start[col][k] = st;
            t_cnt[col][k] = a.cell_start[gc + 1] - st;
        }
        __syncthreads();
        if (tid < ncol) {                       // padded exclusive prefix of each column
            int run = 0;
            for (int k = 0; k < ncell; ++k) {
                t_pfx[tid][k] = run;
                run += t_cnt[tid][k] + (t_cnt[tid][k] & 1);
            }
            t_pfx[tid][ncell] = run;
        }
        __syncthreads();
        // sinks of warp w: cell cz0 + w, the middle column's cell R + w
        const int mid = R * W + R;
        const int s0 = t_start[mid][R + w], ns = min(t_cnt[mid][R + w], kPencilSinks);
        const f2_t eps2 = f2_pack(Bp->eps2, Bp->eps2);
        f2_t xi[K], yi[K], zi[K], ax[K], ay[K], az[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int si = g + 16 * k;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            if (si < ns) p = a.sorted[s0 + si];
            xi[k] = f2_pack(p.x, p.x);
            yi[k] = f2_pack(p.y, p.y);
            zi[k] = f2_pack(p.z, p.z);
            ax[k] = ay[k] = az[k] = 0ull;
        }
        // column 0 in flight
        for (int k = 0; k < ncell; ++k) {
            const int cnt = t_cnt[0][k], base = t_pfx[0][k], st = t_start[0][k];
            for (int t = tid; t < cnt; t += 32 * kPencil) cp_async16(&raw[0][base + t], a.sorted + st + t);
        }
        cp_async_commit();
        for (int col = 0; col < ncol; ++col) {
            const int buf = col & 1;
            cp_async_wait_all();
            __syncthreads();                    // column col landed; the previous sums are done
            if (col + 1 < ncol) {
                for (int k = 0; k < ncell; ++k) {
                    const int cnt = t_cnt[col + 1][k], base = t_pfx[col + 1][k], st = t_start[col + 1][k];
                    for (int t = tid; t < cnt; t += 32 * kPencil)
                        cp_async16(&raw[buf ^ 1][base + t], a.sorted + st + t);
                }
            }
            cp_async_commit();
            // shift into the sinks' frames, structure of arrays, pad odd cells
            const float ox = (float)(col / W - R), oy = (float)(col % W - R);
            for (int k = 0; k < ncell; ++k) {
                const int cnt = t_cnt[col][k], base = t_pfx[col][k];
                for (int t = tid; t < cnt + (cnt & 1); t += 32 * kPencil) {
                    if (t < cnt) {
                        const float4 p = raw[buf][base + t];
                        sxy[0][base + t] = p.x + ox;
                        sxy[1][base + t] = p.y + oy;
#pragma unroll
                        for (int v = 0; v < kPencil; ++v) szw[v][base + t] = p.z + (float)(k - R - v);
                        if (!EQ) sms[base + t] = p.w;
                    } else {
                        sxy[0][base + t] = kFarAway;
                        sxy[1][base + t] = 0.f;
#pragma unroll
                        for (int v = 0; v < kPencil; ++v) szw[v][base + t] = 0.f;
                        if (!EQ) sms[base + t] = 0.f;
                    }
                }
            }
            __syncthreads();
            // warp w: cells w .. w + 2R of the column
            const int lo = t_pfx[col][w] >> 1, npair = (t_pfx[col][w + W] >> 1) - lo;
            f2_t tx[K], ty[K], tz[K];
#pragma unroll
            for (int k = 0; k < K; ++k) tx[k] = ty[k] = tz[k] = 0ull;
            const int n_it = (npair - sp + 1) >> 1;
#pragma unroll 4
            for (int i2 = 0; i2 < n_it; ++i2) {
                const int pp = lo + sp + 2 * i2;
                const f2_t x2 = px[pp], y2 = py[pp], z2 = pz[pp];
                f2_t m2 = 0ull;
                if (!EQ) m2 = pm[pp];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const f2_t dx = f2_sub(x2, xi[k]);
                    const f2_t dy = f2_sub(y2, yi[k]);
                    const f2_t dz = f2_sub(z2, zi[k]);
                    f2_t s2 = f2_fma(dx, dx, eps2);
                    s2 = f2_fma(dy, dy, s2);
                    s2 = f2_fma(dz, dz, s2);
                    const f2_t r = f2_rsqrt(s2);
                    f2_t f = f2_mul(f2_mul(r, r), r);
                    if (!EQ) f = f2_mul(f, m2);
                    tx[k] = f2_fma(f, dx, tx[k]);
                    ty[k] = f2_fma(f, dy, ty[k]);
                    tz[k] = f2_fma(f, dz, tz[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                ax[k] = f2_add(ax[k], tx[k]);
                ay[k] = f2_add(ay[k], ty[k]);
                az[k] = f2_add(az[k], tz[k]);
            }
        }
        // epilogue: fold the packed halves, the two lanes of each sink, scale, un-permute
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const f2_t hs[3] = {ax[k], ay[k], az[k]};
            float v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float h0, h1;
                f2_unpack(hs[c], h0, h1);
                float sum = h0 + h1;
                sum += __shfl_xor_sync(0xffffffffu, sum, 1);
                v[c] = sum;
            }
            const int si = g + 16 * k;
            if (sp == 0 && si < ns) {
                const int i = a.perm[s0 + si];
                const float sc = EQ ? __ldg(&Bp->gm) * __ldg(&Bp->inv_h2) : __ldg(&Bp->inv_h2);
                float *o = reinterpret_cast<float *>(a.out) + 3 * (int64_t)i;
                o[0] = v[0] * sc;
                o[1] = v[1] * sc;
                o[2] = v[2] * sc;
            }
        }
    }
}

// FP64 reference pair kernel: same items and order of work, double
// arithmetic throughout, s^-3/2 as 1 / (s * sqrt(s)). One sink per lane.
__global__ void __launch_bounds__(512) k_pairs_f64(PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *sbase = reinterpret_cast<double *>(smem_raw) +
                    wib * (4 * kTile + (3 * a.tbl + 1) / 2);
    double *sx = sbase, *sy = sbase + kTile, *sz = sbase + 2 * kTile, *sm = sbase + 3 * kTile;
    int *pfx = reinterpret_cast<int *>(sbase + 4 * kTile);
    int *dlt = pfx + a.tbl, *ofs = dlt + a.tbl;
    const int n_items = a.st->n_items;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&a.st->queue_head, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const WorkItem w = a.items[it];
        const int box = w.box_s >> 8, log2s = w.box_s & 0xff;
        const int S = 1 << log2s;
        const int g = lane >> log2s, sp = lane & (S - 1);
        const BoxDev B = a.boxes[box];
        const int nsrc = build_table(a, B, w.cell, pfx, dlt, ofs);
        double xi = 0, yi = 0, zi = 0;
        if (g < w.n) {
            const dbl4 p = a.sorted_d[w.first + g];
            xi = p.x; yi = p.y; zi = p.z;
        }
        double ax = 0, ay = 0, az = 0;
        int ci = 0;
        for (int q0 = 0; q0 < nsrc; q0 += kTile) {
            const int cntT = min(kTile, nsrc - q0);
            for (int t = lane; t < cntT; t += 32) {
                const int q = q0 + t;
                const int c = locate(pfx, a.nbr, q, ci);
                const dbl4 p = a.sorted_d[q + dlt[c]];
                const int code = ofs[c];
                sx[t] = p.x + (double)((code & 0xff) - a.R);
                sy[t] = p.y + (double)(((code >> 8) & 0xff) - a.R);
                sz[t] = p.z + (double)((code >> 16) - a.R);
                sm[t] = p.w;
            }
            __syncwarp();
            for (int j = sp; j < cntT; j += S) {
                const double dx = sx[j] - xi, dy = sy[j] - yi, dz = sz[j] - zi;
                const double s = dx * dx + dy * dy + dz * dz + B.eps2_d;
                const double f = sm[j] / (s * sqrt(s));
                ax += f * dx;
                ay += f * dy;
                az += f * dz;
            }
            __syncwarp();
        }
        for (int o = 1; o < S; o <<= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
            az += __shfl_xor_sync(0xffffffffu, az, o);
        }
        if (sp == 0 && g < w.n) {
            const int i = a.perm[w.first + g];
            const double sc = B.inv_h2_d;
            if (a.out_f64) {
                double *o = reinterpret_cast<double *>(a.out) + 3 * (int64_t)i;
                o[0] = ax * sc; o[1] = ay * sc; o[2] = az * sc;
            } else {
                float *o = reinterpret_cast<float *>(a.out) + 3 * (int64_t)i;
                o[0] = (float)(ax * sc); o[1] = (float)(ay * sc); o[2] = (float)(az * sc);
            }
        }
    }
}

// Adjoint (vector-Jacobian product) pair kernel:
//   g_k = sum_j J(D)(m_k w_j - m_j w_k),  J(D) u = f u + (f'(r)/r) D (D.u)
// for the pair law a = m D f(r).
// LAW 0 (Plummer): f = s^-3/2, f'/r = -3 s^-5/2.
// LAW 1 (spline): f = c0 + c1 r + c2 r^2 and f'/r = c1/r + 2 c2 for
//   r < eps_s, else f = r^-3 and f'/r = -3 r^-5. The branch is chosen by
//   comparing r with eps_s, not the two values as in the forward kernel:
//   the law is C^2 at eps_s, so near it the values agree to rounding and
//   either choice gives the same force, but the slopes f' differ at first
//   order in (r - eps_s)^2 and the wrong branch would show in J. At the self
//   pair (s at its 1e-30 floor) the polynomial branch is taken and every
//   factor is finite; u = 0 there, so the term is 0.
// Each pair's whole J u goes into one accumulator: the two parts of J u grow
// coherently over j (the -m_j w_k term points the same way for every j) and
// only cancel in their sum, so accumulating them apart loses precision.
// Sums are blocked per tile like the forward kernel.
template <int K, bool EQ, int LAW = 0>
__global__ void __launch_bounds__(512) k_vjp(PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    constexpr int NF = EQ ? 6 : 7;
    float *sbase = reinterpret_cast<float *>(smem_raw) + wib * (NF * kTile + 3 * a.tbl);
    float *sx = sbase, *sy = sbase + kTile, *sz = sbase + 2 * kTile;
    float *swx = sbase + 3 * kTile, *swy = sbase + 4 * kTile, *swz = sbase + 5 * kTile;
    float *sm = sbase + 6 * kTile;
    int *pfx = reinterpret_cast<int *>(sbase + NF * kTile);
    int *dlt = pfx + a.tbl, *ofs = dlt + a.tbl;
    const int n_items = a.st->n_items;

    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&a.st->queue_head, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const WorkItem w = a.items[it];
        const int box = w.box_s >> 8, log2s = w.box_s & 0xff;
        const int S = 1 << log2s, G = 32 >> log2s;
        const int g = lane >> log2s, sp = lane & (S - 1);
        const BoxDev B = a.boxes[box];
        const int nsrc = build_table(a, B, w.cell, pfx, dlt, ofs);
        const f2_t eps2 = f2_pack(B.eps2, B.eps2);
        f2_t c0 = 0ull, c1 = 0ull, c2 = 0ull, c2x2 = 0ull;
        float e_s = 0.f;
        if (LAW == 1) {
            c0 = f2_pack(B.sp_c0, B.sp_c0);
            c1 = f2_pack(B.sp_c1, B.sp_c1);
            c2 = f2_pack(B.sp_c2, B.sp_c2);
            c2x2 = f2_pack(2.f * B.sp_c2, 2.f * B.sp_c2);
            e_s = B.sp_eps;
        }

        f2_t xi[K], yi[K], zi[K], wxi[K], wyi[K], wzi[K], mi[K];
        f2_t gx[K], gy[K], gz[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int si = g + G * k;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f), wv = p;
            if (si < w.n) {
                p = a.sorted[w.first + si];
                wv = a.w_sorted[w.first + si];
            }
            xi[k] = f2_pack(p.x, p.x); yi[k] = f2_pack(p.y, p.y); zi[k] = f2_pack(p.z, p.z);
            wxi[k] = f2_pack(wv.x, wv.x); wyi[k] = f2_pack(wv.y, wv.y); wzi[k] = f2_pack(wv.z, wv.z);
            mi[k] = f2_pack(p.w, p.w);
            gx[k] = gy[k] = gz[k] = 0ull;
        }
        const f2_t minus3 = f2_pack(-3.0f, -3.0f);
        int ci = 0, co = 0;   // cell stream, as in k_pairs
        for (int q0 = 0; q0 < nsrc; q0 += kTile) {
            const int cntT = min(kTile, nsrc - q0);
            const int npair = (cntT + 1) >> 1;
            int filled = 0;
            while (filled < cntT && ci < a.nbr) {
                const int p0 = pfx[ci];
                const int left = pfx[ci + 1] - p0 - co;
                if (left <= 0) { ++ci; co = 0; continue; }
                const int take = min(left, cntT - filled);
                const int base = p0 + dlt[ci] + co;
                const int code = ofs[ci];
                const float ox = (float)((code & 0xff) - a.R);
                const float oy = (float)(((code >> 8) & 0xff) - a.R);
                const float oz = (float)((code >> 16) - a.R);
                for (int t = lane; t < take; t += 32) {
                    const float4 p = a.sorted[base + t];
                    const float4 wv = a.w_sorted[base + t];
                    sx[filled + t] = p.x + ox;
                    sy[filled + t] = p.y + oy;
                    sz[filled + t] = p.z + oz;
                    swx[filled + t] = wv.x; swy[filled + t] = wv.y; swz[filled + t] = wv.z;
                    if (!EQ) sm[filled + t] = p.w;
                }
                filled += take;
                co += take;
                if (take == left) { ++ci; co = 0; }
            }
            if ((cntT & 1) && lane == 0) {
                sx[cntT] = kFarAway; sy[cntT] = 0.f; sz[cntT] = 0.f;
                swx[cntT] = 0.f; swy[cntT] = 0.f; swz[cntT] = 0.f;
                if (!EQ) sm[cntT] = 0.f;
            }
            __syncwarp();
            const f2_t *px = reinterpret_cast<const f2_t *>(sx);
            const f2_t *py = reinterpret_cast<const f2_t *>(sy);
            const f2_t *pz = reinterpret_cast<const f2_t *>(sz);
            const f2_t *pwx = reinterpret_cast<const f2_t *>(swx);
            const f2_t *pwy = reinterpret_cast<const f2_t *>(swy);
            const f2_t *pwz = reinterpret_cast<const f2_t *>(swz);
            const f2_t *pm = reinterpret_cast<const f2_t *>(sm);
            f2_t tx[K], ty[K], tz[K];
#pragma unroll
            for (int k = 0; k < K; ++k) tx[k] = ty[k] = tz[k] = 0ull;
            const int n_it = (npair - sp + S - 1) >> log2s;
#pragma unroll 1
            for (int it = 0; it < n_it; ++it) {
                const int pp = sp + (it << log2s);
                const f2_t x2 = px[pp], y2 = py[pp], z2 = pz[pp];
                const f2_t wx2 = pwx[pp], wy2 = pwy[pp], wz2 = pwz[pp];
                f2_t m2 = 0ull;
                if (!EQ) m2 = pm[pp];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const f2_t dx = f2_sub(x2, xi[k]);
                    const f2_t dy = f2_sub(y2, yi[k]);
                    const f2_t dz = f2_sub(z2, zi[k]);
                    f2_t s = f2_fma(dx, dx, eps2);
                    s = f2_fma(dy, dy, s);
                    s = f2_fma(dz, dz, s);
                    const f2_t r = f2_rsqrt(s);
                    const f2_t r2 = f2_mul(r, r);
                    const f2_t r3 = f2_mul(r2, r);
                    const f2_t r5 = f2_mul(r3, r2);
                    f2_t ux, uy, uz;
                    if (EQ) {
                        ux = f2_sub(wx2, wxi[k]);
                        uy = f2_sub(wy2, wyi[k]);
                        uz = f2_sub(wz2, wzi[k]);
                    } else {
                        // m_k w_j - m_j w_k written as m_k (w_j - w_k) + (m_k - m_j) w_k:
                        // for the self pair every factor is an exact zero, so u
                        // stays 0 even if the compiler fuses a product into an
                        // FMA (the self pair carries the large weight eps^-3)
                        const f2_t dm = f2_sub(mi[k], m2);
                        ux = f2_fma(mi[k], f2_sub(wx2, wxi[k]), f2_mul(dm, wxi[k]));
                        uy = f2_fma(mi[k], f2_sub(wy2, wyi[k]), f2_mul(dm, wyi[k]));
                        uz = f2_fma(mi[k], f2_sub(wz2, wzi[k]), f2_mul(dm, wzi[k]));
                    }
                    f2_t du = f2_mul(dx, ux);
                    du = f2_fma(dy, uy, du);
                    du = f2_fma(dz, uz, du);
                    f2_t c, f = r3;
                    if (LAW == 0) {
                        c = f2_mul(f2_mul(du, r5), minus3);
                    } else {
                        const f2_t rr = f2_mul(s, r);
                        const f2_t poly = f2_fma(f2_fma(c2, rr, c1), rr, c0);
                        const f2_t dpoly = f2_fma(c1, r, c2x2);
                        const f2_t dout = f2_mul(r5, minus3);
                        float p0, p1, q0, q1, d0, d1, e0, e1, r0, r1;
                        f2_unpack(poly, p0, p1);
                        f2_unpack(r3, q0, q1);
                        f2_unpack(dpoly, d0, d1);
                        f2_unpack(dout, e0, e1);
                        f2_unpack(rr, r0, r1);
                        const bool in0 = r0 < e_s, in1 = r1 < e_s;
                        f = f2_pack(in0 ? p0 : q0, in1 ? p1 : q1);
                        c = f2_mul(du, f2_pack(in0 ? d0 : e0, in1 ? d1 : e1));
                    }
                    tx[k] = f2_fma(c, dx, f2_fma(f, ux, tx[k]));
                    ty[k] = f2_fma(c, dy, f2_fma(f, uy, ty[k]));
                    tz[k] = f2_fma(c, dz, f2_fma(f, uz, tz[k]));
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                gx[k] = f2_add(gx[k], tx[k]);
                gy[k] = f2_add(gy[k], ty[k]);
                gz[k] = f2_add(gz[k], tz[k]);
            }
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const f2_t gg[3] = {gx[k], gy[k], gz[k]};
            float v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float a0, a1;
                f2_unpack(gg[c], a0, a1);
                float s1 = a0 + a1;
                for (int o = 1; o < S; o <<= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                v[c] = s1;
            }
            const int si = g + G * k;
            if (sp == 0 && si < w.n) {
                const int i = a.perm[w.first + si];
                const float sc = EQ ? B.gm * B.inv_h3 : B.inv_h3;
                float *o = reinterpret_cast<float *>(a.out) + 3 * (int64_t)i;
                o[0] = v[0] * sc;
                o[1] = v[1] * sc;
                o[2] = v[2] * sc;
            }
        }
    }
}

// FP64 reference adjoint: one sink per lane, double arithmetic.
__global__ void __launch_bounds__(512) k_vjp_f64(PairArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *sbase = reinterpret_cast<double *>(smem_raw) +
                    wib * (7 * kTile + (3 * a.tbl + 1) / 2);
    double *sx = sbase, *sy = sbase + kTile, *sz = sbase + 2 * kTile;
    double *swx = sbase + 3 * kTile, *swy = sbase + 4 * kTile, *swz = sbase + 5 * kTile;
    double *sm = sbase + 6 * kTile;
    int *pfx = reinterpret_cast<int *>(sbase + 7 * kTile);
    int *dlt = pfx + a.tbl, *ofs = dlt + a.tbl;
    const int n_items = a.st->n_items;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&a.st->queue_head, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const WorkItem w = a.items[it];
        const int box = w.box_s >> 8, log2s = w.box_s & 0xff;
        const int S = 1 << log2s;
        const int g = lane >> log2s, sp = lane & (S - 1);
        const BoxDev B = a.boxes[box];
        const int nsrc = build_table(a, B, w.cell, pfx, dlt, ofs);
        double xi = 0, yi = 0, zi = 0, mk = 0, wxk = 0, wyk = 0, wzk = 0;
        if (g < w.n) {
            const dbl4 p = a.sorted_d[w.first + g];
            const float4 wv = a.w_sorted[w.first + g];
            xi = p.x; yi = p.y; zi = p.z; mk = p.w;
            wxk = wv.x; wyk = wv.y; wzk = wv.z;
        }
        double gx = 0, gy = 0, gz = 0;
        int ci = 0;
        for (int q0 = 0; q0 < nsrc; q0 += kTile) {
            const int cntT = min(kTile, nsrc - q0);
            for (int t = lane; t < cntT; t += 32) {
                const int q = q0 + t;
                const int c = locate(pfx, a.nbr, q, ci);
                const int j = q + dlt[c];
                const dbl4 p = a.sorted_d[j];
                const float4 wv = a.w_sorted[j];
                const int code = ofs[c];
                sx[t] = p.x + (double)((code & 0xff) - a.R);
                sy[t] = p.y + (double)(((code >> 8) & 0xff) - a.R);
                sz[t] = p.z + (double)((code >> 16) - a.R);
                swx[t] = wv.x; swy[t] = wv.y; swz[t] = wv.z;
                sm[t] = p.w;
            }
            __syncwarp();
            for (int j = sp; j < cntT; j += S) {
                const double dx = sx[j] - xi, dy = sy[j] - yi, dz = sz[j] - zi;
                const double s = dx * dx + dy * dy + dz * dz + B.eps2_d;
                const double r3 = 1.0 / (s * sqrt(s));
                const double r5 = r3 / s;
                // m_k w_j - m_j w_k, exactly 0 for the self pair (see k_vjp)
                const double dm = mk - sm[j];
                const double ux = mk * (swx[j] - wxk) + dm * wxk;
                const double uy = mk * (swy[j] - wyk) + dm * wyk;
                const double uz = mk * (swz[j] - wzk) + dm * wzk;
                const double du = dx * ux + dy * uy + dz * uz;
                gx += r3 * ux - 3.0 * r5 * du * dx;
                gy += r3 * uy - 3.0 * r5 * du * dy;
                gz += r3 * uz - 3.0 * r5 * du * dz;
            }
            __syncwarp();
        }
        for (int o = 1; o < S; o <<= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
        }
        if (sp == 0 && g < w.n) {
            const int i = a.perm[w.first + g];
            float *o = reinterpret_cast<float *>(a.out) + 3 * (int64_t)i;
            const double sc = B.inv_h3_d;
            o[0] = (float)(gx * sc); o[1] = (float)(gy * sc); o[2] = (float)(gz * sc);
        }
    }
}

// Sorted copy of the VJP cotangent: w_sorted[k] = w[perm[k]].
__global__ void k_gather_w(const float *__restrict__ w, int64_t n, const int *__restrict__ perm,
                           float4 *__restrict__ ws) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm[k];
        ws[k] = make_float4(w[3 * i], w[3 * i + 1], w[3 * i + 2], 0.f);
    }
}

// |a|^2 of a float32 acceleration for the momentum scale: the squares and
// the two sums each rounded to float32, in this order (no contraction).
__device__ __forceinline__ float mom_a2(float x, float y, float z) {
    return __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z));
}

// Warp, then block, reduction of s[0..3] into partial[4 * blockIdx.x + c].
__device__ __forceinline__ void mom_block_sum(double s[4], double *partial) {
    __shared__ double red[8][4];
    for (int c = 0; c < 4; ++c) {
        double x = s[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double x = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[w][threadIdx.x];
        partial[4 * blockIdx.x + threadIdx.x] = x;
    }
}

// a10: FP64 momentum diagnostic, P = sum_i m_i a_i (FP64 sums; a product of
// two floats is exact in FP64) and the scale S = sum_i m_i |a_i| (|a_i| a
// float32 magnitude: it only scales the check), two-level fixed-order
// reduction (deterministic). Per-particle masses: sinks in sorted order,
// m_i from the records, a_i gathered through the permutation.
__global__ void __launch_bounds__(256) k_momentum(const float4 *__restrict__ sorted,
                                                  const int *__restrict__ perm, const void *acc,
                                                  int f64, int64_t n, double *partial) {
    double s[4] = {0, 0, 0, 0};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm[k];
        const double m = sorted[k].w;
        double v[3];
        float a2;
        if (f64) {
            const double *p = reinterpret_cast<const double *>(acc) + 3 * i;
            v[0] = p[0]; v[1] = p[1]; v[2] = p[2];
            a2 = (float)(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        } else {
            const float *p = reinterpret_cast<const float *>(acc) + 3 * i;
            const float x = p[0], y = p[1], z = p[2];
            v[0] = x; v[1] = y; v[2] = z;
            a2 = mom_a2(x, y, z);
        }
        s[0] += m * v[0];
        s[1] += m * v[1];
        s[2] += m * v[2];
        s[3] += m * (double)sqrtf(a2);
    }
    mom_block_sum(s, partial);
}

// The same for equal masses (one G m per box): particles in input order, so
// the accelerations are read contiguously and neither the records nor the
// permutation are needed. One box (MULTI false): the sums of a_i and |a_i|,
// scaled by G m in the final kernel; several boxes: each term takes its
// box's G m.
template <bool MULTI>
__global__ void __launch_bounds__(256) k_momentum_eq(const void *acc, int f64, int64_t n,
                                                     const int64_t *__restrict__ poff, int n_boxes,
                                                     const BoxDev *__restrict__ boxes, double *partial) {
    double s[4] = {0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v[3];
        float a2;
        if (f64) {
            const double *p = reinterpret_cast<const double *>(acc) + 3 * i;
            v[0] = p[0]; v[1] = p[1]; v[2] = p[2];
            a2 = (float)(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        } else {
            const float *p = reinterpret_cast<const float *>(acc) + 3 * i;
            const float x = p[0], y = p[1], z = p[2];
            v[0] = x; v[1] = y; v[2] = z;
            a2 = mom_a2(x, y, z);
        }
        const double r = (double)sqrtf(a2);
        if (MULTI) {
            const double m = boxes[box_of_particle(poff, n_boxes, i)].gm_d;
            s[0] += m * v[0];
            s[1] += m * v[1];
            s[2] += m * v[2];
            s[3] += m * r;
        } else {
            s[0] += v[0];
            s[1] += v[1];
            s[2] += v[2];
            s[3] += r;
        }
    }
    mom_block_sum(s, partial);
}

__global__ void k_momentum_final(const double *partial, int nb, const BoxDev *boxes, int scale_by_gm,
                                 double *out) {
    if (threadIdx.x < 4) {
        double x = 0;
        for (int b = 0; b < nb; ++b) x += partial[4 * b + threadIdx.x];
        out[threadIdx.x] = scale_by_gm ? boxes[0].gm_d * x : x;
    }
}

template <typename F>
void *fptr(F f) { return reinterpret_cast<void *>(f); }

void *pair_kernel_ext(int K, int eq, int law, int kde) {
#define NF_SEL2(KK, EE)                                                          \
    if (K == KK && eq == EE) {                                                   \
        if (law == 0) return fptr(k_pairs<KK, EE, 0, 0, true>);                  \
        return kde ? fptr(k_pairs<KK, EE, 0, 1, true>)                           \
                   : fptr(k_pairs<KK, EE, 0, 1, false>);                         \
    }
    NF_SEL2(1, 0) NF_SEL2(1, 1) NF_SEL2(2, 0) NF_SEL2(2, 1) NF_SEL2(4, 0) NF_SEL2(4, 1)
#undef NF_SEL2
    return nullptr;
}

void *pair_kernel(int prec, int K, int eq, int law = 0, int kde = 0, int tile = kTile) {
    if (prec == NF_PREC_FP64_REF) return fptr(k_pairs_f64);
    if (law != 0 || kde) return prec == NF_PREC_FP32 ? pair_kernel_ext(K, eq, law, kde) : nullptr;
    const int comp = prec == NF_PREC_FP32_COMP ? 1 : (prec == NF_PREC_FP32_COMP_PAIR ? 2 : 0);
#define NF_SELT(KK, EE, CC)                                                               \
    if (K == KK && eq == EE && comp == CC) {                                              \
        if (tile == 64) return fptr(k_pairs<KK, EE, CC, 0, false, 64>);                   \
        if (tile == 256) return fptr(k_pairs<KK, EE, CC, 0, false, 256>);                 \
        return fptr(k_pairs<KK, EE, CC, 0, false, 128>);                                  \
    }
#define NF_SEL(KK) \
    NF_SELT(KK, 1, 0) NF_SELT(KK, 1, 1) NF_SELT(KK, 1, 2) NF_SELT(KK, 0, 0) NF_SELT(KK, 0, 1) NF_SELT(KK, 0, 2)
    NF_SEL(1)
    NF_SEL(2)
    NF_SEL(4)
#undef NF_SEL
#undef NF_SELT
    return nullptr;
}

void *vjp_kernel(int prec, int K, int eq, int law) {
    if (prec == NF_PREC_FP64_REF) return law == 0 ? fptr(k_vjp_f64) : nullptr;
#define NF_SELV(KK)                                                                    \
    if (K == KK) {                                                                     \
        if (law == 1) return eq ? fptr(k_vjp<KK, true, 1>) : fptr(k_vjp<KK, false, 1>); \
        return eq ? fptr(k_vjp<KK, true>) : fptr(k_vjp<KK, false>);                     \
    }
    NF_SELV(1)
    NF_SELV(2)
    NF_SELV(4)
#undef NF_SELV
    return nullptr;
}

int table_stride(int R) {
    const int nbr = (2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    return (nbr + 1 + 3) & ~3;
}

size_t smem_per_warp(int prec, int R, int eq, int vjp, int tile = kTile) {
    const int tbl = table_stride(R);
    if (prec == NF_PREC_FP64_REF) {
        const int nf = vjp ? 7 : 4;
        return sizeof(double) * (size_t)(nf * kTile + (3 * tbl + 1) / 2);
    }
    const int nf = vjp ? (eq ? 6 : 7) : (eq ? 3 : 4);
    return sizeof(float) * (size_t)(nf * (vjp ? kTile : tile) + 3 * tbl);
}

cudaError_t prepare(void *fn, size_t smem) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_generic(Ctx *c, void *fn, int vjp, const PairArgs &args, const nf_tuning &t,
                           cudaStream_t s, int tile = kTile) {
    const int warps = t.warps_per_block;
    const size_t smem = smem_per_warp(c->precision, c->R, c->equal_mass, vjp, tile) * warps;
    cudaError_t e = prepare(fn, smem);
    if (e) return e;
    int per_sm = t.blocks_per_sm;
    if (per_sm <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem);
        if (e) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const int grid = c->sm_count * per_sm;
    void *params[] = {const_cast<PairArgs *>(&args)};
    c->launches += 1;
    return cudaLaunchKernel(fn, dim3(grid), dim3(warps * 32), params, smem, s);
}

PairArgs make_args(Ctx *c, void *out, int out_f64) {
    PairArgs a;
    a.sorted = c->sorted;
    a.sorted_d = c->sorted_d;
    a.w_sorted = c->w_sorted;
    a.cell_start = c->cell_start;
    a.perm = c->perm;
    a.boxes = c->boxes_d;
    a.items = c->items;
    a.st = c->state;
    a.out = out;
    a.out_f64 = out_f64;
    a.R = c->R;
    a.nbr = (2 * c->R + 1) * (2 * c->R + 1) * (2 * c->R + 1);
    a.tbl = table_stride(c->R);
    a.dens = nullptr;
    a.n_boxes = c->n_boxes;
    return a;
}

}  // namespace

// Remainder decomposition: for r sinks left over after full items of 32K,
// pick items (count, S) minimising the modelled warp time
// sum_items n_src * (22 K / S + 1.5), the two terms being pair arithmetic
// per lane and per-source staging/loop overhead.
void make_decomp(int K, Decomp *d) {
    const int full = 32 * K;
    double best[129];
    int choice[129];
    best[0] = 0;
    choice[0] = -1;
    for (int r = 1; r < full; ++r) {
        best[r] = 1e30;
        choice[r] = 0;
        for (int l = 0; l <= 5; ++l) {
            const int slots = full >> l;
            if (slots < 1) continue;
            const double cost = 22.0 * K / (1 << l) + 1.5;
            const double tot = slots >= r ? cost : cost + best[r - slots];
            if (tot < best[r] - 1e-12) {
                best[r] = tot;
                choice[r] = l;
            }
        }
    }
    for (int r = 0; r < 128; ++r) {
        d->n_entries[r] = 0;
        if (r == 0 || r >= full) continue;
        int left = r;
        while (left > 0) {
            int l = choice[left];
            if (d->n_entries[r] == kDecompMax - 1)   // last slot: cover the rest
                for (l = 5; l > 0 && (full >> l) < left; --l) {}
            const int slots = full >> l;
            const int take = slots >= left ? left : slots;
            d->entry[r][d->n_entries[r]++] = (take << 8) | l;
            left -= take;
        }
    }
}

cudaError_t launch_worklist(Ctx *c, cudaStream_t s, bool pencils, bool small) {
    cudaError_t e;
    // reset counters (everything but the error word)
    if ((e = cudaMemsetAsync(&c->state->n_items, 0, sizeof(DevState) - sizeof(int), s))) return e;
    WLArgs a;
    a.boxes = c->boxes_d;
    a.n_boxes = c->n_boxes;
    a.R = c->R;
    a.K = c->decomp_k;
    a.n_cells = c->n_sink_cells;
    a.count = c->count;
    a.cell_start = c->cell_start;
    a.nsrc_cell = c->nsrc_cell;
    a.decomp = c->decomp_d + (c->decomp_k == 1 ? 0 : (c->decomp_k == 2 ? 1 : 2));
    a.st = c->state;
    a.items = c->items;
    a.pencils_on = pencils ? 1 : 0;
    a.small_on = small ? 1 : 0;
    a.pencil_ok = c->pencil_ok;
    a.pencils = c->pencils;
    const unsigned blocks = (unsigned)((c->n_sink_cells + 255) / 256 + (c->n_sink_cells == 0));
    if (pencils) {
        k_wl_pencils<<<blocks, 256, 0, s>>>(a);
        c->launches += 1;
    }
    k_wl_count<<<blocks, 256, 0, s>>>(a);
    k_wl_scan<<<1, 32, 0, s>>>(c->state);
    k_wl_write<<<blocks, 256, 0, s>>>(a);
    c->launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_pairs(Ctx *c, void *acc, int out_f64, const nf_tuning &t, cudaStream_t s,
                         float *dens) {
    const int K = c->precision == NF_PREC_FP64_REF ? 1 : t.sinks_per_lane;
    const int law = c->softening == NF_SOFT_SPLINE ? 1 : 0;
    // the source tile is a tuning choice of the plain Plummer kernels only
    const int tile = (law == 0 && !dens && c->precision != NF_PREC_FP64_REF && t.source_tile) ? t.source_tile
                                                                                             : kTile;
    void *fn = pair_kernel(c->precision, K, c->equal_mass, law, dens != nullptr, tile);
    if (!fn) return cudaErrorInvalidValue;
    PairArgs args = make_args(c, acc, out_f64);
    args.dens = dens;
    cudaError_t e = launch_generic(c, fn, 0, args, t, s, tile);
    if (!e && small_active(c, t, dens == nullptr && !out_f64)) {
        // the small items, after the tiled ones
        void *sf = c->equal_mass ? fptr(k_pairs_small<true>) : fptr(k_pairs_small<false>);
        const size_t smem = sizeof(int) * 4 * (size_t)args.tbl * 4;
        int per_sm = 0;
        if (!e) e = prepare(sf, smem);
        if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sf, 128, smem);
        if (per_sm < 1) per_sm = 1;
        void *sparams[] = {&args};
        if (!e) {
            c->launches += 1;
            e = cudaLaunchKernel(sf, dim3(c->sm_count * per_sm), dim3(128), sparams, smem, s);
        }
    }
    if (e || !pencils_active(c, t, dens == nullptr && !out_f64)) return e;
    // the pencils, after the other items
    void *pf = c->equal_mass ? fptr(k_pencils<true>) : fptr(k_pencils<false>);
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pf, 32 * kPencil, 0))) return e;
    if (per_sm < 1) per_sm = 1;
    const int *pens = c->pencils;
    void *params[] = {&args, &pens};
    c->launches += 1;
    return cudaLaunchKernel(pf, dim3(c->sm_count * per_sm), dim3(32 * kPencil), params, 0, s);
}

// The pencil kernel serves the plain FP32 Plummer forward pass with FP32
// output and no density, at K = 4 and R <= 2, when the tuning allows it.
bool small_active(const Ctx *c, const nf_tuning &t, bool plain_out) {
    return t.small_items && plain_out && c->precision == NF_PREC_FP32 && c->softening == NF_SOFT_PLUMMER &&
           t.sinks_per_lane == 4;
}

bool pencils_active(const Ctx *c, const nf_tuning &t, bool plain_out) {
    return t.use_pencils && plain_out && c->precision == NF_PREC_FP32 &&
           c->softening == NF_SOFT_PLUMMER && c->R <= 2 && t.sinks_per_lane == 4;
}

cudaError_t launch_vjp(Ctx *c, const float *w, float *grad, const nf_tuning &t, cudaStream_t s) {
    if (c->n > 0) {
        const int64_t n = c->n;
        int grid = (int)((n + 255) / 256);
        if (grid > c->sm_count * 8) grid = c->sm_count * 8;
        k_gather_w<<<grid, 256, 0, s>>>(w, n, c->perm, c->w_sorted);
        c->launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e) return e;
    }
    const int K = c->precision == NF_PREC_FP64_REF ? 1 : t.sinks_per_lane;
    void *fn = vjp_kernel(c->precision, K, c->equal_mass, c->softening == NF_SOFT_SPLINE ? 1 : 0);
    if (!fn) return cudaErrorInvalidValue;
    return launch_generic(c, fn, 1, make_args(c, grad, 0), t, s);
}

cudaError_t launch_momentum(Ctx *c, const void *acc, int acc_f64, cudaStream_t s) {
    const bool one_box = c->n_boxes == 1;
    if (!c->equal_mass)
        k_momentum<<<kMomBlocks, 256, 0, s>>>(c->sorted, c->perm, acc, acc_f64, c->n, c->mom_partial);
    else if (one_box)
        k_momentum_eq<false><<<kMomBlocks, 256, 0, s>>>(acc, acc_f64, c->n, c->poff_d, c->n_boxes,
                                                        c->boxes_d, c->mom_partial);
    else
        k_momentum_eq<true><<<kMomBlocks, 256, 0, s>>>(acc, acc_f64, c->n, c->poff_d, c->n_boxes,
                                                       c->boxes_d, c->mom_partial);
    k_momentum_final<<<1, 32, 0, s>>>(c->mom_partial, kMomBlocks, c->boxes_d, c->equal_mass && one_box,
                                      c->mom_result);
    c->launches += 2;
    return cudaGetLastError();
}

}  // namespace nf

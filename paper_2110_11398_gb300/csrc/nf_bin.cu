// nf_bin.cu -- cell binning (the cubic cell lattice of Maksimova et al. 2021,
// Sec. 3.1): per-particle cell id, per-cell count, exclusive prefix scan,
// stable sort by cell (LSD radix sort whose digit ranks keep input order) and
// the gather into cell-sorted float4 records of cell-relative coordinates.
//
// Cell arithmetic, identical on every device and host: u = (x * CPD) / L in
// IEEE double with no contraction, cell = floor(u) (CPD rounds down to
// CPD-1), relative coordinate float32(u - (cell + 0.5)) in cell units.
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
constexpr int kRadixThreads = 256;                  // 8 warps
constexpr int kRadixItems = 16;                     // chunks of 32 per warp
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixTile = kRadixThreads * kRadixItems;  // 4096 keys
constexpr int kRadixDigits = 256;

__device__ __forceinline__ int box_of_particle(const int64_t *poff, int n_boxes, int64_t i) {
    int lo = 0, hi = n_boxes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (poff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

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

// a1 + a2: cell id of every particle and per-cell counts.
__global__ void k_cell_ids(const float *__restrict__ pos, int64_t n,
                           const int64_t *__restrict__ poff, int n_boxes,
                           const BoxDev *__restrict__ boxes, int pow2,
                           int *__restrict__ cid, int *__restrict__ count,
                           DevState *st) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i - lane < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool live = i < n;
        int cell = -1;
        if (live) {
            const int b = n_boxes == 1 ? 0 : box_of_particle(poff, n_boxes, i);
            const BoxDev B = boxes[b];
            int c3[3];
            bool ok = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float xf = pos[3 * i + a];
                // range test (false for NaN); for a power-of-two L, L is a
                // float and the test is exact in FP32
                const bool in = pow2 ? (xf >= 0.f && xf < B.Lf)
                                     : ((double)xf >= 0.0 && (double)xf < B.L);
                ok = ok && in;
                int cc = 0;
                float rr;
                if (in && !(pow2 && cell_rel_pow2(xf, (float)B.cpd, B.inv_Lf, B.cpd, cc, rr)))
                    cc = cell_index(cell_unit((double)xf, B, pow2 != 0), B.cpd);
                c3[a] = cc;
            }
            if (!ok) atomicOr(&st->error, 1);
            cell = B.cell_off + (c3[0] * B.cpd + c3[1]) * B.cpd + c3[2];
            cid[i] = cell;
        }
        // warp-aggregated histogram: particles in input order are often
        // spatially coherent, so many lanes hit the same counter
        const unsigned live_mask = __ballot_sync(0xffffffffu, live);
        if (live) {
            const unsigned peers = __match_any_sync(live_mask, cell);
            if (lane == __ffs(peers) - 1) atomicAdd(&count[cell], __popc(peers));
        }
    }
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

// ------------------------------------------------------------ radix sort
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Digit histogram of one tile; hist is digit-major: hist[d * ntiles + tile].
__global__ void __launch_bounds__(kRadixThreads)
k_radix_upsweep(const int *__restrict__ keys, int64_t n, int shift, int64_t ntiles,
                int *__restrict__ hist) {
    __shared__ int h[kRadixDigits];
    for (int d = threadIdx.x; d < kRadixDigits; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kRadixTile + warp * (32 * kRadixItems);
#pragma unroll 4
    for (int c = 0; c < kRadixItems; ++c) {
        const int64_t idx = base + c * 32 + lane;
        const bool live = idx < n;
        const int d = live ? ((keys[idx] >> shift) & 0xff) : (0x100 + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (live && lane == __ffs(peers) - 1) atomicAdd(&h[d], __popc(peers));
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixDigits; d += blockDim.x)
        hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter of one tile: warps own consecutive sub-tiles, chunks of 32
// are ranked in order with match_any, so equal digits keep input order.
// vals_in == nullptr means the identity (first pass).
__global__ void __launch_bounds__(kRadixThreads)
k_radix_downsweep(const int *__restrict__ keys_in, const int *__restrict__ vals_in, int64_t n,
                  int shift, int64_t ntiles, const int *__restrict__ hist_scanned,
                  int *__restrict__ keys_out, int *__restrict__ vals_out, int write_keys) {
    __shared__ int woff[kRadixWarps][kRadixDigits];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kRadixWarps * kRadixDigits; d += blockDim.x)
        (&woff[0][0])[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile + warp * (32 * kRadixItems);
    int key[kRadixItems], dig[kRadixItems];
#pragma unroll
    for (int c = 0; c < kRadixItems; ++c) {
        const int64_t idx = base + c * 32 + lane;
        const bool live = idx < n;
        key[c] = live ? keys_in[idx] : 0;
        dig[c] = live ? ((key[c] >> shift) & 0xff) : (0x100 + lane);
    }
    // per-warp digit counts
#pragma unroll
    for (int c = 0; c < kRadixItems; ++c) {
        const unsigned peers = __match_any_sync(0xffffffffu, dig[c]);
        if (dig[c] < 0x100 && lane == __ffs(peers) - 1) woff[warp][dig[c]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive scan over warps per digit, plus the tile's global base
    for (int d = threadIdx.x; d < kRadixDigits; d += blockDim.x) {
        int run = hist_scanned[(int64_t)d * ntiles + blockIdx.x];
        for (int w = 0; w < kRadixWarps; ++w) {
            int t = woff[w][d];
            woff[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int c = 0; c < kRadixItems; ++c) {
        const unsigned peers = __match_any_sync(0xffffffffu, dig[c]);
        const bool live = dig[c] < 0x100;
        int dest = 0;
        if (live) dest = woff[warp][dig[c]] + __popc(peers & lt);
        __syncwarp();
        if (live && lane == __ffs(peers) - 1) woff[warp][dig[c]] += __popc(peers);
        __syncwarp();
        if (live) {
            const int64_t idx = base + c * 32 + lane;
            const int v = vals_in ? vals_in[idx] : (int)idx;
            if (write_keys) keys_out[dest] = key[c];
            vals_out[dest] = v;
        }
    }
}

// a4 + a5: sorted record k = particle perm[k]: cell-relative coordinates in
// cell units and its mass.
__global__ void k_gather(const float *__restrict__ pos, const float *__restrict__ mass, float m0,
                         int64_t n, const int *__restrict__ perm,
                         const int64_t *__restrict__ poff, int n_boxes,
                         const BoxDev *__restrict__ boxes, int pow2,
                         float4 *__restrict__ sorted, dbl4 *__restrict__ sorted_d) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int i = perm[k];
        const int b = n_boxes == 1 ? 0 : box_of_particle(poff, n_boxes, i);
        const BoxDev B = boxes[b];
        float rf[3];
        double rd[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float xf = pos[3 * (int64_t)i + a];
            const double x = (double)xf;
            const bool in = pow2 ? (xf >= 0.f && xf < B.Lf) : (x >= 0.0 && x < B.L);
            int c;
            float r32;
            if (in && !sorted_d && pow2 && cell_rel_pow2(xf, (float)B.cpd, B.inv_Lf, B.cpd, c, r32)) {
                rf[a] = r32;
                rd[a] = (double)r32;
            } else {
                const double u = in ? cell_unit(x, B, pow2 != 0) : 0.5;
                c = in ? cell_index(u, B.cpd) : 0;
                rd[a] = __dsub_rn(u, (double)c + 0.5);
                rf[a] = __double2float_rn(rd[a]);
            }
        }
        const float m = mass ? mass[i] : B.gm;
        sorted[k] = make_float4(rf[0], rf[1], rf[2], m);
        if (sorted_d) sorted_d[k] = dbl4_make(rd[0], rd[1], rd[2], (double)m);
    }
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
int64_t radix_tiles(int64_t n) { return (n + kRadixTile - 1) / kRadixTile; }

cudaError_t launch_bin(Ctx *c, const float *pos, const float *mass, float m0, int64_t n,
                       cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->count, 0, sizeof(int) * c->n_cells, s))) return e;
    if ((e = cudaMemsetAsync(&c->state->error, 0, sizeof(int), s))) return e;
    if (n > 0) {
        k_cell_ids<<<grid_for(n, 256, c->sm_count), 256, 0, s>>>(
            pos, n, c->poff_d, c->n_boxes, c->boxes_d, c->pow2_all, c->keys_a, c->count, c->state);
        if ((e = cudaGetLastError())) return e;
        c->launches += 1;
    }
    if ((e = scan_exclusive(c->count, c->cell_start, c->n_cells, c->scan_tmp, s, &c->launches))) return e;
    if (n == 0) {
        c->perm = c->vals_a;
        return cudaSuccess;
    }
    // passes of 8 bits over the used key bits
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < c->n_cells) ++bits;
    const int passes = bits <= 8 ? 1 : (bits + 7) / 8;
    const int64_t nt = radix_tiles(n);
    int *kin = c->keys_a, *kout = c->keys_b;
    int *vin = nullptr, *vout = c->vals_a;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_radix_upsweep<<<(unsigned)nt, kRadixThreads, 0, s>>>(kin, n, shift, nt, c->radix_hist);
        if ((e = cudaGetLastError())) return e;
        if ((e = scan_exclusive(c->radix_hist, c->radix_hist, nt * kRadixDigits, c->scan_tmp, s,
                                    &c->launches)))
            return e;
        const int last = p == passes - 1;
        k_radix_downsweep<<<(unsigned)nt, kRadixThreads, 0, s>>>(
            kin, vin, n, shift, nt, c->radix_hist, kout, vout, !last);
        if ((e = cudaGetLastError())) return e;
        c->launches += 2;
        // ping-pong
        int *t = kin; kin = kout; kout = t;
        vin = vout;
        vout = (vout == c->vals_a) ? c->vals_b : c->vals_a;
    }
    c->perm = vin;
    k_gather<<<grid_for(n, 256, c->sm_count), 256, 0, s>>>(
        pos, mass, m0, n, c->perm, c->poff_d, c->n_boxes, c->boxes_d, c->pow2_all, c->sorted,
        c->precision == NF_PREC_FP64_REF ? c->sorted_d : nullptr);
    c->launches += 1;
    return cudaGetLastError();
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
constexpr int64_t kNoAllocTiles = (kNoAllocMaxParticles + nf::kRadixTile - 1) / nf::kRadixTile;
constexpr int64_t kNoAllocScanInts = 256;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffKeysA = 0;
constexpr size_t kOffKeysB = kOffKeysA + align256(4 * kNoAllocMaxParticles);
constexpr size_t kOffValsA = kOffKeysB + align256(4 * kNoAllocMaxParticles);
constexpr size_t kOffValsB = kOffValsA + align256(4 * kNoAllocMaxParticles);
constexpr size_t kOffCount = kOffValsB + align256(4 * kNoAllocMaxParticles);
constexpr size_t kOffHist = kOffCount + align256(4 * kNoAllocMaxCells);
constexpr size_t kOffScan = kOffHist + align256(4 * (nf::kRadixDigits * kNoAllocTiles + 1));
constexpr size_t kOffState = kOffScan + align256(4 * kNoAllocScanInts);
constexpr size_t kOffBox = kOffState + align256(sizeof(nf::DevState));
constexpr size_t kOffPoff = kOffBox + align256(sizeof(nf::BoxDev));
constexpr size_t kNoAllocBytes = kOffPoff + align256(2 * sizeof(int64_t));   // about 17.3 MB

// Shared by every call on a device and kept (with the last call's contents)
// until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_base[kNoAllocMaxDevices] = {};
int g_noalloc_sms[kNoAllocMaxDevices] = {};

// Device address of the array on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up
// once per device with that device current.
int noalloc_setup(int dev, unsigned char **base, int *sms) {
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
    if (noalloc_setup(dev, &base, &sms) != NF_OK) {
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
    c.radix_hist = reinterpret_cast<int *>(base + kOffHist);
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
    if (!e && n > 0) e = cudaMemcpyAsync(perm, c.perm, sizeof(int) * n, cudaMemcpyDeviceToDevice, s);
    int err_word = 0;
    if (!e) e = cudaMemcpyAsync(&err_word, &c.state->error, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) {
        cudaGetLastError();
        set_thread_error(cudaGetErrorString(e));
        return NF_ECUDA;
    }
    if (err_word) {
        set_thread_error("nf_bin_cells_noalloc: a position component is not finite or outside [0, L)");
        return NF_ERANGE;
    }
    return NF_OK;
}

// nf_step.cu -- particle update of the leapfrog integrator with a global
// timestep (Maksimova et al. 2021, Sec. 2.5): kick, drift (wrapped into the
// periodic box), and the small-scale timestep criterion, the minimum over
// cells of velocity dispersion / maximum particle acceleration times eta.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nf_ctx.h"
#include "nf_internal.cuh"

namespace nf {

namespace {

// v += a * h, element by element over N x 3, in double: the product and the
// sum are each rounded (no fused multiply-add, so the sequence is the plain
// IEEE one), then the result is rounded once to float (a float h would carry
// its own rounding into every update).
__global__ void k_kick(float *__restrict__ vel, const float *__restrict__ acc, int64_t n3, double h) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x)
        vel[i] = (float)__dadd_rn((double)vel[i], __dmul_rn((double)acc[i], h));
}

__device__ __forceinline__ int box_of(const int64_t *poff, int n_boxes, int64_t i) {
    int lo = 0, hi = n_boxes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (poff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// x += v * dt in double (product and sum each rounded, no fused
// multiply-add), wrapped into [0, L) of the particle's box by the exact
// remainder fmod(x, L) plus L when that is negative, rounded once to float;
// a value that rounds up to L is the periodic image of 0.
__global__ void k_drift(float *__restrict__ pos, const float *__restrict__ vel, int64_t n,
                        const int64_t *__restrict__ poff, int n_boxes,
                        const BoxDev *__restrict__ boxes, double dt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = n_boxes == 1 ? 0 : box_of(poff, n_boxes, i);
        const double L = boxes[b].L;
        const float Lf = (float)L;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double x = __dadd_rn((double)pos[3 * i + a], __dmul_rn(dt, (double)vel[3 * i + a]));
            double r = fmod(x, L);                  // exact
            if (r < 0.0) r = __dadd_rn(r, L);
            else if (r == 0.0) r = 0.0;             // -0 becomes +0
            float f = (float)r;
            if (f >= Lf || f < 0.f) f = 0.f;
            pos[3 * i + a] = f;
        }
    }
}

// One warp per cell: n, sum v, sum |v|^2 (double) and max |a|^2 over the
// cell's particles (cell order from the last binning); the cell's bound
// sigma_v / max|a| goes into an atomic minimum over the float bit pattern
// (non-negative floats order like their bits).
__global__ void k_cell_timestep(const float *__restrict__ vel, const float *__restrict__ acc,
                                const int *__restrict__ cell_start, const int *__restrict__ perm,
                                int64_t n_cells, unsigned *__restrict__ best_bits) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = warp; c < n_cells; c += nwarps) {
        const int s = cell_start[c], e = cell_start[c + 1];
        if (e - s < 2) continue;
        double sx = 0, sy = 0, sz = 0, svv = 0;
        float amax2 = 0.f;
        for (int k = s + lane; k < e; k += 32) {
            const int64_t i = perm[k];
            const double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
            sx += vx; sy += vy; sz += vz;
            svv += vx * vx + vy * vy + vz * vz;
            const float ax = acc[3 * i], ay = acc[3 * i + 1], az = acc[3 * i + 2];
            amax2 = fmaxf(amax2, ax * ax + ay * ay + az * az);
        }
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
            svv += __shfl_xor_sync(0xffffffffu, svv, o);
            amax2 = fmaxf(amax2, __shfl_xor_sync(0xffffffffu, amax2, o));
        }
        if (lane == 0 && amax2 > 0.f) {
            const double m = (double)(e - s);
            double var = svv / m - (sx * sx + sy * sy + sz * sz) / (m * m);
            var = var > 0.0 ? var : 0.0;
            const float r = (float)(sqrt(var) / sqrt((double)amax2));
            atomicMin(best_bits, __float_as_uint(r));
        }
    }
}

int grid_for(int64_t n, int threads, int sm_count) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_kick(Ctx *c, float *vel, const float *acc, double h, cudaStream_t s) {
    if (c->n == 0) return cudaSuccess;
    k_kick<<<grid_for(3 * c->n, 256, c->sm_count), 256, 0, s>>>(vel, acc, 3 * c->n, h);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_drift(Ctx *c, float *pos, const float *vel, double dt, cudaStream_t s) {
    if (c->n == 0) return cudaSuccess;
    k_drift<<<grid_for(c->n, 256, c->sm_count), 256, 0, s>>>(pos, vel, c->n, c->poff_d, c->n_boxes,
                                                             c->boxes_d, dt);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_cell_timestep(Ctx *c, const float *vel, const float *acc, unsigned *best_bits,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(best_bits, 0x7f, sizeof(unsigned), s);   // 0x7f7f7f7f: a huge float
    if (e) return e;
    const int64_t threads = 32 * c->n_sink_cells;
    k_cell_timestep<<<grid_for(threads, 256, c->sm_count), 256, 0, s>>>(vel, acc, c->cell_start, c->perm,
                                                                        c->n_sink_cells, best_bits);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace nf

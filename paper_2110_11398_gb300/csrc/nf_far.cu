// nf_far.cu -- far field of the near/far split (Maksimova et al. 2021,
// Sec. 3.1): Taylor series of order p about every cell centre, whose
// coefficients are the cyclic convolution, over the CPD^3 cells and carried
// out in Fourier space, of the cells' multipole moments with the derivatives
// tensor of the periodic Green's function; the tensor depends on the grid
// only and is built once per context.
//
// Conventions (cell units, origin at the cell centre):
//   multipoles    M_m(c)  = sum_{j in c} G m_j z_j^m,          |m| <= p
//   tensor        D_q(d)  = sum over periodic images of d^q (1/r) at d + n CPD,
//                           the image inside the near field ([-R, R]^3) left
//                           out; Ewald sum with a uniform background, |q| <= 2p
//   Taylor        T_k(c)  = sum_c' sum_m (-1)^|m| / m!  D_{k+m}(c - c') M_m(c')
//   acceleration  a(y)    = grad_y sum_k T_k y^k / k!   (times (CPD / L)^2)
// Away from its sources the tensor is harmonic: D_{q+2x} + D_{q+2y} + D_{q+2z}
// = 0 for |q| >= 1 (4 pi / CPD^3 for q = 0, the background). Hence (i) a
// multipole term with x-exponent >= 2 equals minus the same term moved to
// m - 2x + 2y and m - 2x + 2z, so the weighted multipoles W_m = (-1)^|m|/m! M_m
// fold down to the 2l+1 per order with x-exponent <= 1 ("reduced" set); and
// (ii) only the reduced T_k need the convolution, the others following from
// T_k = -T_{k-2x+2y} - T_{k-2x+2z} (plus 4 pi M_tot / CPD^3 for k = (2,0,0)).
// With p = 8 that is 81 x 81 products per frequency instead of 165 x 165,
// 162 transforms per step instead of 330, and the tensor is stored only for
// x-exponents <= 2.
// The tensor is real and has the parity of its order, D_q(-d) = (-1)^|q|
// D_q(d) (1/r is even, and the image sum and the near block are symmetric),
// so its transform is i^|q| times a real function E_q. Only E_q is kept, and
// T_k = i^|k| sum_m E_{k+m} (i^|m| W_m): a real number times a complex one per
// product, half the arithmetic and half the storage of complex products.
// The tensor is split as in Ewald's method: d^q [erfc(alpha r)/r] summed in
// real space over the few lattice vectors it reaches (once, on the GPU), and
// the rest, (4 pi / k^2) exp(-k^2 / 4 alpha^2) (i k)^q, written straight into
// its discrete Fourier transform. cuFFT does the transforms; the multipoles,
// the per-frequency products and the Taylor gradient are kernels here.
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "nf_ctx.h"
#include "nf_internal.cuh"

namespace nf {

// Multi-indices (a, b, c), a + b + c <= n, enumerated by degree, then c
// ascending, then b ascending (a = degree - b - c).
struct MultiIndex {
    int n = 0;
    std::vector<int> a, b, c;
    std::vector<int> pos;   // (a, b, c) -> position, (n+1)^3 table, -1 where a+b+c > n
    void build(int order) {
        n = order;
        a.clear(); b.clear(); c.clear();
        pos.assign((size_t)(n + 1) * (n + 1) * (n + 1), -1);
        for (int t = 0; t <= n; ++t)
            for (int cc = 0; cc <= t; ++cc)
                for (int bb = 0; bb <= t - cc; ++bb) {
                    const int aa = t - bb - cc;
                    pos[((size_t)aa * (n + 1) + bb) * (n + 1) + cc] = (int)a.size();
                    a.push_back(aa); b.push_back(bb); c.push_back(cc);
                }
    }
    int size() const { return (int)a.size(); }
    int at(int aa, int bb, int cc) const { return pos[((size_t)aa * (n + 1) + bb) * (n + 1) + cc]; }
};

// Derivatives tensor of one CPD (boxes of equal CPD share it) and the
// batched transform plans of that size.
struct FarTensor {
    int P = 0;
    int64_t ncell = 0, nfreq = 0;
    double *E = nullptr;               // [nd][nfreq] i^-|q| x transformed tensor, x-exponent <= 2
    cufftHandle r2c = 0, c2r = 0;      // nr components at a time
    bool r2c_ok = false, c2r_ok = false;
};

// Per-box buffers of a step.
struct FarBox {
    int tensor = 0;
    int64_t cell0 = 0;                 // first global cell of the box
    double inv_h2 = 0.0;
    double *W = nullptr;               // [nr][ncell] reduced weighted multipoles, then the reduced T
    cufftDoubleComplex *Wh = nullptr;  // [nr][nfreq]
    cufftDoubleComplex *Th = nullptr;  // [nr][nfreq]
};

struct FarState {
    int p = 0, np = 0, nr = 0, nd = 0;
    int *mabc = nullptr;               // [3][np] all multi-indices of order <= p
    double *coef = nullptr;            // [np] (-1)^|m| / m!
    // fold: reduced W_r = sum_e fval[e] * (coef M)[fcol[e]], e in [fptr[r], fptr[r+1])
    int *fptr = nullptr, *fcol = nullptr;
    double *fval = nullptr;
    // completion: T_k = sum_e gval[e] * T_red[gcol[e]] + gbg[k] * (4 pi M_tot / CPD^3), k < np
    int *gptr = nullptr, *gcol = nullptr;
    double *gval = nullptr, *gbg = nullptr;
    int *conv_add = nullptr;           // [nr][nr] position of k + m among the stored tensor components
    int *rdeg = nullptr;               // [nr] order |m| of each reduced component
    // gradient terms |j| <= p - 1: positions of j + e_x, j + e_y, j + e_z among
    // the multi-indices of order <= p, and 1 / j!
    int nterm = 0;
    int4 *tix = nullptr;
    float *tfac = nullptr;
    float4 *tc = nullptr;              // [max ncell][nterm] completed coefficients (scratch, box by box)
    int *scell = nullptr;              // [capacity] cell of each sorted particle (scratch)
    std::vector<FarTensor> tensors;
    std::vector<FarBox> boxes;
};

namespace {

// ------------------------------------------------------------ short-range tensor
// Lattice vectors of the real-space part: every integer s with
// |s| < r_cut, plus the near-field block [-R, R]^3, grouped by the grid cell
// s mod P that they add to (host bookkeeping; the arithmetic is in
// k_far_realspace). The near flag marks the vectors whose image the near
// field already has.
struct RealSpaceVectors {
    std::vector<int4> vec;        // (x, y, z, near)
    std::vector<int> first;       // CSR over cells: vec[first[t] .. first[t+1])
    std::vector<int64_t> cell;    // grid cell of each group
};

RealSpaceVectors real_space_vectors(int P, int R, double r_cut) {
    const int smax = (int)std::ceil(r_cut);
    struct V { int64_t cell; int x, y, z, near; };
    std::vector<V> all;
    for (int x = -smax; x <= smax; ++x)
        for (int y = -smax; y <= smax; ++y)
            for (int z = -smax; z <= smax; ++z) {
                const int near = std::abs(x) <= R && std::abs(y) <= R && std::abs(z) <= R;
                if (!near && std::sqrt((double)x * x + (double)y * y + (double)z * z) >= r_cut) continue;
                const int64_t g = ((int64_t)(((x % P) + P) % P) * P + ((y % P) + P) % P) * P + ((z % P) + P) % P;
                all.push_back({g, x, y, z, near});
            }
    std::stable_sort(all.begin(), all.end(), [](const V &u, const V &v) { return u.cell < v.cell; });
    RealSpaceVectors out;
    for (size_t i = 0; i < all.size(); ++i) {
        if (i == 0 || all[i].cell != all[i - 1].cell) {
            out.first.push_back((int)i);
            out.cell.push_back(all[i].cell);
        }
        out.vec.push_back(make_int4(all[i].x, all[i].y, all[i].z, all[i].near));
    }
    out.first.push_back((int)all.size());
    return out;
}

// Real-space part of the tensor, one block per touched grid cell, its
// lattice vectors in a fixed order. For a vector s (cell units, r = |s|):
//   radial factors h_n = (1/r d/dr)^n f, n <= Q, of f = erfc(alpha r)/r,
//     h_n = (-1)^n B_n, B_0 = erfc(alpha r)/r,
//     B_n = ((2n-1) B_{n-1} + (2 alpha^2)^n exp(-alpha^2 r^2)/(alpha sqrt(pi))) / r^2;
//   or, for the near image, of f = -erf(alpha r)/r (its series, which does
//   not cancel at r ~ 1/alpha and is finite at r = 0):
//     h_n = -(2 alpha/sqrt(pi)) (-2 alpha^2)^n sum_j (-alpha^2 r^2)^j / (j! (2n+2j+1));
//   Cartesian derivatives by the Hermite-type recursion
//     H^(n)_{a,b,c} = z H^(n+1)_{a,b,c-1} + (c-1) H^(n+1)_{a,b,c-2} (likewise y, x),
//     H^(n)_000 = h_n, d^(a,b,c) f = H^(0)_abc,
//   one degree at a time in shared memory. The kept components of the
//   cell's sum go to the zeroed grid (component-major).
__global__ void k_far_realspace(const int4 *__restrict__ vec, const int *__restrict__ first,
                                const int64_t *__restrict__ cell, int ncells_t, int Q, int nq,
                                const int *__restrict__ qa, const int *__restrict__ qb, const int *__restrict__ qc,
                                const int *__restrict__ qpos, const int *__restrict__ keep, int nk, double alpha,
                                int64_t ncell, double *__restrict__ grid) {
    extern __shared__ double fsm[];
    double *H = fsm;                               // [(Q+1)][nq]
    double *full = H + (size_t)(Q + 1) * nq;       // [nq]
    double *h = full + nq;                         // [Q+1]
    const int t = threadIdx.x, nt = blockDim.x;
    const int Q1 = Q + 1;
    for (int ct = blockIdx.x; ct < ncells_t; ct += gridDim.x) {
        for (int i = t; i < nq; i += nt) full[i] = 0.0;
        for (int v = first[ct]; v < first[ct + 1]; ++v) {
            const int4 s4 = vec[v];
            const double sx = s4.x, sy = s4.y, sz = s4.z;
            const double r = sqrt(sx * sx + sy * sy + sz * sz);
            __syncthreads();
            if (s4.w) {   // near image: the series of -erf(alpha r)/r, one n per thread
                const double x = alpha * alpha * r * r;
                for (int n = t; n <= Q; n += nt) {
                    double term = 1.0, sum = 0.0;
                    for (int j = 0; j < 400; ++j) {
                        const double u = term / (2.0 * (n + j) + 1.0);
                        sum += u;
                        if (j > x && fabs(u) < 1e-19 * fabs(sum)) break;
                        term *= -x / (j + 1);
                    }
                    h[n] = -2.0 * alpha / sqrt(M_PI) * pow(-2.0 * alpha * alpha, (double)n) * sum;
                }
            } else if (t == 0) {
                const double gauss = exp(-alpha * alpha * r * r) / (alpha * sqrt(M_PI));
                double B = erfc(alpha * r) / r, pw = 1.0;
                h[0] = B;
                for (int n = 1; n <= Q; ++n) {
                    pw *= 2.0 * alpha * alpha;
                    B = ((2 * n - 1) * B + pw * gauss) / (r * r);
                    h[n] = (n & 1) ? -B : B;
                }
            }
            __syncthreads();
            for (int deg = 0; deg <= Q; ++deg) {
                const int i0 = deg * (deg + 1) * (deg + 2) / 6, cnt = (deg + 1) * (deg + 2) / 2;
                const int levels = Q1 - deg;
                for (int w = t; w < cnt * levels; w += nt) {
                    const int i = i0 + w % cnt, n = w / cnt;
                    const int a = qa[i], b = qb[i], c = qc[i];
                    double val;
                    if (deg == 0) {
                        val = h[n];
                    } else if (c > 0) {
                        val = sz * H[(size_t)(n + 1) * nq + qpos[(a * Q1 + b) * Q1 + c - 1]];
                        if (c > 1) val += (c - 1) * H[(size_t)(n + 1) * nq + qpos[(a * Q1 + b) * Q1 + c - 2]];
                    } else if (b > 0) {
                        val = sy * H[(size_t)(n + 1) * nq + qpos[(a * Q1 + b - 1) * Q1 + c]];
                        if (b > 1) val += (b - 1) * H[(size_t)(n + 1) * nq + qpos[(a * Q1 + b - 2) * Q1 + c]];
                    } else {
                        val = sx * H[(size_t)(n + 1) * nq + qpos[((a - 1) * Q1 + b) * Q1 + c]];
                        if (a > 1) val += (a - 1) * H[(size_t)(n + 1) * nq + qpos[((a - 2) * Q1 + b) * Q1 + c]];
                    }
                    H[(size_t)n * nq + i] = val;
                }
                __syncthreads();
            }
            for (int i = t; i < nq; i += nt) full[i] += H[i];
        }
        __syncthreads();
        for (int k = t; k < nk; k += nt) grid[(int64_t)k * ncell + cell[ct]] = full[keep[k]];
        __syncthreads();
    }
}

// ------------------------------------------------------------ kernels
// Long-range part, added in Fourier space: for frequency w (cuFFT R2C layout
// [x][y][z <= P/2]) and every alias m = w + G P with 0 < |k| < k_cut,
// k = 2 pi m / P:  Dh_q(w) += (4 pi / k^2) exp(-k^2 / 4 alpha^2) (i k)^q.
__global__ void k_far_longrange(cufftDoubleComplex *__restrict__ Dh, int P, int64_t nfreq, int nq,
                                const int *__restrict__ qa, const int *__restrict__ qb,
                                const int *__restrict__ qc, double alpha, double k_cut) {
    const int Pz = P / 2 + 1;
    const double two_pi_P = 2.0 * M_PI / P;
    const int G = (int)ceil(k_cut / (2.0 * M_PI)) + 1;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nfreq;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int wz = (int)(f % Pz), wy = (int)((f / Pz) % P), wx = (int)(f / ((int64_t)Pz * P));
        for (int gx = -G; gx <= G; ++gx)
            for (int gy = -G; gy <= G; ++gy)
                for (int gz = -G; gz <= G; ++gz) {
                    const int mx = wx + gx * P, my = wy + gy * P, mz = wz + gz * P;
                    if (mx == 0 && my == 0 && mz == 0) continue;
                    const double kx = two_pi_P * mx, ky = two_pi_P * my, kz = two_pi_P * mz;
                    const double k2 = kx * kx + ky * ky + kz * kz;
                    if (k2 >= k_cut * k_cut) continue;
                    const double w = 4.0 * M_PI / k2 * exp(-k2 / (4.0 * alpha * alpha));
                    double px[33], py[33], pz[33];
                    px[0] = py[0] = pz[0] = 1.0;
                    for (int j = 1; j < 33; ++j) {
                        px[j] = px[j - 1] * kx; py[j] = py[j - 1] * ky; pz[j] = pz[j - 1] * kz;
                    }
                    for (int q = 0; q < nq; ++q) {
                        const int a = qa[q], b = qb[q], c = qc[q];
                        const double v = w * px[a] * py[b] * pz[c];
                        cufftDoubleComplex &d = Dh[(int64_t)q * nfreq + f];
                        switch ((a + b + c) & 3) {   // i^|q|
                            case 0: d.x += v; break;
                            case 1: d.y += v; break;
                            case 2: d.x -= v; break;
                            default: d.y -= v; break;
                        }
                    }
                }
    }
}

// The transformed tensor is i^|q| times a real function (parity of the
// order); E_q = i^-|q| Dh_q keeps that real function. What is dropped, the
// other part, is rounding: about 1e-16 of the kept one.
__global__ void k_far_realify(const cufftDoubleComplex *__restrict__ Dh, double *__restrict__ E, int64_t nfreq,
                              int64_t total, const int *__restrict__ qa, const int *__restrict__ qb,
                              const int *__restrict__ qc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(i / nfreq);
        const cufftDoubleComplex d = Dh[i];
        switch ((qa[q] + qb[q] + qc[q]) & 3) {   // i^-|q| d, real part
            case 0: E[i] = d.x; break;
            case 1: E[i] = d.y; break;
            case 2: E[i] = -d.x; break;
            default: E[i] = -d.y; break;
        }
    }
}

// Multipoles: one block per cell, 128 threads. A tile of up to 128 sorted
// records is staged with each particle's powers x^e, y^e, z^e (e <= p,
// particle-major so that a warp reading one particle's powers hits distinct
// banks or one broadcast); thread t then owns components t and t + 128 and
// sums mass * x^a y^b z^c over the tile in FP32, folded into an FP64 total
// per tile. The cell's W_m = coef_m M_m are then folded down to the reduced
// set by a fixed sparse map (one reduced component per thread) and written
// component-major.
constexpr int kFarThreads = 128;
constexpr int kFarMaxP = 8;

__global__ void __launch_bounds__(kFarThreads) k_far_multipoles(
    const float4 *__restrict__ sorted, const int *__restrict__ cell_start, int64_t ncell, int p, int np,
    const int *__restrict__ mabc, const double *__restrict__ coef, const int *__restrict__ fptr,
    const int *__restrict__ fcol, const double *__restrict__ fval, int nr, double *__restrict__ W) {
    __shared__ float pw[3][kFarThreads][kFarMaxP + 1];
    __shared__ float ms[kFarThreads];
    __shared__ double Ws[2 * kFarThreads];
    const int t = threadIdx.x;
    const int i0 = t, i1 = t + kFarThreads;
    int a0 = 0, b0 = 0, c0 = 0, a1 = 0, b1 = 0, c1 = 0;
    if (i0 < np) { a0 = mabc[i0]; b0 = mabc[np + i0]; c0 = mabc[2 * np + i0]; }
    if (i1 < np) { a1 = mabc[i1]; b1 = mabc[np + i1]; c1 = mabc[2 * np + i1]; }
    for (int64_t cell = blockIdx.x; cell < ncell; cell += gridDim.x) {
        const int s = cell_start[cell], e = cell_start[cell + 1];
        double acc0 = 0.0, acc1 = 0.0;
        for (int base = s; base < e; base += kFarThreads) {
            const int cnt = min(kFarThreads, e - base);
            __syncthreads();
            if (t < cnt) {
                const float4 r = sorted[base + t];
                pw[0][t][0] = pw[1][t][0] = pw[2][t][0] = 1.f;
                for (int j = 1; j <= p; ++j) {
                    pw[0][t][j] = pw[0][t][j - 1] * r.x;
                    pw[1][t][j] = pw[1][t][j - 1] * r.y;
                    pw[2][t][j] = pw[2][t][j - 1] * r.z;
                }
                ms[t] = r.w;
            }
            __syncthreads();
            float f0 = 0.f, f1 = 0.f;
            for (int j = 0; j < cnt; ++j) {
                const float m = ms[j];
                f0 = fmaf(m * pw[0][j][a0] * pw[1][j][b0], pw[2][j][c0], f0);
                f1 = fmaf(m * pw[0][j][a1] * pw[1][j][b1], pw[2][j][c1], f1);
            }
            acc0 += (double)f0;
            acc1 += (double)f1;
        }
        __syncthreads();
        if (i0 < np) Ws[i0] = coef[i0] * acc0;
        if (i1 < np) Ws[i1] = coef[i1] * acc1;
        __syncthreads();
        for (int r = t; r < nr; r += kFarThreads) {
            double v = 0.0;
            for (int q = fptr[r]; q < fptr[r + 1]; ++q) v = fma(fval[q], Ws[fcol[q]], v);
            W[(int64_t)r * ncell + cell] = v;
        }
    }
}

// i^n v, exact (a swap and sign changes).
__device__ __forceinline__ double2 times_i_pow(double2 v, int n) {
    switch (n & 3) {
        case 0: return v;
        case 1: return make_double2(-v.y, v.x);
        case 2: return make_double2(-v.x, -v.y);
        default: return make_double2(v.y, -v.x);
    }
}

// Per-frequency products T_k(w) = i^|k| sum_m E_{k+m}(w) (i^|m| W_m(w)) over
// the reduced k and m (E real: two FP64 FMAs per product): a block takes 32
// consecutive frequencies (one per lane); i^|m| W_m(w) is staged in shared
// memory; warp y of the block computes k = y, y + blockDim.y, ...
__global__ void k_far_convolve(const double *__restrict__ E, const cufftDoubleComplex *__restrict__ Wh,
                               cufftDoubleComplex *__restrict__ Th, int64_t nfreq, int nr,
                               const int *__restrict__ add, const int *__restrict__ rdeg) {
    extern __shared__ double2 cm[];   // [nr][32]
    const int lane = threadIdx.x, wy = threadIdx.y, ny = blockDim.y;
    for (int64_t f0 = (int64_t)blockIdx.x * 32; f0 < nfreq; f0 += (int64_t)gridDim.x * 32) {
        const int64_t f = f0 + lane;
        const bool ok = f < nfreq;
        __syncthreads();
        for (int m = wy; m < nr; m += ny) {
            double2 v = make_double2(0.0, 0.0);
            if (ok) {
                const cufftDoubleComplex x = Wh[(int64_t)m * nfreq + f];
                v = times_i_pow(make_double2(x.x, x.y), __ldg(&rdeg[m]));
            }
            cm[m * 32 + lane] = v;
        }
        __syncthreads();
        for (int k = wy; k < nr; k += ny) {
            double re = 0.0, im = 0.0;
            const int *ak = add + (int64_t)k * nr;
            if (ok) {
                for (int m = 0; m < nr; ++m) {
                    const double d = E[(int64_t)__ldg(&ak[m]) * nfreq + f];
                    const double2 x = cm[m * 32 + lane];
                    re = fma(d, x.x, re);
                    im = fma(d, x.y, im);
                }
                Th[(int64_t)k * nfreq + f] = times_i_pow(make_double2(re, im), __ldg(&rdeg[k]));
            }
        }
    }
}

// Position of (a, b, c) among the multi-indices of order <= p (enumeration:
// degree t, then c ascending, then b ascending).
__host__ __device__ constexpr int mi_pos(int a, int b, int c) {
    return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + c * (a + b + c + 1) - c * (c - 1) / 2 + b;
}

// Completion of the Taylor coefficients, 32 cells per block. The cells'
// reduced T (inverse transform / CPD^3, FP64) are completed to all |k| <= p
// by the harmonic relation: a fixed sparse map, which also carries the
// background term 4 pi M_tot / CPD^3 (M_tot is the zero-frequency value of
// W_0). They are scaled to box units and written per cell as the terms of
// the gradient, the float4 (T_{j+e_x}, T_{j+e_y}, T_{j+e_z}) / j! for
// |j| <= p - 1 (enumeration of mi_pos). The block also writes, for every
// particle of its cells, the cell's index: the Taylor kernel takes
// particles, not cells.
constexpr int kCompCells = 32;
constexpr int kFarMaxNp = 165;   // multi-indices of order <= 8 (odd: no bank conflicts)
constexpr int kFarMaxNr = 81;    // reduced components at p = 8

__global__ void __launch_bounds__(kFarThreads) k_far_complete(
    const double *__restrict__ Tr, const int *__restrict__ cell_start, int64_t ncell, int np, int nr,
    const int *__restrict__ gptr, const int *__restrict__ gcol, const double *__restrict__ gval,
    const double *__restrict__ gbg, const cufftDoubleComplex *__restrict__ w0_dc, double inv_n, double inv_h2,
    int nterm, const int4 *__restrict__ tix, const float *__restrict__ tfac, float4 *__restrict__ Tc,
    int *__restrict__ scell) {
    __shared__ double Tred[kFarMaxNr][kCompCells];
    __shared__ float Tk[kCompCells][kFarMaxNp];
    __shared__ int cs[kCompCells + 1];
    const int t = threadIdx.x;
    const double bg = 4.0 * M_PI * w0_dc->x * inv_n;   // 4 pi M_tot / CPD^3
    for (int64_t c0 = (int64_t)blockIdx.x * kCompCells; c0 < ncell; c0 += (int64_t)gridDim.x * kCompCells) {
        const int nc = (int)min((int64_t)kCompCells, ncell - c0);
        __syncthreads();
        for (int i = t; i < nr * kCompCells; i += kFarThreads) {
            const int r = i / kCompCells, cl = i % kCompCells;
            Tred[r][cl] = cl < nc ? Tr[(int64_t)r * ncell + c0 + cl] * inv_n : 0.0;
        }
        for (int i = t; i <= nc; i += kFarThreads) cs[i] = cell_start[c0 + i];
        __syncthreads();
        for (int i = t; i < np * kCompCells; i += kFarThreads) {
            const int k = i / kCompCells, cl = i % kCompCells;
            double v = gbg[k] * bg;
            for (int q = gptr[k]; q < gptr[k + 1]; ++q) v = fma(gval[q], Tred[gcol[q]][cl], v);
            Tk[cl][k] = (float)(v * inv_h2);
        }
        __syncthreads();
        float4 *out = Tc + c0 * nterm;
        for (int i = t; i < nc * nterm; i += kFarThreads) {
            const int cl = i / nterm, j = i - cl * nterm;
            const int4 x = tix[j];
            const float w = tfac[j];
            out[i] = make_float4(Tk[cl][x.x] * w, Tk[cl][x.y] * w, Tk[cl][x.z] * w, 0.f);
        }
        for (int cl = 0; cl < nc; ++cl)
            for (int j = cs[cl] + t; j < cs[cl + 1]; j += kFarThreads) scell[j] = (int)(c0 + cl);
    }
}

// Taylor gradient, one thread per particle of the box (sorted order, so a
// warp takes 32 consecutive particles of one to a few cells, whatever the
// cells' occupancy): with y the cell-relative position,
//   a(y) = sum_{|j| <= p-1} y^j (T_{j+e_x}, T_{j+e_y}, T_{j+e_z}) / j!,
// one 16-byte load per term from the cell's row of the completed
// coefficients. The order is a template parameter, so the loops unroll with
// the term positions as constants and the powers of y in registers.
template <int P>
__global__ void __launch_bounds__(kFarThreads) k_far_taylor(
    const float4 *__restrict__ sorted, const int *__restrict__ perm, const int *__restrict__ scell,
    const float4 *__restrict__ Tc, int64_t p0, int64_t p1, float *__restrict__ acc, int accumulate) {
    constexpr int NT = P * (P + 1) * (P + 2) / 6;   // terms |j| <= P - 1
    for (int64_t j = p0 + (int64_t)blockIdx.x * kFarThreads + threadIdx.x; j < p1;
         j += (int64_t)gridDim.x * kFarThreads) {
        const float4 r = sorted[j];
        const float4 *tc = Tc + (int64_t)scell[j] * NT;
        float px[P], py[P], pz[P];
        px[0] = py[0] = pz[0] = 1.f;
#pragma unroll
        for (int q = 1; q < P; ++q) {
            px[q] = px[q - 1] * r.x;
            py[q] = py[q - 1] * r.y;
            pz[q] = pz[q - 1] * r.z;
        }
        float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
        for (int a = 0; a < P; ++a)
#pragma unroll
            for (int b = 0; a + b < P; ++b) {
                const float xy = px[a] * py[b];
#pragma unroll
                for (int c = 0; a + b + c < P; ++c) {
                    const float y = xy * pz[c];
                    const float4 t = __ldg(&tc[mi_pos(a, b, c)]);
                    ax = fmaf(y, t.x, ax);
                    ay = fmaf(y, t.y, ay);
                    az = fmaf(y, t.z, az);
                }
            }
        float *o = acc + 3 * (int64_t)perm[j];
        if (accumulate) {
            o[0] += ax; o[1] += ay; o[2] += az;
        } else {
            o[0] = ax; o[1] = ay; o[2] = az;
        }
    }
}

template <typename T>
cudaError_t dmalloc(T **p, size_t count) {
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (count ? count : 1));
}

template <typename T>
cudaError_t upload(T **d, const std::vector<T> &h) {
    cudaError_t e = dmalloc(d, h.size());
    if (e) return e;
    return cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

int grid_blocks(int64_t n, int threads, int sm_count, int per_sm) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count * per_sm;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace

void far_release(Ctx *c) {
    FarState *f = c->far;
    if (!f) return;
    void *bufs[] = {f->mabc, f->coef, f->fptr, f->fcol, f->fval, f->gptr, f->gcol, f->gval, f->gbg,
                    f->conv_add, f->rdeg, f->tix, f->tfac, f->tc, f->scell};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (FarTensor &t : f->tensors) {
        if (t.E) cudaFree(t.E);
        if (t.r2c_ok) cufftDestroy(t.r2c);
        if (t.c2r_ok) cufftDestroy(t.c2r);
    }
    for (FarBox &b : f->boxes) {
        void *bb[] = {b.W, b.Wh, b.Th};
        for (void *x : bb)
            if (x) cudaFree(x);
    }
    delete f;
    c->far = nullptr;
}

// Builds the far-field state: index tables (one set for the order), one
// derivatives tensor in Fourier space per distinct CPD, per-box buffers and
// FFT plans. Synchronous. Returns NF_OK, or NF_ENOMEM / NF_ECUDA with `err` set.
int far_setup(Ctx *c, int order, cudaStream_t s, std::string &err) {
    far_release(c);
    FarState *f = new FarState();
    c->far = f;
    f->p = order;
    MultiIndex mp, mq;
    mp.build(order);
    mq.build(2 * order);
    f->np = mp.size();
    auto cuda_err = [&](cudaError_t e, const char *what) {
        err = std::string("nf_far_init: ") + what + ": " + cudaGetErrorString(e);
        far_release(c);
        return e == cudaErrorMemoryAllocation ? NF_ENOMEM : NF_ECUDA;
    };
    auto fft_err = [&](cufftResult r, const char *what) {
        err = std::string("nf_far_init: ") + what + ": cuFFT error " + std::to_string((int)r);
        far_release(c);
        return r == CUFFT_ALLOC_FAILED ? NF_ENOMEM : NF_ECUDA;
    };
    cudaError_t e;
    // ---- index tables
    std::vector<int> red, red_of(f->np, -1);
    for (int i = 0; i < f->np; ++i)
        if (mp.a[i] <= 1) { red_of[i] = (int)red.size(); red.push_back(i); }
    f->nr = (int)red.size();
    std::vector<int> stored, stored_of(mq.size(), -1);   // tensor components kept: x-exponent <= 2
    for (int i = 0; i < mq.size(); ++i)
        if (mq.a[i] <= 2) { stored_of[i] = (int)stored.size(); stored.push_back(i); }
    f->nd = (int)stored.size();
    {
        std::vector<int> mabc(3 * (size_t)f->np), add((size_t)f->nr * f->nr), dabc(3 * (size_t)f->nd);
        std::vector<double> coef(f->np);
        for (int i = 0; i < f->np; ++i) {
            mabc[i] = mp.a[i]; mabc[f->np + i] = mp.b[i]; mabc[2 * f->np + i] = mp.c[i];
            double fac = 1.0;
            for (int x = 2; x <= mp.a[i]; ++x) fac *= x;
            for (int x = 2; x <= mp.b[i]; ++x) fac *= x;
            for (int x = 2; x <= mp.c[i]; ++x) fac *= x;
            coef[i] = (((mp.a[i] + mp.b[i] + mp.c[i]) & 1) ? -1.0 : 1.0) / fac;
        }
        // fold of W (x-exponent from p down to 2: W[m-2x+2y] -= W[m], W[m-2x+2z] -= W[m]),
        // carried out on sparse linear combinations of the original components
        std::vector<std::vector<std::pair<int, double>>> comb(f->np);
        for (int i = 0; i < f->np; ++i) comb[i] = {{i, 1.0}};
        auto axpy = [](std::vector<std::pair<int, double>> &dst, const std::vector<std::pair<int, double>> &src,
                       double a) {
            for (const auto &e : src) {
                bool found = false;
                for (auto &d : dst)
                    if (d.first == e.first) { d.second += a * e.second; found = true; break; }
                if (!found) dst.push_back({e.first, a * e.second});
            }
        };
        for (int a = order; a >= 2; --a)
            for (int i = 0; i < f->np; ++i)
                if (mp.a[i] == a) {
                    axpy(comb[mp.at(a - 2, mp.b[i] + 2, mp.c[i])], comb[i], -1.0);
                    axpy(comb[mp.at(a - 2, mp.b[i], mp.c[i] + 2)], comb[i], -1.0);
                    comb[i].clear();
                }
        std::vector<int> fptr(1, 0), fcol;
        std::vector<double> fval;
        for (int r = 0; r < f->nr; ++r) {
            auto row = comb[red[r]];
            std::sort(row.begin(), row.end());
            for (const auto &e : row)
                if (e.second != 0.0) { fcol.push_back(e.first); fval.push_back(e.second); }
            fptr.push_back((int)fcol.size());
        }
        // completion of T (x-exponent from 2 up: T[k] = -T[k-2x+2y] - T[k-2x+2z], plus
        // the background on (2,0,0)), as combinations of the reduced T and the background
        std::vector<std::vector<std::pair<int, double>>> tcomb(f->np);
        std::vector<double> gbg(f->np, 0.0);
        for (int r = 0; r < f->nr; ++r) tcomb[red[r]] = {{r, 1.0}};
        for (int a = 2; a <= order; ++a)
            for (int i = 0; i < f->np; ++i)
                if (mp.a[i] == a) {
                    const int s1 = mp.at(a - 2, mp.b[i] + 2, mp.c[i]), s2 = mp.at(a - 2, mp.b[i], mp.c[i] + 2);
                    tcomb[i].clear();
                    axpy(tcomb[i], tcomb[s1], -1.0);
                    axpy(tcomb[i], tcomb[s2], -1.0);
                    gbg[i] = -gbg[s1] - gbg[s2] + (a == 2 && mp.b[i] == 0 && mp.c[i] == 0 ? 1.0 : 0.0);
                }
        std::vector<int> gptr(1, 0), gcol;
        std::vector<double> gval;
        for (int k = 0; k < f->np; ++k) {
            auto row = tcomb[k];
            std::sort(row.begin(), row.end());
            for (const auto &e : row)
                if (e.second != 0.0) { gcol.push_back(e.first); gval.push_back(e.second); }
            gptr.push_back((int)gcol.size());
        }
        std::vector<int> rdeg(f->nr);
        for (int r = 0; r < f->nr; ++r) rdeg[r] = mp.a[red[r]] + mp.b[red[r]] + mp.c[red[r]];
        std::vector<int4> tix;
        std::vector<float> tfac;
        for (int i = 0; i < f->np; ++i) {
            const int a = mp.a[i], b = mp.b[i], cc = mp.c[i];
            if (a + b + cc > order - 1) break;   // degree-major: the terms are a prefix
            tix.push_back(make_int4(mp.at(a + 1, b, cc), mp.at(a, b + 1, cc), mp.at(a, b, cc + 1), 0));
            double fac = 1.0;
            for (int x = 2; x <= a; ++x) fac *= x;
            for (int x = 2; x <= b; ++x) fac *= x;
            for (int x = 2; x <= cc; ++x) fac *= x;
            tfac.push_back((float)(1.0 / fac));
        }
        f->nterm = (int)tix.size();
        for (int k = 0; k < f->nr; ++k)
            for (int m = 0; m < f->nr; ++m) {
                const int ik = red[k], im = red[m];
                add[(size_t)k * f->nr + m] =
                    stored_of[mq.at(mp.a[ik] + mp.a[im], mp.b[ik] + mp.b[im], mp.c[ik] + mp.c[im])];
            }
        for (int i = 0; i < f->nd; ++i) {
            dabc[i] = mq.a[stored[i]]; dabc[f->nd + i] = mq.b[stored[i]]; dabc[2 * f->nd + i] = mq.c[stored[i]];
        }
        if ((e = upload(&f->mabc, mabc)) || (e = upload(&f->coef, coef)) || (e = upload(&f->fptr, fptr)) ||
            (e = upload(&f->fcol, fcol)) || (e = upload(&f->fval, fval)) || (e = upload(&f->gptr, gptr)) ||
            (e = upload(&f->gcol, gcol)) || (e = upload(&f->gval, gval)) || (e = upload(&f->gbg, gbg)) ||
            (e = upload(&f->conv_add, add)) || (e = upload(&f->rdeg, rdeg)) || (e = upload(&f->tix, tix)) ||
            (e = upload(&f->tfac, tfac)))
            return cuda_err(e, "tables");
    }
    std::vector<int> dabc(3 * (size_t)f->nd);
    for (int i = 0; i < f->nd; ++i) {
        dabc[i] = mq.a[stored[i]]; dabc[f->nd + i] = mq.b[stored[i]]; dabc[2 * f->nd + i] = mq.c[stored[i]];
    }
    // ---- one tensor per distinct CPD
    for (int b = 0; b < c->n_boxes; ++b) {
        const BoxDev &B = c->boxes_h[b];
        const int P = B.cpd;
        int ti = -1;
        for (size_t t = 0; t < f->tensors.size(); ++t)
            if (f->tensors[t].P == P) ti = (int)t;
        if (ti < 0) {
            ti = (int)f->tensors.size();
            f->tensors.emplace_back();
            FarTensor &T = f->tensors.back();
            T.P = P;
            T.ncell = (int64_t)P * P * P;
            T.nfreq = (int64_t)P * P * (P / 2 + 1);
            // splitting: the real-space part reaches r < (6.5 + q/4)/alpha cells and the
            // Fourier part |k| < (13 + q/2) alpha; alpha = max(0.5, 3.5/P) keeps both small
            const double alpha = std::max(0.5, 3.5 / P);
            const double r_cut = (6.5 + 0.25 * mq.n) / alpha;
            const double k_cut = (13.0 + 0.5 * mq.n) * alpha;
            int *da = nullptr;
            if ((e = upload(&da, dabc))) return cuda_err(e, "tables");
            // real-space part: lattice vectors grouped by grid cell (host), their
            // derivatives summed on the GPU into a zeroed FP64 grid
            const RealSpaceVectors rs = real_space_vectors(P, c->R, r_cut);
            double *grid = nullptr;
            int4 *dvec = nullptr;
            int *dfirst = nullptr, *dq = nullptr, *dqpos = nullptr, *dkeep = nullptr;
            int64_t *dcell = nullptr;
            cufftDoubleComplex *Dh = nullptr;   // the transformed tensor while it is built
            if ((e = dmalloc(&Dh, (size_t)f->nd * T.nfreq))) { cudaFree(da); return cuda_err(e, "tensor"); }
            auto free_rs = [&]() {
                cudaFree(grid); cudaFree(dvec); cudaFree(dfirst); cudaFree(dq); cudaFree(dqpos);
                cudaFree(dkeep); cudaFree(dcell);
                grid = nullptr; dvec = nullptr; dfirst = dq = dqpos = dkeep = nullptr; dcell = nullptr;
            };
            auto free_build = [&]() { free_rs(); cudaFree(Dh); cudaFree(da); };
            std::vector<int> qall(3 * (size_t)mq.size());
            for (int i = 0; i < mq.size(); ++i) {
                qall[i] = mq.a[i]; qall[mq.size() + i] = mq.b[i]; qall[2 * (size_t)mq.size() + i] = mq.c[i];
            }
            if ((e = dmalloc(&grid, (size_t)f->nd * T.ncell)) || (e = upload(&dvec, rs.vec)) ||
                (e = upload(&dfirst, rs.first)) || (e = upload(&dcell, rs.cell)) || (e = upload(&dq, qall)) ||
                (e = upload(&dqpos, mq.pos)) || (e = upload(&dkeep, stored))) {
                free_build();
                return cuda_err(e, "tensor");
            }
            e = cudaMemsetAsync(grid, 0, sizeof(double) * (size_t)f->nd * T.ncell, s);
            if (!e) {
                const size_t smem = sizeof(double) * ((size_t)(mq.n + 1) * mq.size() + mq.size() + mq.n + 1);
                e = cudaFuncSetAttribute(k_far_realspace, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (!e) {
                    const int ncells_t = (int)rs.cell.size();
                    k_far_realspace<<<std::min(ncells_t, c->sm_count * 2), 256, smem, s>>>(
                        dvec, dfirst, dcell, ncells_t, mq.n, mq.size(), dq, dq + mq.size(), dq + 2 * mq.size(), dqpos,
                        dkeep, f->nd, alpha, T.ncell, grid);
                    e = cudaGetLastError();
                }
            }
            // the tensor's components are transformed 64 at a time, the rest by a
            // second plan: chunk starts stay at even component offsets, which
            // keeps them 16-byte aligned as cuFFT requires of its data
            cufftHandle plan = 0, plan_rest = 0;
            int dims[3] = {P, P, P};
            const int chunk = 64, rest = f->nd % chunk;
            const char *stage = "tensor transform: plan";
            cufftResult fr = CUFFT_SUCCESS;
            if (!e && f->nd >= chunk)
                fr = cufftPlanMany(&plan, 3, dims, nullptr, 1, (int)T.ncell, nullptr, 1, (int)T.nfreq, CUFFT_D2Z, chunk);
            if (!e && fr == CUFFT_SUCCESS && rest)
                fr = cufftPlanMany(&plan_rest, 3, dims, nullptr, 1, (int)T.ncell, nullptr, 1, (int)T.nfreq, CUFFT_D2Z,
                                   rest);
            if (!e && fr == CUFFT_SUCCESS) {
                stage = "tensor transform: stream";
                if (plan) fr = cufftSetStream(plan, s);
                if (fr == CUFFT_SUCCESS && plan_rest) fr = cufftSetStream(plan_rest, s);
            }
            for (int q0 = 0; !e && fr == CUFFT_SUCCESS && q0 < f->nd; q0 += chunk) {
                stage = "tensor transform: exec";
                fr = cufftExecD2Z(q0 + chunk <= f->nd ? plan : plan_rest, grid + (size_t)q0 * T.ncell,
                                  Dh + (size_t)q0 * T.nfreq);
            }
            if (!e && fr == CUFFT_SUCCESS) {
                k_far_longrange<<<grid_blocks(T.nfreq, 128, c->sm_count, 8), 128, 0, s>>>(
                    Dh, P, T.nfreq, f->nd, da, da + f->nd, da + 2 * f->nd, alpha, k_cut);
                e = cudaGetLastError();
            }
            if (!e) e = cudaStreamSynchronize(s);
            if (plan) cufftDestroy(plan);
            if (plan_rest) cufftDestroy(plan_rest);
            free_rs();   // the real-space grid goes before the real tensor is allocated
            // keep the real function E_q = i^-|q| Dh_q
            if (!e && fr == CUFFT_SUCCESS) e = dmalloc(&T.E, (size_t)f->nd * T.nfreq);
            if (!e && fr == CUFFT_SUCCESS) {
                const int64_t total = (int64_t)f->nd * T.nfreq;
                k_far_realify<<<grid_blocks(total, 256, c->sm_count, 8), 256, 0, s>>>(
                    Dh, T.E, T.nfreq, total, da, da + f->nd, da + 2 * f->nd);
                e = cudaGetLastError();
                if (!e) e = cudaStreamSynchronize(s);
            }
            free_build();
            if (fr != CUFFT_SUCCESS) return fft_err(fr, stage);
            if (e) return cuda_err(e, "tensor");
            // per-step plans of this size (reduced components)
            fr = cufftPlanMany(&T.r2c, 3, dims, nullptr, 1, (int)T.ncell, nullptr, 1, (int)T.nfreq, CUFFT_D2Z, f->nr);
            if (fr != CUFFT_SUCCESS) return fft_err(fr, "plan");
            T.r2c_ok = true;
            fr = cufftPlanMany(&T.c2r, 3, dims, nullptr, 1, (int)T.nfreq, nullptr, 1, (int)T.ncell, CUFFT_Z2D, f->nr);
            if (fr != CUFFT_SUCCESS) return fft_err(fr, "plan");
            T.c2r_ok = true;
        }
        f->boxes.emplace_back();
        FarBox &X = f->boxes.back();
        X.tensor = ti;
        X.cell0 = B.cell_off;
        X.inv_h2 = B.inv_h2_d;
        const FarTensor &T = f->tensors[ti];
        if ((e = dmalloc(&X.W, (size_t)f->nr * T.ncell)) || (e = dmalloc(&X.Wh, (size_t)f->nr * T.nfreq)) ||
            (e = dmalloc(&X.Th, (size_t)f->nr * T.nfreq)))
            return cuda_err(e, "buffers");
    }
    int64_t max_cells = 0;
    for (const FarTensor &T : f->tensors) max_cells = std::max(max_cells, T.ncell);
    if ((e = dmalloc(&f->tc, (size_t)max_cells * f->nterm)) || (e = dmalloc(&f->scell, (size_t)c->capacity)))
        return cuda_err(e, "buffers");
    return NF_OK;
}

// Far-field accelerations of the binned particles, input order, written to
// (or, with accumulate, added into) acc. Enqueued on s, phase by phase over
// the boxes.
cudaError_t far_compute(Ctx *c, float *acc, int accumulate, cudaStream_t s, std::string &fft_fail) {
    FarState *f = c->far;
    cudaError_t e = cudaEventRecord(c->ev_far[0], s);
    if (e) return e;
    for (const FarBox &X : f->boxes) {
        const FarTensor &T = f->tensors[X.tensor];
        k_far_multipoles<<<grid_blocks(T.ncell * kFarThreads, kFarThreads, c->sm_count, 16), kFarThreads, 0, s>>>(
            c->sorted, c->cell_start + X.cell0, T.ncell, f->p, f->np, f->mabc, f->coef, f->fptr, f->fcol, f->fval,
            f->nr, X.W);
        c->launches += 1;
        if ((e = cudaGetLastError())) return e;
        cufftResult fr = cufftSetStream(T.r2c, s);
        if (fr == CUFFT_SUCCESS) fr = cufftExecD2Z(T.r2c, X.W, X.Wh);
        if (fr != CUFFT_SUCCESS) {
            fft_fail = "forward transform of the multipoles: cuFFT error " + std::to_string((int)fr);
            return cudaErrorUnknown;
        }
    }
    // W_0 is reduced component 0: its zero-frequency value is the box's total
    // mass, read by the Taylor kernel for the background term (the inverse
    // transforms overwrite Th only)
    const int ny = 8;
    const size_t smem = sizeof(double2) * 32 * (size_t)f->nr;
    e = cudaFuncSetAttribute(k_far_convolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    if ((e = cudaEventRecord(c->ev_far[2], s))) return e;
    for (const FarBox &X : f->boxes) {
        const FarTensor &T = f->tensors[X.tensor];
        k_far_convolve<<<grid_blocks(T.nfreq, 32, c->sm_count, 4), dim3(32, ny), smem, s>>>(
            T.E, X.Wh, X.Th, T.nfreq, f->nr, f->conv_add, f->rdeg);
        c->launches += 1;
        if ((e = cudaGetLastError())) return e;
    }
    if ((e = cudaEventRecord(c->ev_far[3], s))) return e;
    void (*taylor)(const float4 *, const int *, const int *, const float4 *, int64_t, int64_t, float *, int) =
        nullptr;
    switch (f->p) {
        case 1: taylor = k_far_taylor<1>; break;
        case 2: taylor = k_far_taylor<2>; break;
        case 3: taylor = k_far_taylor<3>; break;
        case 4: taylor = k_far_taylor<4>; break;
        case 5: taylor = k_far_taylor<5>; break;
        case 6: taylor = k_far_taylor<6>; break;
        case 7: taylor = k_far_taylor<7>; break;
        default: taylor = k_far_taylor<8>; break;
    }
    for (size_t b = 0; b < f->boxes.size(); ++b) {
        const FarBox &X = f->boxes[b];
        const FarTensor &T = f->tensors[X.tensor];
        cufftResult fr = cufftSetStream(T.c2r, s);
        if (fr == CUFFT_SUCCESS) fr = cufftExecZ2D(T.c2r, X.Th, X.W);
        if (fr != CUFFT_SUCCESS) {
            fft_fail = "inverse transform of the Taylor coefficients: cuFFT error " + std::to_string((int)fr);
            return cudaErrorUnknown;
        }
        // the box's particles are the sorted range [poff[b], poff[b+1]) (its cells are contiguous)
        const int64_t p0 = c->poff_h[b], p1 = c->poff_h[b + 1];
        k_far_complete<<<grid_blocks(T.ncell, kCompCells, c->sm_count, 8), kFarThreads, 0, s>>>(
            X.W, c->cell_start + X.cell0, T.ncell, f->np, f->nr, f->gptr, f->gcol, f->gval, f->gbg, X.Wh,
            1.0 / (double)T.ncell, X.inv_h2, f->nterm, f->tix, f->tfac, f->tc, f->scell);
        c->launches += 1;
        if ((e = cudaGetLastError())) return e;
        if (p1 > p0) {
            taylor<<<grid_blocks(p1 - p0, kFarThreads, c->sm_count, 16), kFarThreads, 0, s>>>(
                c->sorted, c->perm, f->scell, f->tc, p0, p1, acc, accumulate);
            c->launches += 1;
            if ((e = cudaGetLastError())) return e;
        }
    }
    return cudaEventRecord(c->ev_far[1], s);
}

}  // namespace nf

/*
 * oracle.c -- plain FP64 CPU oracle for the near-field direct sum.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or
 * includes this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it. It shares no code with the CUDA path.
 *
 * What it computes (Maksimova et al. 2021, "AbacusSummit", Sec. 3.1):
 *   - the periodic box of side L is cut into CPD^3 cubic cells (CPD cells per
 *     dimension; a slab is one CPD^2 plane of cells);
 *   - the force on a particle is split into a near field, sourced by the
 *     particles of the cells within the near-field radius R of its own cell,
 *     and a far field (not computed here). Each pairwise interaction,
 *     including each periodic image, belongs to exactly one of the two, so
 *     the near field takes, for each neighbouring cell offset d in [-R,R]^3,
 *     the one periodic image of cell (c + d) mod CPD that sits at offset d;
 *   - the near field is a direct O(N^2) sum over those cells.
 * The force law is Plummer softening, the gradient of the potential
 * -G m / sqrt(r^2 + eps^2) that Sec. 5.2 names as the common alternative to
 * the production spline law:  a_i = sum_j G m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2).
 * G is folded into the masses.
 *
 * Every routine here is the plain definition, evaluated in double precision
 * in a fixed order, with no blocking or reordering. Compile with
 * -ffp-contract=off so that the binning arithmetic is the same IEEE sequence
 * on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ERANGE (-2)
#define ORC_ENOMEM (-3)

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Cell coordinate of one position component (Sec. 3.1: CPD cells per
 * dimension). u = (x * CPD) / L in double; the cell is floor(u), and a value
 * that rounds up to CPD belongs to the last cell. */
static double cell_unit(double x, int cpd, double L) { return (x * (double)cpd) / L; }

static int cell_index(double u, int cpd)
{
    int c = (int)floor(u);
    if (c >= cpd) c = cpd - 1;
    return c;
}

/*
 * orc_bin: bin float32 positions into cells (Sec. 3.1).
 *   pos        [n*3] float32, each component in [0, L)
 *   cid        [n]   out: linear cell id (cx*CPD + cy)*CPD + cz (x slowest,
 *                    so that an x-slab is a contiguous run of cells)
 *   cell_start [CPD^3+1] out: first sorted slot of each cell
 *   perm       [n]   out: perm[k] = input index of the k-th sorted particle;
 *                    within a cell particles keep their input order
 *   rel        [n*3] out (may be NULL): cell-relative coordinates in cell
 *                    units of the k-th sorted particle,
 *                    float32(u - (c + 0.5)) with u = (x*CPD)/L
 * Returns ORC_ERANGE if a component is not finite or outside [0, L).
 * This is the textbook stable counting sort: count, exclusive prefix sum,
 * then one pass in input order.
 */
int orc_bin(int64_t n, const float *pos, double L, int cpd,
            int32_t *cid, int64_t *cell_start, int64_t *perm, float *rel)
{
    if (n < 0 || cpd < 1 || !(L > 0.0)) return ORC_EINVAL;
    int64_t ncell = (int64_t)cpd * cpd * cpd;
    for (int64_t i = 0; i < n; ++i) {
        int c3[3];
        for (int a = 0; a < 3; ++a) {
            double x = (double)pos[3 * i + a];
            if (!(x >= 0.0 && x < L)) return ORC_ERANGE;
            c3[a] = cell_index(cell_unit(x, cpd, L), cpd);
        }
        cid[i] = (int32_t)(((int64_t)c3[0] * cpd + c3[1]) * cpd + c3[2]);
    }
    int64_t *cursor = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    if (!cursor) return ORC_ENOMEM;
    for (int64_t i = 0; i < n; ++i) cursor[cid[i] + 1] += 1;
    for (int64_t c = 0; c < ncell; ++c) cursor[c + 1] += cursor[c];
    memcpy(cell_start, cursor, (size_t)(ncell + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = cursor[cid[i]]++;
        perm[k] = i;
    }
    free(cursor);
    if (rel) {
        for (int64_t k = 0; k < n; ++k) {
            int64_t i = perm[k];
            for (int a = 0; a < 3; ++a) {
                double u = cell_unit((double)pos[3 * i + a], cpd, L);
                int c = cell_index(u, cpd);
                rel[3 * k + a] = (float)(u - ((double)c + 0.5));
            }
        }
    }
    return ORC_OK;
}

/* Cell lists from given linear cell ids (the binning is an input so that a
 * finite-difference test can hold it fixed while positions move). */
static int build_lists(int64_t n, const int32_t *cid, int64_t ncell,
                       int64_t **start_out, int64_t **list_out)
{
    int64_t *start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *list = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *cur = (int64_t *)malloc((size_t)(ncell + 1) * sizeof(int64_t));
    if (!start || !list || !cur) { free(start); free(list); free(cur); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        if (cid[i] < 0 || cid[i] >= ncell) { free(start); free(list); free(cur); return ORC_EINVAL; }
        start[cid[i] + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    memcpy(cur, start, (size_t)(ncell + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) list[cur[cid[i]]++] = i;
    free(cur);
    *start_out = start;
    *list_out = list;
    return ORC_OK;
}

static inline int wrap(int t, int cpd) { int w = t % cpd; return w < 0 ? w + cpd : w; }

/*
 * orc_accel: near-field accelerations by direct summation (Sec. 3.1).
 *   pos    [n*3] double positions
 *   cid    [n]   linear cell id of each particle (from orc_bin, or held fixed)
 *   mass   [n]   G*m per particle, or NULL for all equal to m0
 *   L, cpd, R, eps : box side, cells per dimension, near-field radius in
 *                    cells, Plummer softening length
 *   sinks  [ns]  particle indices to evaluate, or NULL for all (ns = n)
 *   acc    [ns*3] out
 * For sink i in cell c and each d in [-R,R]^3 the source cell is
 * c' = (c + d) mod CPD and its image shift is S = ((c + d) - c') / CPD, so
 * Delta = (x_j - x_i) + S*L. The j = i term is included (it is exactly 0).
 */
int orc_accel(int64_t n, const double *pos, const int32_t *cid, const double *mass,
              double m0, double L, int cpd, int R, double eps,
              const int64_t *sinks, int64_t ns, double *acc)
{
    if (n < 0 || cpd < 1 || R < 0 || !(L > 0.0) || !(eps > 0.0)) return ORC_EINVAL;
    if (2 * R + 1 > cpd) return ORC_EINVAL;
    int64_t ncell = (int64_t)cpd * cpd * cpd;
    int64_t *start, *list;
    int rc = build_lists(n, cid, ncell, &start, &list);
    if (rc) return rc;
    if (!sinks) ns = n;
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < ns; ++q) {
        int64_t i = sinks ? sinks[q] : q;
        int c = cid[i];
        int cx = c / (cpd * cpd), cy = (c / cpd) % cpd, cz = c % cpd;
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int dx = -R; dx <= R; ++dx)
        for (int dy = -R; dy <= R; ++dy)
        for (int dz = -R; dz <= R; ++dz) {
            int tx = cx + dx, ty = cy + dy, tz = cz + dz;
            int wx = wrap(tx, cpd), wy = wrap(ty, cpd), wz = wrap(tz, cpd);
            double sx = (double)((tx - wx) / cpd) * L;
            double sy = (double)((ty - wy) / cpd) * L;
            double sz = (double)((tz - wz) / cpd) * L;
            int64_t cc = ((int64_t)wx * cpd + wy) * cpd + wz;
            for (int64_t k = start[cc]; k < start[cc + 1]; ++k) {
                int64_t j = list[k];
                double ddx = (pos[3 * j + 0] - pos[3 * i + 0]) + sx;
                double ddy = (pos[3 * j + 1] - pos[3 * i + 1]) + sy;
                double ddz = (pos[3 * j + 2] - pos[3 * i + 2]) + sz;
                double s = ddx * ddx + ddy * ddy + ddz * ddz + eps2;
                double mj = mass ? mass[j] : m0;
                double f = mj / (s * sqrt(s));
                ax += f * ddx;
                ay += f * ddy;
                az += f * ddz;
            }
        }
        acc[3 * q + 0] = ax;
        acc[3 * q + 1] = ay;
        acc[3 * q + 2] = az;
    }
    free(start);
    free(list);
    return ORC_OK;
}

/*
 * orc_accel_ex: the near-field sum of orc_accel with a choice of pair law,
 * plus the kernel density estimate of Sec. 3.3.
 *   law 0 (Plummer, Sec. 5.2): f(r) = (r^2 + eps^2)^(-3/2)
 *   law 1 (spline): the force returns to exactly 1/r^2 at r >= eps (Sec. 2.5,
 *       Sec. 5.2 describe such a spline without printing it); inside,
 *       F(r) = r (10 - 15 u + 6 u^2) / eps^3 with u = r / eps, the lowest-order
 *       form r P(u) that meets 1/r^2 at u = 1 with continuous first and second
 *       derivatives. Here eps is the radius where the law becomes 1/r^2.
 *   The acceleration term is m_j f(r) Delta with f = F / r.
 *   kde_b > 0: dens[q] = sum_j m_j (1 - r^2 / b^2) over the same
 *       neighbourhood for r < b (Sec. 3.3: weighting 1 - r^2/b^2), self pair
 *       included (it adds m_i). dens may be NULL when kde_b <= 0.
 */
int orc_accel_ex(int64_t n, const double *pos, const int32_t *cid, const double *mass,
                 double m0, double L, int cpd, int R, double eps, int law, double kde_b,
                 const int64_t *sinks, int64_t ns, double *acc, double *dens)
{
    if (n < 0 || cpd < 1 || R < 0 || !(L > 0.0) || !(eps > 0.0)) return ORC_EINVAL;
    if (2 * R + 1 > cpd || law < 0 || law > 1) return ORC_EINVAL;
    if (kde_b > 0.0 && !dens) return ORC_EINVAL;
    int64_t ncell = (int64_t)cpd * cpd * cpd;
    int64_t *start, *list;
    int rc = build_lists(n, cid, ncell, &start, &list);
    if (rc) return rc;
    if (!sinks) ns = n;
    const double eps2 = eps * eps, b2 = kde_b * kde_b;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < ns; ++q) {
        int64_t i = sinks ? sinks[q] : q;
        int c = cid[i];
        int cx = c / (cpd * cpd), cy = (c / cpd) % cpd, cz = c % cpd;
        double ax = 0.0, ay = 0.0, az = 0.0, rho = 0.0;
        for (int dx = -R; dx <= R; ++dx)
        for (int dy = -R; dy <= R; ++dy)
        for (int dz = -R; dz <= R; ++dz) {
            int tx = cx + dx, ty = cy + dy, tz = cz + dz;
            int wx = wrap(tx, cpd), wy = wrap(ty, cpd), wz = wrap(tz, cpd);
            double sx = (double)((tx - wx) / cpd) * L;
            double sy = (double)((ty - wy) / cpd) * L;
            double sz = (double)((tz - wz) / cpd) * L;
            int64_t cc = ((int64_t)wx * cpd + wy) * cpd + wz;
            for (int64_t k = start[cc]; k < start[cc + 1]; ++k) {
                int64_t j = list[k];
                double ddx = (pos[3 * j + 0] - pos[3 * i + 0]) + sx;
                double ddy = (pos[3 * j + 1] - pos[3 * i + 1]) + sy;
                double ddz = (pos[3 * j + 2] - pos[3 * i + 2]) + sz;
                double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                double mj = mass ? mass[j] : m0;
                double f;
                if (law == 0) {
                    double s = r2 + eps2;
                    f = 1.0 / (s * sqrt(s));
                } else {
                    double r = sqrt(r2);
                    if (r >= eps) {
                        f = r2 > 0.0 ? 1.0 / (r2 * r) : 0.0;
                    } else {
                        double u = r / eps;
                        f = (10.0 - 15.0 * u + 6.0 * u * u) / (eps2 * eps);
                    }
                }
                ax += mj * f * ddx;
                ay += mj * f * ddy;
                az += mj * f * ddz;
                if (kde_b > 0.0 && r2 < b2) rho += mj * (1.0 - r2 / b2);
            }
        }
        acc[3 * q + 0] = ax;
        acc[3 * q + 1] = ay;
        acc[3 * q + 2] = az;
        if (kde_b > 0.0) dens[q] = rho;
    }
    free(start);
    free(list);
    return ORC_OK;
}

/*
 * orc_vjp: vector-Jacobian product of the near-field accelerations with
 * respect to the positions, for the scalar  Lw = sum_i w_i . a_i  with the
 * binning held fixed.
 *
 * With a_i = sum_j m_j P(Delta_ij), P(D) = D (|D|^2+eps^2)^(-3/2), the
 * Jacobian of P is J(D) = s^(-3/2) I - 3 s^(-5/2) D D^T, s = |D|^2 + eps^2.
 * da_i/dx_j = m_j J(Delta_ij) for j != i and da_i/dx_i = -sum_j m_j J(Delta_ij).
 * J is even in D and the neighbour relation is symmetric (with mirrored
 * images), so
 *     g_k = dLw/dx_k = sum_{j in nbr(k)} J(Delta_kj) (m_k w_j - m_j w_k).
 *   w [n*3] cotangent; g [ns*3] out; other arguments as orc_accel.
 */
int orc_vjp_ex(int64_t n, const double *pos, const int32_t *cid, const double *mass,
               double m0, double L, int cpd, int R, double eps, int law, const double *w,
               const int64_t *sinks, int64_t ns, double *g);

int orc_vjp(int64_t n, const double *pos, const int32_t *cid, const double *mass,
            double m0, double L, int cpd, int R, double eps, const double *w,
            const int64_t *sinks, int64_t ns, double *g)
{
    return orc_vjp_ex(n, pos, cid, mass, m0, L, cpd, R, eps, 0, w, sinks, ns, g);
}

/*
 * orc_vjp_ex: orc_vjp for either pair law of orc_accel_ex. With
 * P(D) = D f(r), r = |D|, the Jacobian is J(D) = f I + (f'(r)/r) D D^T:
 *   law 0: f = s^(-3/2), f'/r = -3 s^(-5/2)           (s = r^2 + eps^2)
 *   law 1, r >= eps: f = r^-3, f'/r = -3 r^-5
 *   law 1, 0 < r < eps: f = (10 - 15u + 6u^2)/eps^3, f'(r) = (-15 + 12u)/eps^4
 *   law 1, r = 0: J = f(0) I (the D D^T term vanishes as D -> 0).
 * The spline's f and f' are continuous at r = eps, so J is too.
 */
int orc_vjp_ex(int64_t n, const double *pos, const int32_t *cid, const double *mass,
               double m0, double L, int cpd, int R, double eps, int law, const double *w,
               const int64_t *sinks, int64_t ns, double *g)
{
    if (n < 0 || cpd < 1 || R < 0 || !(L > 0.0) || !(eps > 0.0)) return ORC_EINVAL;
    if (2 * R + 1 > cpd || law < 0 || law > 1) return ORC_EINVAL;
    int64_t ncell = (int64_t)cpd * cpd * cpd;
    int64_t *start, *list;
    int rc = build_lists(n, cid, ncell, &start, &list);
    if (rc) return rc;
    if (!sinks) ns = n;
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < ns; ++q) {
        int64_t k = sinks ? sinks[q] : q;
        int c = cid[k];
        int cx = c / (cpd * cpd), cy = (c / cpd) % cpd, cz = c % cpd;
        double mk = mass ? mass[k] : m0;
        double gx = 0.0, gy = 0.0, gz = 0.0;
        for (int dx = -R; dx <= R; ++dx)
        for (int dy = -R; dy <= R; ++dy)
        for (int dz = -R; dz <= R; ++dz) {
            int tx = cx + dx, ty = cy + dy, tz = cz + dz;
            int wx = wrap(tx, cpd), wy = wrap(ty, cpd), wz = wrap(tz, cpd);
            double sx = (double)((tx - wx) / cpd) * L;
            double sy = (double)((ty - wy) / cpd) * L;
            double sz = (double)((tz - wz) / cpd) * L;
            int64_t cc = ((int64_t)wx * cpd + wy) * cpd + wz;
            for (int64_t t = start[cc]; t < start[cc + 1]; ++t) {
                int64_t j = list[t];
                double D[3];
                D[0] = (pos[3 * j + 0] - pos[3 * k + 0]) + sx;
                D[1] = (pos[3 * j + 1] - pos[3 * k + 1]) + sy;
                D[2] = (pos[3 * j + 2] - pos[3 * k + 2]) + sz;
                double s = D[0] * D[0] + D[1] * D[1] + D[2] * D[2] + eps2;
                double mj = mass ? mass[j] : m0;
                double u[3];
                for (int a = 0; a < 3; ++a) u[a] = mk * w[3 * j + a] - mj * w[3 * k + a];
                double Du = D[0] * u[0] + D[1] * u[1] + D[2] * u[2];
                if (law == 0) {
                    double s32 = 1.0 / (s * sqrt(s));      /* s^(-3/2) */
                    double s52 = s32 / s;                   /* s^(-5/2) */
                    /* J u = s^(-3/2) u - 3 s^(-5/2) D (D . u) */
                    gx += s32 * u[0] - 3.0 * s52 * D[0] * Du;
                    gy += s32 * u[1] - 3.0 * s52 * D[1] * Du;
                    gz += s32 * u[2] - 3.0 * s52 * D[2] * Du;
                } else {
                    double r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
                    double r = sqrt(r2), f, dfr;
                    if (r >= eps) {
                        f = 1.0 / (r2 * r);
                        dfr = -3.0 * f / r2;
                    } else if (r2 > 0.0) {
                        double uu = r / eps;
                        f = (10.0 - 15.0 * uu + 6.0 * uu * uu) / (eps2 * eps);
                        dfr = (-15.0 + 12.0 * uu) / (eps2 * eps2 * r);
                    } else {
                        f = 10.0 / (eps2 * eps);
                        dfr = 0.0;
                    }
                    /* J u = f u + (f'/r) D (D . u) */
                    gx += f * u[0] + dfr * D[0] * Du;
                    gy += f * u[1] + dfr * D[1] * Du;
                    gz += f * u[2] + dfr * D[2] * Du;
                }
            }
        }
        g[3 * q + 0] = gx;
        g[3 * q + 1] = gy;
        g[3 * q + 2] = gz;
    }
    free(start);
    free(list);
    return ORC_OK;
}

/*
 * orc_interactions: number of pairwise interactions ("directs", Sec. 4.3)
 * of the near-field sum, sum over cells c of n_c * sum_{d in [-R,R]^3} n_{c+d},
 * self pairs included; also the per-sink source count when nsrc != NULL.
 */
int64_t orc_interactions(int64_t n, const int32_t *cid, int cpd, int R, int64_t *nsrc)
{
    int64_t ncell = (int64_t)cpd * cpd * cpd;
    int64_t *cnt = (int64_t *)calloc((size_t)ncell, sizeof(int64_t));
    int64_t *src = (int64_t *)calloc((size_t)ncell, sizeof(int64_t));
    if (!cnt || !src) { free(cnt); free(src); return -1; }
    for (int64_t i = 0; i < n; ++i) cnt[cid[i]] += 1;
    int64_t total = 0;
    for (int64_t c = 0; c < ncell; ++c) {
        if (!cnt[c]) continue;
        int cx = (int)(c / ((int64_t)cpd * cpd)), cy = (int)((c / cpd) % cpd), cz = (int)(c % cpd);
        int64_t s = 0;
        for (int dx = -R; dx <= R; ++dx)
        for (int dy = -R; dy <= R; ++dy)
        for (int dz = -R; dz <= R; ++dz) {
            int64_t cc = ((int64_t)wrap(cx + dx, cpd) * cpd + wrap(cy + dy, cpd)) * cpd + wrap(cz + dz, cpd);
            s += cnt[cc];
        }
        src[c] = s;
        total += cnt[c] * s;
    }
    if (nsrc)
        for (int64_t i = 0; i < n; ++i) nsrc[i] = src[cid[i]];
    free(cnt);
    free(src);
    return total;
}

/*
 * orc_cell_timestep: the small-scale timestep criterion of Sec. 2.5, the
 * minimum over cells of (per-cell velocity dispersion) / (per-cell maximum
 * particle acceleration), times eta. The dispersion is the 3-D rms of
 * v - <v>_cell; cells with fewer than two particles or with all
 * accelerations zero give no bound. Returns +inf if no cell bounds the step.
 *   vel, acc [n*3] double; cid [n] cell of each particle.
 */
double orc_cell_timestep(int64_t n, const double *vel, const double *acc, const int32_t *cid,
                         int cpd, double eta)
{
    int64_t ncell = (int64_t)cpd * cpd * cpd;
    int64_t *start, *list;
    if (build_lists(n, cid, ncell, &start, &list)) return -1.0;
    double best = INFINITY;
    for (int64_t c = 0; c < ncell; ++c) {
        int64_t m = start[c + 1] - start[c];
        if (m < 2) continue;
        double mean[3] = {0.0, 0.0, 0.0}, amax = 0.0;
        for (int64_t k = start[c]; k < start[c + 1]; ++k) {
            int64_t i = list[k];
            for (int a = 0; a < 3; ++a) mean[a] += vel[3 * i + a];
            double a2 = acc[3 * i] * acc[3 * i] + acc[3 * i + 1] * acc[3 * i + 1] + acc[3 * i + 2] * acc[3 * i + 2];
            if (a2 > amax) amax = a2;
        }
        for (int a = 0; a < 3; ++a) mean[a] /= (double)m;
        double var = 0.0;
        for (int64_t k = start[c]; k < start[c + 1]; ++k) {
            int64_t i = list[k];
            for (int a = 0; a < 3; ++a) {
                double d = vel[3 * i + a] - mean[a];
                var += d * d;
            }
        }
        var /= (double)m;
        if (amax <= 0.0) continue;
        double r = sqrt(var) / sqrt(amax);
        if (r < best) best = r;
    }
    free(start);
    free(list);
    return eta * best;
}

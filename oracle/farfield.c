/*
 * farfield.c -- plain FP64 CPU oracle for the far-field force of the
 * near/far split (Maksimova et al. 2021, "AbacusSummit", Sec. 3.1).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark use it. It shares no code with the CUDA path.
 *
 * What Sec. 3.1 fixes:
 *   - the force on a particle is the near field (the direct sum over the
 *     (2R+1)^3 cells around its cell, one periodic image per cell offset,
 *     computed by oracle.c) plus the far field, which holds every other
 *     pairwise interaction, including all the other periodic images of the
 *     near-field particles;
 *   - the far field is a Taylor series of order p about each cell centre; its
 *     coefficients come from convolving, cyclically over the CPD^3 cells, the
 *     multipole moments of the cells with the "derivatives tensor", the
 *     derivatives of the periodic Green's function at each cell offset, which
 *     depends only on the grid. p = 8 with R = 2 in production.
 * Readings (the paper does not print the formulas):
 *   - Cartesian moments about the cell centre, M_m(c) = sum_j m_j z_j^m, for
 *     all multi-indices |m| <= p, and Taylor coefficients T_k for |k| <= p,
 *         T_k(c) = sum_c' sum_|m|<=p (-1)^|m| / m!  M_m(c')  D_{k+m}(c - c'),
 *     so the tensor is needed to order 2p;
 *   - D_q(d) = sum over periodic images n of the q-th Cartesian derivative of
 *     1/|d + n CPD| (cell units), leaving out the one image that lies in the
 *     near field, i.e. d + n CPD in [-R, R]^3;
 *   - the periodic sum is the Ewald sum with a uniform background and no
 *     surface term (the usual cosmological convention, forces from density
 *     fluctuations); for |q| >= 3 it equals the plain image sum, which
 *     converges absolutely there;
 *   - acceleration a = grad_y sum_k T_k y^k / k! at the particle's offset y
 *     from its cell centre, scaled by 1 / h^2 to box units (h = L / CPD).
 *
 * Every routine is the plain definition in double precision, with no
 * blocking; compiled with the near-field oracle into one library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define FF_OK 0
#define FF_EINVAL (-1)
#define FF_ENOMEM (-3)

/* ------------------------------------------------------------ multi-indices */
/* All (a, b, c) with a + b + c <= Q, ordered by total degree, then a
 * descending, then b descending. lut maps (a, b, c) to the position. */
typedef struct {
    int Q, n;
    int (*abc)[3];
    int *lut;
} MIdx;

static int midx_count(int Q) { return (Q + 1) * (Q + 2) * (Q + 3) / 6; }

static int midx_init(MIdx *m, int Q)
{
    m->Q = Q;
    m->n = midx_count(Q);
    m->abc = (int (*)[3])malloc(sizeof(int[3]) * (size_t)m->n);
    m->lut = (int *)malloc(sizeof(int) * (size_t)(Q + 1) * (Q + 1) * (Q + 1));
    if (!m->abc || !m->lut) { free(m->abc); free(m->lut); return FF_ENOMEM; }
    int i = 0;
    for (int t = 0; t <= Q; ++t)
        for (int a = t; a >= 0; --a)
            for (int b = t - a; b >= 0; --b) {
                int c = t - a - b;
                m->abc[i][0] = a; m->abc[i][1] = b; m->abc[i][2] = c;
                m->lut[(a * (Q + 1) + b) * (Q + 1) + c] = i;
                ++i;
            }
    return FF_OK;
}

static void midx_free(MIdx *m) { free(m->abc); free(m->lut); }

static inline int midx_at(const MIdx *m, int a, int b, int c)
{
    return m->lut[(a * (m->Q + 1) + b) * (m->Q + 1) + c];
}

/* ------------------------------------------------------------ radial functions */
/* g[n] = (1/r d/dr)^n f(r), n = 0..Q, for three radial functions. */

/* f = erfc(alpha r) / r:  g_n = (-1)^n B_n with
 * B_0 = erfc(alpha r)/r, B_n = ((2n-1) B_{n-1} + (2 alpha^2)^n exp(-alpha^2 r^2) / (alpha sqrt(pi))) / r^2 */
static void g_erfc(double r, double alpha, int Q, double *g)
{
    const double e = exp(-alpha * alpha * r * r) / (alpha * sqrt(M_PI));
    double B = erfc(alpha * r) / r, p2a = 1.0, sign = 1.0;
    g[0] = B;
    for (int n = 1; n <= Q; ++n) {
        p2a *= 2.0 * alpha * alpha;
        B = ((2.0 * n - 1.0) * B + p2a * e) / (r * r);
        sign = -sign;
        g[n] = sign * B;
    }
}

/* f = 1/r:  g_n = (-1)^n (2n-1)!! / r^(2n+1) */
static void g_inv(double r, int Q, double *g)
{
    double v = 1.0 / r;
    g[0] = v;
    for (int n = 1; n <= Q; ++n) {
        v *= -(2.0 * n - 1.0) / (r * r);
        g[n] = v;
    }
}

/* f = -erf(alpha r)/r = erfc(alpha r)/r - 1/r, smooth and finite at r = 0.
 * From the series erf(alpha r)/r = (2/sqrt(pi)) sum_m (-1)^m alpha^(2m+1) r^(2m) / (m! (2m+1)):
 *   g_n = -(2 alpha/sqrt(pi)) (-2 alpha^2)^n sum_j (-alpha^2 r^2)^j / (j! (2n + 2j + 1)).
 * Summed directly; the difference of the erfc and 1/r forms would cancel to
 * a few digits at high n. Used at near-field distances (alpha r of order 1). */
static void g_minus_erf(double r, double alpha, int Q, double *g)
{
    const double x = alpha * alpha * r * r;
    double pref = -2.0 * alpha / sqrt(M_PI);
    for (int n = 0; n <= Q; ++n) {
        double term = 1.0, sum = 0.0;
        for (int j = 0; j < 400; ++j) {
            const double t = term / (2.0 * n + 2.0 * j + 1.0);
            sum += t;
            if (j > x && fabs(t) < 1e-19 * fabs(sum)) break;
            term *= -x / (j + 1.0);
        }
        g[n] = pref * sum;
        pref *= -2.0 * alpha * alpha;
    }
}

/* Cartesian derivatives of a radial function at s: out[i] += d^(a,b,c) f(s)
 * for every multi-index i = (a, b, c) of mi, from g[n] = (1/r d/dr)^n f, by
 * the recursion R^(n)_{a+1,b,c} = a R^(n+1)_{a-1,b,c} + x R^(n+1)_{a,b,c}
 * (and the same in y, z), R^(n)_000 = g[n], d^(a,b,c) f = R^(0)_abc.
 * work holds (Q+1) x mi->n doubles. */
static void radial_derivs_add(const double s[3], const double *g, const MIdx *mi, double *work,
                              double *out)
{
    const int Q = mi->Q, N = mi->n;
    for (int i = 0; i < N; ++i) {
        const int a = mi->abc[i][0], b = mi->abc[i][1], c = mi->abc[i][2];
        const int t = a + b + c;
        for (int n = 0; n <= Q - t; ++n) {
            double v;
            if (t == 0) {
                v = g[n];
            } else if (a > 0) {
                v = s[0] * work[(n + 1) * N + midx_at(mi, a - 1, b, c)];
                if (a > 1) v += (a - 1) * work[(n + 1) * N + midx_at(mi, a - 2, b, c)];
            } else if (b > 0) {
                v = s[1] * work[(n + 1) * N + midx_at(mi, a, b - 1, c)];
                if (b > 1) v += (b - 1) * work[(n + 1) * N + midx_at(mi, a, b - 2, c)];
            } else {
                v = s[2] * work[(n + 1) * N + midx_at(mi, a, b, c - 1)];
                if (c > 1) v += (c - 1) * work[(n + 1) * N + midx_at(mi, a, b, c - 2)];
            }
            work[n * N + i] = v;
        }
    }
    for (int i = 0; i < N; ++i) out[i] += work[i];
}

/* ------------------------------------------------------------ derivatives tensor */
/* Ewald sum of the Cartesian derivatives of the periodic 1/r at the point d
 * (cell units, period P), all |q| <= Q:
 *   out[q] = sum_n d^q [erfc(alpha s)/s](s = d + n P)
 *          + (4 pi / P^3) sum_{k != 0} exp(-k^2 / (4 alpha^2)) / k^2  Re[(i k)^q exp(i k . d)]
 *          (q = 0 also gets the background constant -pi / (alpha^2 P^3)),
 * k = 2 pi m / P. With R >= 0, d integer: the image with d + n P in
 * [-R, R]^3 (the near field) is left out, i.e. its real-space term becomes
 * d^q [-erf(alpha s)/s]. With R < 0 nothing is left out (d must then not be a
 * lattice point). Cutoffs alpha r < 6.5 + Q/4 and k < (13 + Q/2) alpha: past
 * them every term, powers of r and k included, is below double rounding. */
static void ewald_dtensor(const double d[3], int P, int R, double alpha, const MIdx *mi,
                          double *work, double *out)
{
    const int Q = mi->Q, N = mi->n;
    double g[64];
    for (int i = 0; i < N; ++i) out[i] = 0.0;
    /* real space; the cutoffs grow with the order, whose terms carry
       powers (alpha r)^(2n) and k^q against the Gaussians */
    const double rc = (6.5 + 0.25 * Q) / alpha;
    const int nmax = (int)ceil(rc / P) + 1;
    for (int nx = -nmax; nx <= nmax; ++nx)
    for (int ny = -nmax; ny <= nmax; ++ny)
    for (int nz = -nmax; nz <= nmax; ++nz) {
        const double s[3] = {d[0] + nx * (double)P, d[1] + ny * (double)P, d[2] + nz * (double)P};
        const double r = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
        const int near = R >= 0 && fabs(s[0]) <= R && fabs(s[1]) <= R && fabs(s[2]) <= R;
        if (near) {
            g_minus_erf(r, alpha, Q, g);
        } else {
            if (r >= rc) continue;
            g_erfc(r, alpha, Q, g);
        }
        radial_derivs_add(s, g, mi, work, out);
    }
    /* reciprocal space */
    const double V = (double)P * P * P;
    const double kc = (13.0 + 0.5 * Q) * alpha;
    const int mmax = (int)ceil(kc * P / (2.0 * M_PI));
    double kp[3][64];
    for (int mx = -mmax; mx <= mmax; ++mx)
    for (int my = -mmax; my <= mmax; ++my)
    for (int mz = -mmax; mz <= mmax; ++mz) {
        if (!mx && !my && !mz) continue;
        const double k[3] = {2.0 * M_PI * mx / P, 2.0 * M_PI * my / P, 2.0 * M_PI * mz / P};
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        if (k2 > kc * kc) continue;
        const double w = 4.0 * M_PI / V * exp(-k2 / (4.0 * alpha * alpha)) / k2;
        const double ph = k[0] * d[0] + k[1] * d[1] + k[2] * d[2];
        const double cs = cos(ph), sn = sin(ph);
        for (int a = 0; a < 3; ++a) {
            kp[a][0] = 1.0;
            for (int j = 1; j <= Q; ++j) kp[a][j] = kp[a][j - 1] * k[a];
        }
        for (int i = 0; i < N; ++i) {
            const int a = mi->abc[i][0], b = mi->abc[i][1], c = mi->abc[i][2];
            const double kq = kp[0][a] * kp[1][b] * kp[2][c];
            /* Re[i^t (cos + i sin)] for t = |q| mod 4 */
            double re;
            switch ((a + b + c) & 3) {
                case 0: re = cs; break;
                case 1: re = -sn; break;
                case 2: re = -cs; break;
                default: re = sn; break;
            }
            out[i] += w * kq * re;
        }
    }
    out[0] -= M_PI / (alpha * alpha * V);
}

/*
 * orc_far_dtensor: the tensor above at one point d (cell units), all |q| <= Q,
 * in the multi-index order of this file (degree, then a, then b descending).
 *   P period (CPD), R near-field radius (or -1: leave nothing out), out[(Q+1)(Q+2)(Q+3)/6].
 */
int orc_far_dtensor(const double *d, int P, int R, double alpha, int Q, double *out)
{
    if (P < 1 || Q < 0 || Q > 40 || !(alpha > 0.0)) return FF_EINVAL;
    MIdx mi;
    if (midx_init(&mi, Q)) return FF_ENOMEM;
    double *work = (double *)malloc(sizeof(double) * (size_t)(Q + 1) * mi.n);
    if (!work) { midx_free(&mi); return FF_ENOMEM; }
    ewald_dtensor(d, P, R, alpha, &mi, work, out);
    free(work);
    midx_free(&mi);
    return FF_OK;
}

/* Multi-index listing for the tests: abc[3 * i + axis]. */
int orc_far_multi_indices(int Q, int32_t *abc)
{
    if (Q < 0 || Q > 40) return FF_EINVAL;
    MIdx mi;
    if (midx_init(&mi, Q)) return FF_ENOMEM;
    for (int i = 0; i < mi.n; ++i)
        for (int a = 0; a < 3; ++a) abc[3 * i + a] = mi.abc[i][a];
    midx_free(&mi);
    return FF_OK;
}

/* ------------------------------------------------------------ Ewald total force */
/*
 * orc_ewald_accel: the total periodic acceleration of every particle, Ewald
 * sum with a uniform background (the exact far + near, unsoftened):
 *   a_i = sum_{j != i} m_j grad psi(x_i - x_j),
 *   psi(r) = sum_n erfc(alpha|r + nL|)/|r + nL| + (4 pi/L^3) sum_{k != 0} exp(-k^2/4alpha^2)/k^2 cos(k.r),
 * k = 2 pi m / L; alpha in 1/box units.
 */
int orc_ewald_accel(int64_t n, const double *pos, const double *mass, double m0, double L,
                    double alpha, double *acc)
{
    if (n < 0 || !(L > 0.0) || !(alpha > 0.0)) return FF_EINVAL;
    const double rc = 6.5 / alpha, kc = 13.0 * alpha, V = L * L * L;
    const int nmax = (int)ceil(rc / L) + 1;
    const int mmax = (int)ceil(kc * L / (2.0 * M_PI));
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double mj = mass ? mass[j] : m0;
            const double r0[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                                  pos[3 * i + 2] - pos[3 * j + 2]};
            double gx = 0.0, gy = 0.0, gz = 0.0;
            for (int nx = -nmax; nx <= nmax; ++nx)
            for (int ny = -nmax; ny <= nmax; ++ny)
            for (int nz = -nmax; nz <= nmax; ++nz) {
                const double s[3] = {r0[0] + nx * L, r0[1] + ny * L, r0[2] + nz * L};
                const double r = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
                if (r >= rc) continue;
                /* grad [erfc(alpha r)/r] = -s (erfc(alpha r)/r^3 + 2 alpha/sqrt(pi) exp(-alpha^2 r^2)/r^2) */
                const double B1 = (erfc(alpha * r) / r + 2.0 * alpha / sqrt(M_PI) * exp(-alpha * alpha * r * r)) / (r * r);
                gx -= s[0] * B1; gy -= s[1] * B1; gz -= s[2] * B1;
            }
            for (int mx = -mmax; mx <= mmax; ++mx)
            for (int my = -mmax; my <= mmax; ++my)
            for (int mz = -mmax; mz <= mmax; ++mz) {
                if (!mx && !my && !mz) continue;
                const double k[3] = {2.0 * M_PI * mx / L, 2.0 * M_PI * my / L, 2.0 * M_PI * mz / L};
                const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                if (k2 > kc * kc) continue;
                /* grad cos(k.r) = -k sin(k.r) */
                const double w = -4.0 * M_PI / V * exp(-k2 / (4.0 * alpha * alpha)) / k2 *
                                 sin(k[0] * r0[0] + k[1] * r0[1] + k[2] * r0[2]);
                gx += w * k[0]; gy += w * k[1]; gz += w * k[2];
            }
            ax += mj * gx; ay += mj * gy; az += mj * gz;
        }
        acc[3 * i] = ax; acc[3 * i + 1] = ay; acc[3 * i + 2] = az;
    }
    return FF_OK;
}

/* ------------------------------------------------------------ far field */
static double factorial(int k) { double f = 1.0; for (int i = 2; i <= k; ++i) f *= i; return f; }

/*
 * orc_far_accel: far-field acceleration of every particle by the multipole /
 * derivatives-tensor / Taylor method of Sec. 3.1, order p.
 *   pos [n*3] box units in [0, L); cid [n] cell ids of the near-field binning
 *   (x slowest); mass [n] or NULL (m0); R near-field radius; alpha Ewald
 *   splitting in 1/cell units; acc [n*3] out, box units.
 * Steps: (1) multipoles M_m(c), |m| <= p, about cell centres; (2) tensor
 * D_q(d), |q| <= 2p, for every cell offset d in [0, CPD)^3; (3) T_k(c) by the
 * cyclic convolution, summed directly over cell pairs; (4) Taylor gradient at
 * each particle.
 */
int orc_far_accel(int64_t n, const double *pos, const int32_t *cid, const double *mass, double m0,
                  double L, int cpd, int R, int p, double alpha, double *acc)
{
    if (n < 0 || cpd < 1 || R < 0 || 2 * R + 1 > cpd || p < 1 || p > 16 || !(L > 0.0) || !(alpha > 0.0))
        return FF_EINVAL;
    const int64_t ncell = (int64_t)cpd * cpd * cpd;
    MIdx mp, mq;
    if (midx_init(&mp, p)) return FF_ENOMEM;
    if (midx_init(&mq, 2 * p)) { midx_free(&mp); return FF_ENOMEM; }
    const int NP = mp.n, NQ = mq.n;
    double *M = (double *)calloc((size_t)ncell * NP, sizeof(double));
    double *D = (double *)malloc(sizeof(double) * (size_t)ncell * NQ);
    double *T = (double *)calloc((size_t)ncell * NP, sizeof(double));
    int *add = (int *)malloc(sizeof(int) * (size_t)NP * NP);
    double *coef = (double *)malloc(sizeof(double) * (size_t)NP);
    if (!M || !D || !T || !add || !coef) {
        free(M); free(D); free(T); free(add); free(coef); midx_free(&mp); midx_free(&mq);
        return FF_ENOMEM;
    }
    const double u = (double)cpd / L;   /* box -> cell units */
    /* (1) multipoles, serial in particle order */
    for (int64_t j = 0; j < n; ++j) {
        const int c = cid[j];
        const int cx = c / (cpd * cpd), cy = (c / cpd) % cpd, cz = c % cpd;
        const double z[3] = {pos[3 * j] * u - (cx + 0.5), pos[3 * j + 1] * u - (cy + 0.5),
                             pos[3 * j + 2] * u - (cz + 0.5)};
        const double mj = mass ? mass[j] : m0;
        for (int i = 0; i < NP; ++i)
            M[(int64_t)c * NP + i] += mj * pow(z[0], mp.abc[i][0]) * pow(z[1], mp.abc[i][1]) *
                                      pow(z[2], mp.abc[i][2]);
    }
    /* (2) derivatives tensor at every integer offset */
    int rc = FF_OK;
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * (size_t)(2 * p + 1) * NQ);
        if (!work) {
#pragma omp atomic write
            rc = FF_ENOMEM;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t e = 0; e < ncell; ++e) {
                const double d[3] = {(double)(e / ((int64_t)cpd * cpd)), (double)((e / cpd) % cpd),
                                     (double)(e % cpd)};
                ewald_dtensor(d, cpd, R, alpha, &mq, work, D + e * NQ);
            }
            free(work);
        }
    }
    if (rc) goto out;
    /* (3) T_k(c) = sum_c' sum_m (-1)^|m| / m! M_m(c') D_{k+m}(c - c') */
    for (int k = 0; k < NP; ++k)
        for (int m = 0; m < NP; ++m)
            add[k * NP + m] = midx_at(&mq, mp.abc[k][0] + mp.abc[m][0], mp.abc[k][1] + mp.abc[m][1],
                                      mp.abc[k][2] + mp.abc[m][2]);
    for (int m = 0; m < NP; ++m) {
        const int a = mp.abc[m][0], b = mp.abc[m][1], c = mp.abc[m][2];
        coef[m] = (((a + b + c) & 1) ? -1.0 : 1.0) / (factorial(a) * factorial(b) * factorial(c));
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < ncell; ++c) {
        const int cx = (int)(c / ((int64_t)cpd * cpd)), cy = (int)((c / cpd) % cpd), cz = (int)(c % cpd);
        for (int64_t c2 = 0; c2 < ncell; ++c2) {
            const int x2 = (int)(c2 / ((int64_t)cpd * cpd)), y2 = (int)((c2 / cpd) % cpd), z2 = (int)(c2 % cpd);
            const int64_t e = ((int64_t)((cx - x2 + cpd) % cpd) * cpd + (cy - y2 + cpd) % cpd) * cpd +
                              (cz - z2 + cpd) % cpd;
            const double *Dd = D + e * NQ;
            const double *Mc = M + c2 * NP;
            for (int k = 0; k < NP; ++k) {
                double s = 0.0;
                for (int m = 0; m < NP; ++m) s += coef[m] * Mc[m] * Dd[add[k * NP + m]];
                T[c * NP + k] += s;
            }
        }
    }
    /* (4) a = grad_y sum_k T_k y^k / k!  -> a_x = sum_j T_{j + e_x} y^j / j!, |j| <= p - 1 */
    {
        const double sc = u * u;   /* cell -> box units for an acceleration */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            const int c = cid[i];
            const int cx = c / (cpd * cpd), cy = (c / cpd) % cpd, cz = c % cpd;
            const double y[3] = {pos[3 * i] * u - (cx + 0.5), pos[3 * i + 1] * u - (cy + 0.5),
                                 pos[3 * i + 2] * u - (cz + 0.5)};
            double a3[3] = {0.0, 0.0, 0.0};
            for (int j = 0; j < NP; ++j) {
                const int ja = mp.abc[j][0], jb = mp.abc[j][1], jc = mp.abc[j][2];
                if (ja + jb + jc > p - 1) continue;
                const double yj = pow(y[0], ja) * pow(y[1], jb) * pow(y[2], jc) /
                                  (factorial(ja) * factorial(jb) * factorial(jc));
                a3[0] += T[(int64_t)c * NP + midx_at(&mp, ja + 1, jb, jc)] * yj;
                a3[1] += T[(int64_t)c * NP + midx_at(&mp, ja, jb + 1, jc)] * yj;
                a3[2] += T[(int64_t)c * NP + midx_at(&mp, ja, jb, jc + 1)] * yj;
            }
            acc[3 * i] = a3[0] * sc; acc[3 * i + 1] = a3[1] * sc; acc[3 * i + 2] = a3[2] * sc;
        }
    }
out:
    free(M); free(D); free(T); free(add); free(coef);
    midx_free(&mp); midx_free(&mq);
    return rc;
}

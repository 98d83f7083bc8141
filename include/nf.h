/*
 * nf.h -- C ABI of libnf, the GB300 (sm_103a) near-field direct-sum library.
 *
 * The operation (Maksimova et al. 2021, "AbacusSummit", Sec. 3.1): a periodic
 * box of side L is cut into CPD^3 cubic cells; the near-field acceleration of
 * a particle is the direct sum over every particle of the cells whose offset
 * d from its own cell lies in [-R, R]^3 (R = near-field radius in cells, 2 in
 * the paper), each source cell taken at the one periodic image that sits at
 * offset d. The pair law is Plummer softening, the gradient of the potential
 * -G m / sqrt(r^2 + eps^2) named in Sec. 5.2:
 *
 *     a_i = sum_j G m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2)
 *
 * G is folded into the masses. The self pair (j = i) is included and is 0.
 *
 * Conventions for every entry point:
 *   - All array pointers are DEVICE pointers owned by the caller, except
 *     where a parameter says "host". Arrays are C-contiguous; a position or
 *     acceleration array is N x 3 float32, particle-major (x, y, z per row),
 *     in the caller's (input) particle order.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream). Calls return once the work is enqueued,
 *     except where a function says it synchronises.
 *   - The library owns its internal buffers (cell-sorted particles, cell
 *     table, work list). It keeps no pointer to caller memory after a call
 *     returns: nf_bin_particles copies positions into cell-sorted storage, so
 *     compute calls use that snapshot.
 *   - Errors are returned as negative nf_status codes; no C++ exception
 *     crosses the ABI and no kernel traps. nf_last_error() gives the message.
 *   - One context is bound to one device and is not thread-safe: calls on
 *     the same context must be serialised by the caller.
 */
#ifndef NF_H
#define NF_H

#include <stdint.h>

#if defined(__GNUC__)
#define NF_API __attribute__((visibility("default")))
#else
#define NF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nf_ctx nf_ctx;

typedef enum nf_status {
    NF_OK = 0,
    NF_EINVAL = -1,    /* bad argument (sizes, CPD < 2R+1, eps <= 0, N > capacity, ...) */
    NF_ERANGE = -2,    /* a position component is not finite or outside [0, L) */
    NF_ENOMEM = -3,    /* device or host allocation failed */
    NF_ECUDA = -4,     /* a CUDA runtime call failed; see nf_last_error */
    NF_ESTATE = -5,    /* call out of order (e.g. compute before binning) */
    NF_ETIMEOUT = -6   /* a bounded device-side wait gave up (the cell sort's
                          look-back); the result of that call is invalid */
} nf_status;

typedef enum nf_softening {
    NF_SOFT_PLUMMER = 0,    /* Plummer law above (Sec. 5.2) */
    NF_SOFT_SPLINE = 1      /* spline law that is exactly Newtonian for r >= eps
                               (Sec. 2.5, Sec. 5.2): inside, the pair force is
                               G m r (10 - 15 u + 6 u^2) / eps^3 with u = r / eps,
                               the lowest-order r P(r/eps) meeting 1/r^2 at eps
                               with continuous first and second derivatives; eps
                               is the radius where the law becomes 1/r^2.
                               NF_PREC_FP32 contexts only; forward pass,
                               density estimate and adjoint. */
} nf_softening;

typedef enum nf_precision {
    NF_PREC_FP32 = 0,       /* FP32 pair arithmetic on cell-relative coordinates;
                               each 128-source tile is summed afresh and the
                               tile sums are added to the per-sink total */
    NF_PREC_FP32_COMP = 1,  /* same pair loop; the tile sums are folded into a
                               compensated (hi, lo) per-sink total by TwoSum */
    NF_PREC_FP64_REF = 2,   /* FP64 pair arithmetic on the GPU (reference timing) */
    NF_PREC_FP32_COMP_PAIR = 3  /* FP32, every pair term added to a compensated
                                   (hi, lo) total by TwoSum (slowest FP32 form) */
} nf_precision;

/* Figures of the last binning / compute on a context (see nf_get_stats). */
typedef struct nf_stats {
    int64_t n_particles;     /* particles binned by the last nf_bin_particles */
    int64_t n_cells;         /* total cells over all boxes */
    int64_t interactions;    /* pairwise interactions of one force pass, self
                                pairs included: sum_c n_c * sum_{|d|<=R} n_{c+d} */
    int64_t max_occupancy;   /* largest cell population */
    int64_t n_items;         /* work items of the last compute */
    double  momentum[3];     /* sum_i m_i a_i of the last nf_compute_accel, FP64 */
    double  abs_momentum;    /* sum_i m_i |a_i| (scale for momentum[]) */
    double  bin_ms;          /* device time of the last binning (CUDA events) */
    double  pair_ms;         /* device time of the last pair (or adjoint) kernel */
    int64_t kernel_launches; /* kernels launched by this context so far, graph
                                replays counted kernel by kernel */
    double  far_ms;          /* device time of the last nf_compute_far (0 if none) */
    double  far_conv_ms;     /* of which the per-frequency tensor products */
    int64_t n_pencils;       /* pencils (four-cell runs served by one block) of the last compute */
    int64_t n_small;         /* work items of the last compute served by the small-item kernel */
} nf_stats;

/* Launch shape of the pair kernels. sinks_per_lane in {1,2,4}; warps_per_block
 * in {2,4,8,16}; blocks_per_sm = 0 picks the occupancy maximum; use_graph = 1
 * replays the compute phase from a captured CUDA graph; source_tile in
 * {0, 64, 128, 256}: sources staged in shared memory per tile by the plain
 * (Plummer, no density) FP32 kernels, 0 meaning 128 (the other kernels
 * always stage 128); use_pencils = 1 lets the plain FP32 forward pass
 * (sinks_per_lane 4, R <= 2) serve runs of four z-adjacent cells with one
 * block whose warps share the staged sources (the first 64 sinks of each
 * cell; where the neighbourhood is sparse enough), the rest as usual;
 * small_items = 1 lets the same pass (sinks_per_lane 4) serve the work items
 * of at most 8 sinks over at most 32,768 sources, mostly the sinks a cell has
 * left after its full groups, with a kernel whose lanes read their sources
 * straight from the records instead of staging tiles of the whole
 * neighbourhood. */
typedef struct nf_tuning {
    int sinks_per_lane;
    int warps_per_block;
    int blocks_per_sm;
    int use_graph;
    int vjp_sinks_per_lane;   /* sinks per lane of the adjoint kernel; 0 = as sinks_per_lane */
    int source_tile;
    int use_pencils;
    int small_items;
} nf_tuning;

/*
 * nf_init -- create a context for n_boxes independent periodic boxes.
 *   out        host: receives the context (set to NULL on failure)
 *   device     CUDA device ordinal
 *   n_boxes    >= 1
 *   box_size   host [n_boxes]: L of each box (> 0)
 *   cpd        host [n_boxes]: cells per dimension of each box, 2R+1 <= CPD <= 1024
 *   radius     near-field radius R in cells, 1..3 (the paper uses 2; Sec. 3.1)
 *   eps        host [n_boxes]: Plummer softening length of each box (> 0)
 *   softening  NF_SOFT_PLUMMER, or NF_SOFT_SPLINE (with NF_PREC_FP32 only)
 *   precision  an nf_precision value
 *   capacity   largest total particle count that will be binned (< 2^31)
 * Allocates all device buffers for `capacity` particles up front.
 * Returns NF_OK, NF_EINVAL, NF_ENOMEM or NF_ECUDA.
 */
NF_API int nf_init(nf_ctx **out, int device, int n_boxes, const double *box_size, const int *cpd,
            int radius, const double *eps, int softening, int precision, int64_t capacity);

/*
 * nf_bin_particles -- assign particles to cells and sort them by cell
 * (the cell lattice of Sec. 3.1): cell id, per-cell count, exclusive prefix
 * scan, stable scatter into cell order with cell-relative FP32 coordinates.
 *   pos          device [N x 3] float32, every component in [0, L) of its box
 *   mass         device [N] float32 G*m per particle, or NULL for equal masses
 *   mass_if_null G*m used for every particle when mass == NULL
 *   n            total particles N (0 <= N <= capacity)
 *   box_offsets  host [n_boxes+1]: particles of box b are rows
 *                [box_offsets[b], box_offsets[b+1]); NULL when n_boxes == 1
 *   stream       cudaStream_t
 * Synchronises `stream` once at the end to report NF_ERANGE for an invalid
 * position (such particles are binned to a safe cell and the context is
 * marked unbinned). Returns NF_OK, NF_EINVAL, NF_ERANGE, NF_ETIMEOUT (a
 * look-back wait of the sort gave up; nothing is binned), NF_ESTATE or
 * NF_ECUDA.
 */
NF_API int nf_bin_particles(nf_ctx *ctx, const float *pos, const float *mass, double mass_if_null,
                     int64_t n, const int64_t *box_offsets, void *stream);

/*
 * nf_set_box_masses -- equal masses per box: later nf_bin_particles calls
 * with mass == NULL give every particle of box b the mass gm[b] (instead of
 * mass_if_null), so boxes of different particle mass keep the equal-mass
 * pair kernel (G m applied once per sink).
 *   gm   host [n_boxes] G*m per box, or NULL to return to mass_if_null
 * Returns NF_OK or NF_EINVAL (non-finite value).
 */
NF_API int nf_set_box_masses(nf_ctx *ctx, const double *gm);

/*
 * nf_compute_accel -- near-field accelerations of every binned particle
 * (the direct O(N^2) near-field sum of Sec. 3.1 over (2R+1)^3 cells).
 *   acc     device [N x 3] float32 out, input particle order, caller-owned
 * Also accumulates the FP64 momentum diagnostic sum_i m_i a_i (nf_get_stats).
 * Returns NF_OK, NF_EINVAL, NF_ESTATE (not binned) or NF_ECUDA. Asynchronous.
 */
NF_API int nf_compute_accel(nf_ctx *ctx, float *acc, void *stream);

/*
 * nf_compute_accel_f64 -- as nf_compute_accel, with the accelerations written
 * as float64 (the natural output of NF_PREC_FP64_REF; the other precisions
 * widen their FP32 sums).
 *   acc     device [N x 3] float64 out, input particle order
 */
NF_API int nf_compute_accel_f64(nf_ctx *ctx, double *acc, void *stream);

/*
 * nf_compute_accel_density -- nf_compute_accel plus, in the same pair pass,
 * the kernel density estimate with which halo finding starts (Sec. 3.3):
 *     density_i = sum_{j near i} G m_j max(0, 1 - r_ij^2 / b^2),
 * over the same (2R+1)^3 cells, self pair included (it adds G m_i). The
 * paper takes b = 0.4 of the mean interparticle spacing; the sum is the
 * unnormalised kernel sum (divide by 8 pi b^3 / 15 for a mass density).
 *   acc      device [N x 3] float32 out, input order
 *   density  device [N] float32 out, input order
 *   kde_b    host [n_boxes]: b of each box, 0 < b <= R * L / CPD (so that
 *            every particle within b lies in the near field)
 * NF_PREC_FP32 contexts only. Returns NF_OK, NF_EINVAL, NF_ESTATE, NF_ECUDA.
 */
NF_API int nf_compute_accel_density(nf_ctx *ctx, float *acc, float *density, const double *kde_b,
                                    void *stream);

/*
 * nf_compute_accel_vjp -- vector-Jacobian product of the accelerations with
 * respect to the positions, for the scalar sum_i w_i . a_i with the binning of
 * the last nf_bin_particles held fixed:
 *     g_k = sum_{j near k} J(D_kj) (m_k w_j - m_j w_k),  D_kj = x_j - x_k,
 * with J(D) = f I + (f'(r)/r) D D^T the Jacobian of the pair term D f(r):
 *     NF_SOFT_PLUMMER: J(D) = s^(-3/2) I - 3 s^(-5/2) D D^T,  s = |D|^2 + eps^2;
 *     NF_SOFT_SPLINE:  f = (10 - 15u + 6u^2)/eps_s^3 with f'(r) = (-15 + 12u)/eps_s^4
 *                      for u = r/eps_s < 1, else f = r^-3, f'/r = -3 r^-5
 *                      (no counterpart in the paper, which does not use the
 *                      adjoint; the derivative of its near-field sum, Sec. 3.1).
 * Pair terms are recomputed, not stored.
 *   w         device [N x 3] float32 cotangent, input order
 *   grad_pos  device [N x 3] float32 out, input order, caller-owned
 * Returns NF_OK, NF_ESTATE or NF_ECUDA. Asynchronous. FP32 (and FP32_COMP
 * contexts) use FP32 arithmetic; NF_PREC_FP64_REF contexts use FP64.
 */
NF_API int nf_compute_accel_vjp(nf_ctx *ctx, const float *w, float *grad_pos, void *stream);

/*
 * nf_far_init -- enables the far field of the near/far split (Sec. 3.1:
 * Taylor series of order p about every cell centre, their
 * coefficients the cyclic convolution, done in Fourier space, of the cells'
 * multipole moments with the derivatives tensor of the periodic Green's
 * function). Builds that tensor once per distinct CPD of the context's boxes
 * (each box is its own periodic volume), for the near-field radius R, with
 * every image in the near field left out:
 *     D_q(d) = sum_n d^q (1/r) at d + n CPD, d + n CPD not in [-R, R]^3,
 * |q| <= 2p, as an Ewald sum with a uniform background (forces from density
 * fluctuations, the periodic convention of cosmological codes).
 *   order   p in [1, 8] (the paper uses 8)
 * Only the tensor components with x-exponent <= 2 are kept (the tensor is
 * harmonic, which fixes the rest): 409 of them at p = 8. Each is kept in
 * Fourier space as a real function, its transform over i^|q| (the tensor has
 * the parity of its order), about 4 x 409 CPD^3 bytes (3.5 GB at
 * CPD = 129); about four times that is held while it is built. Per step:
 * 3 x 8 (p+1)^2 CPD^3 bytes of buffers per box, plus, shared by the boxes,
 * 16 x p(p+1)(p+2)/6 bytes per cell of the largest box and 4 bytes per
 * particle of capacity. Synchronous.
 * Returns NF_OK, NF_EINVAL (order, a CPD above 192), NF_ENOMEM or NF_ECUDA
 * (cuFFT errors included).
 */
NF_API int nf_far_init(nf_ctx *ctx, int order, void *stream);

/*
 * nf_compute_far -- far-field accelerations of the binned particles:
 * multipoles M_m(c) = sum_j G m_j z_j^m (z relative to the cell centre, cell
 * units, |m| <= p), their transform, T_k = sum_m (-1)^|m| / m! D_{k+m} M_m per
 * frequency, the inverse transform, and a = grad sum_k T_k y^k / k! at each
 * particle, scaled to box units. The Plummer or spline softening of the near
 * field does not enter: the far field is unsoftened.
 *   acc         device [N x 3] float32, input order; written, or with
 *               accumulate != 0 added to (e.g. onto the near field)
 * Returns NF_OK, NF_ESTATE (no nf_far_init or no binning), NF_EINVAL or
 * NF_ECUDA (a cuFFT failure included, named in nf_last_error). Asynchronous.
 */
NF_API int nf_compute_far(nf_ctx *ctx, float *acc, int accumulate, void *stream);

/*
 * Particle update with a global timestep (Sec. 2.5: second-order leapfrog,
 * kick-drift-kick). All arrays are device [N x 3] float32 in input order, N
 * and the box of each particle being those of the last nf_bin_particles.
 *
 * nf_kick  -- v += a dt in double (the product and the sum each rounded,
 *             no fused multiply-add), then rounded once to float32.
 * nf_drift -- x += v dt in double (likewise unfused), wrapped into [0, L) of
 *             the particle's box by the exact remainder fmod(x, L) (plus L
 *             when negative), and rounded once to float32 (a value that
 *             rounds up to L becomes 0, its periodic image).
 * nf_timestep -- the small-scale criterion: eta times the minimum over cells
 *             of (3-D velocity dispersion about the cell mean) / (maximum
 *             particle |a| in the cell); cells with fewer than two particles
 *             or no acceleration give no bound (the result is +inf if none
 *             does). Cells are those of the last binning. Synchronises.
 * nf_kdk_step -- one step: v += a dt/2; x += v dt; re-bin x (same masses and
 *             box offsets as nf_bin_particles); a = near-field accelerations
 *             at the new x, plus the far field when nf_far_init has enabled
 *             it (the total force); v += a dt/2. On entry acc must hold the
 *             accelerations of the binned positions (near + far likewise);
 *             on exit it holds those of the new positions. Synchronises
 *             (through the re-binning).
 * Return NF_OK, NF_EINVAL, NF_ESTATE, NF_ERANGE (re-binning) or NF_ECUDA.
 */
NF_API int nf_kick(nf_ctx *ctx, float *vel, const float *acc, double dt, void *stream);
NF_API int nf_drift(nf_ctx *ctx, float *pos, const float *vel, double dt, void *stream);
NF_API int nf_timestep(nf_ctx *ctx, const float *vel, const float *acc, double eta, double *dt_out,
                       void *stream);
NF_API int nf_kdk_step(nf_ctx *ctx, float *pos, float *vel, float *acc, const float *mass,
                       double mass_if_null, double dt, const int64_t *box_offsets, void *stream);

/*
 * nf_accel_host -- end-to-end convenience call on HOST buffers: positions
 * (and masses) in, binning, accelerations out, then synchronises `stream`.
 *   pos_host   host [N x 3] float32. If it is page-locked memory the device
 *              can address (cudaHostAlloc / cudaHostRegister), the binning's
 *              first kernel loads it directly and keeps a device copy for the
 *              rest of the binning; otherwise it is copied to the device first.
 *   mass_host  host [N] float32 or NULL (then mass_if_null); copied.
 *   acc_host   host [N x 3] float32 out. If it is page-locked memory the
 *              device can address, the pair kernels store the accelerations
 *              into it directly, so the transfer overlaps the pass; otherwise
 *              they go to a device buffer that is copied back after the pass.
 * Device staging buffers are allocated on first use and kept by the context.
 */
NF_API int nf_accel_host(nf_ctx *ctx, const float *pos_host, const float *mass_host, double mass_if_null,
                  int64_t n, const int64_t *box_offsets, float *acc_host, void *stream);

/*
 * nf_copy_binning -- copy the result of the last nf_bin_particles (the cell
 * lattice and cell order of Sec. 3.1) into caller buffers, for inspection and
 * testing. Any pointer may be NULL.
 *   cell_start  device [n_cells + 1] int32: first sorted slot of each cell;
 *               box b's cells start at sum_{b' < b} CPD_b'^3, and within a box
 *               the cell id is (cx * CPD + cy) * CPD + cz
 *   perm        device [N] int32: input index of each sorted slot (stable:
 *               particles of one cell keep their input order)
 *   sorted      device [N x 4] float32: per sorted slot (rx, ry, rz, G m) with
 *               r = float32(u - (c + 0.5)), u = (x * CPD) / L in double, in
 *               cell units
 * Asynchronous on `stream`. Returns NF_OK, NF_EINVAL, NF_ESTATE or NF_ECUDA.
 */
NF_API int nf_copy_binning(nf_ctx *ctx, int32_t *cell_start, int32_t *perm, float *sorted,
                           void *stream);

/* nf_get_stats -- copy the figures of the last calls into *out (host).
 * Synchronises the stream of the last compute call. */
NF_API int nf_get_stats(nf_ctx *ctx, nf_stats *out);

/* nf_set_tuning / nf_get_tuning -- read or replace the launch shape. */
NF_API int nf_set_tuning(nf_ctx *ctx, const nf_tuning *t);
NF_API int nf_get_tuning(const nf_ctx *ctx, nf_tuning *t);

/*
 * nf_autotune -- time every candidate launch shape of the pair kernel on the
 * currently binned particles (CUDA events on `stream`, `reps` launches each):
 * sinks_per_lane in {1,2,4} x warps_per_block in {4,8} x source_tile in
 * {64,128,256} (the tile only where the kernel takes it). Keeps the fastest
 * in the context and copies it to *best (may be NULL). Synchronises
 * `stream`. Requires a prior nf_bin_particles.
 */
NF_API int nf_autotune(nf_ctx *ctx, int reps, nf_tuning *best, void *stream);

/*
 * Slab decomposition (Sec. 3.2: the box is split into x slabs, a node owns a
 * contiguous range of them, and a node's near field needs the R slabs on
 * either side of its range; Sec. 3.1: the near-field radius R sets that
 * width). A slab context holds one rank's owned slabs and R ghost slabs on
 * each side. Its accelerations equal, bit for bit, those of a whole-box
 * context for the same particles (same cells, same source order per cell).
 *
 * nf_init_slab -- a context for the owned x slabs [x_begin, x_begin +
 *   x_count) of one periodic box (other arguments as nf_init).
 *   x_begin    0 <= x_begin < cpd (global slab index)
 *   x_count    R <= x_count <= cpd; every rank must own at least R slabs
 *   precision  NF_PREC_FP32, NF_PREC_FP32_COMP or NF_PREC_FP32_COMP_PAIR
 *   capacity   largest owned + ghost particle count
 * nf_bin_particles then takes the OWNED particles only (a particle outside
 * the owned slabs is NF_ERANGE), and a compute call needs the ghosts of that
 * binning imported first (else NF_ESTATE). The adjoint, the far field,
 * nf_kdk_step and nf_accel_host are not available on slab contexts
 * (NF_EINVAL); nf_kick, nf_drift, nf_timestep (owned cells) and the density
 * estimate are.
 *
 * nf_slab_export -- the R boundary slabs a neighbour needs as ghosts, from
 *   the last binning: side 0 the first R owned slabs (for the rank on the
 *   left, whose right ghosts they are), side 1 the last R (for the rank on
 *   the right). Synchronises `stream` once to read the record count.
 *   counts     device [R * cpd * cpd] int32 out, or NULL: particles per cell
 *              of those slabs, cell order (x, y, z), x slowest
 *   records    device [records_cap x 4] float32 out, or NULL: their
 *              cell-sorted records (rx, ry, rz, G m), as nf_copy_binning
 *   n_records  host out: number of records of those slabs
 *   Returns NF_OK, NF_EINVAL (not a slab context, side, records_cap below
 *   n_records), NF_ESTATE (not binned) or NF_ECUDA.
 *
 * nf_slab_import -- install the ghost slabs for the current binning: the
 *   left neighbour's side-1 export as left ghosts and the right neighbour's
 *   side-0 export as right ghosts (with one rank, its own exports). The
 *   records are copied behind the owned ones and the cell table is rebuilt.
 *   Synchronises `stream` to check that every ghost count is >= 0 and that
 *   each side's counts add up to its n.
 *   left_counts, right_counts    device [R * cpd * cpd] int32
 *   left_records, right_records  device [n_left x 4], [n_right x 4] float32
 *   Returns NF_OK, NF_EINVAL (sizes, counts, capacity), NF_ESTATE or NF_ECUDA.
 *
 * nf_slab_of -- the global x slab floor((x * cpd) / L) (the binning's own
 *   arithmetic, Sec. 3.1) of each of n particles, -1 for an x outside [0, L)
 *   or not finite, on the current device; for routing particles to the rank
 *   that owns their slab.
 *   pos   device [n x 3] float32;  slab  device [n] int32 out
 *   Returns NF_OK, NF_EINVAL or NF_ECUDA (message via nf_last_error(NULL)).
 *   Asynchronous.
 */
NF_API int nf_init_slab(nf_ctx **out, int device, double box_size, int cpd, int radius, double eps,
                        int softening, int precision, int64_t capacity, int x_begin, int x_count);
NF_API int nf_slab_export(nf_ctx *ctx, int side, int32_t *counts, float *records, int64_t records_cap,
                          int64_t *n_records, void *stream);
NF_API int nf_slab_import(nf_ctx *ctx, const int32_t *left_counts, const float *left_records,
                          int64_t n_left, const int32_t *right_counts, const float *right_records,
                          int64_t n_right, void *stream);
NF_API int nf_slab_of(const float *pos, int64_t n, double box_size, int cpd, int32_t *slab,
                      void *stream);

/*
 * nf_bin_cells_noalloc -- the binning of nf_bin_particles for one box, for
 * callers that cannot allocate device memory: for example a host program
 * whose own pool allocator already holds the GPU's memory (a further
 * cudaMalloc would fail or fragment that pool), or a latency-critical loop
 * that cannot afford cudaMalloc's implicit device-wide synchronisation. The
 * paper has no counterpart to this call; it exists for such callers only.
 *
 * It allocates nothing. Its scratch (radix keys and values, cell counts,
 * histograms, scan partials, error word) lives in one file-scope device array
 * of about 17 MB, which every GPU that loads libnf holds until the process
 * exits. Limits: n <= 1,048,576 particles and CPD^3 <= 262,144 cells
 * (CPD <= 64); larger requests return NF_EINVAL.
 *   pos          device [n x 3] float32 in [0, box_size)
 *   mass         device [n] float32 G*m, or NULL for mass_if_null
 *   cell_start   device [CPD^3 + 1] int32 out (as nf_copy_binning)
 *   perm         device [n] int32 out
 *   sorted       device [n x 4] float32 out, 16-byte aligned, records
 *                (rx, ry, rz, G m) in cell units (as nf_copy_binning)
 * Runs on the current CUDA device and synchronises `stream` before
 * returning (to report NF_ERANGE). The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and caches it for the life
 * of the process; make that first call before any stream capture, and do not
 * reset the device (cudaDeviceReset) between calls, which would move the
 * array and leave the cached address stale. All calls on a device share the
 * one array, which keeps the last call's contents: calls that overlap on the
 * GPU (different streams or threads) race and must be serialised by the
 * caller.
 * Errors: NF_EINVAL, NF_ERANGE, NF_ETIMEOUT, NF_ECUDA; message via
 * nf_last_error(NULL).
 */
NF_API int nf_bin_cells_noalloc(const float *pos, const float *mass, double mass_if_null,
                                int64_t n, double box_size, int cpd, int32_t *cell_start,
                                int32_t *perm, float *sorted, void *stream);

/* nf_last_error -- message of the last failing call on ctx (never NULL);
 * with ctx == NULL, the message of the last failing nf_init or
 * nf_bin_cells_noalloc in this thread. */
NF_API const char *nf_last_error(const nf_ctx *ctx);

/* nf_status_string -- static name of a status code. */
NF_API const char *nf_status_string(int status);

/* nf_free -- release the context and all its device memory; NULL is a no-op. */
NF_API void nf_free(nf_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* NF_H */

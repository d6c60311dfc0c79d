/*
 * gslens — general spherical harmonic transforms for CMB lensing on GB300.
 *
 * C ABI of the CUDA library libgslens.so.  The operations are those of
 * Reinecke, Belkner & Carron, "Improved CMB (de-)lensing using general
 * spherical harmonic transforms" (arXiv:2304.10431):
 *
 *   forward  (Sect. 2, Eq. "forward"; spin s > 0: Eq. "forwardpol")
 *       spin 0: T_i        =                sum_lm a_lm          Y_lm(n'_i)
 *       spin s: (Q+iU)_i   = - e^{i s chi_i} sum_lm (G+iC)_lm   sY_lm(n'_i)
 *   adjoint  (Sect. 2, Eq. "adjoint"; spin s: the pair of equations and the
 *             G/C decomposition that follow Eq. "forwardpol")
 *       spin 0: a_lm = sum_i T_i Y*_lm(n'_i)
 *       spin s: +-sA_lm = sum_i e^{-+ i s chi_i} (Q +- iU)_i +-sY*_lm(n'_i),
 *               G = -(sA + (-1)^s (-s)A)/2,  C = -(sA - (-1)^s (-s)A)/(2i)
 *
 * computed as in Sect. 3: Legendre synthesis on an equiangular grid with a
 * ring on each pole, doubling of the sphere onto a torus, 2D FFT with kernel
 * deconvolution and zero padding, and non-uniform FFT interpolation (type 2);
 * the adjoint runs type-1 spreading, FFT, folding and adjoint synthesis.
 *
 * Conventions.
 *   - a_lm storage: index(l, m) = m (2 lmax + 1 - m) / 2 + l for
 *     0 <= m <= mmax, m <= l <= lmax; complex interleaved (re, im).  Element
 *     type: float (LENS_FP32) or double (LENS_FP64).  Real fields:
 *     a_{l,-m} = (-1)^m conj(a_lm).  For spin s the two components G and C are
 *     stored one after the other: [2][nalm] complex.
 *   - Y_lm orthonormal with the Condon-Shortley phase; spin-weighted
 *     sY_lm = sqrt((l-s)!/(l+s)!) eth^s Y_lm (equivalently
 *     (-1)^s sqrt((2l+1)/4pi) d^l_{m,-s}(theta) e^{i m phi}).
 *   - Maps: real, [ncomp][npoints] (spin 0: T; spin s: Q then U), element
 *     type float or double as above.
 *   - Points: double theta in [0, pi], any finite phi, optional chi (the spin
 *     phase of Fig. 1; NULL = 0), always FP64 on input.
 *   - The adjoint returns m >= 0 only.  With the real-field inner product
 *     <a,b> = sum_l Re(a_l0 conj b_l0) + 2 sum_{m>0} Re(a_lm conj b_lm) it is
 *     the exact transpose of the forward operator.
 *
 * Ownership and threading.
 *   - All buffer arguments are raw pointers; the caller owns them.  "_d"
 *     pointers are CUDA device pointers on the device that was current when
 *     the plan was created; "_h" pointers are host memory (pinned or not).
 *   - A plan owns its sorted point tables, tables and workspace (device
 *     memory).  One plan may be used by one call at a time; calls are
 *     asynchronous on the given stream (NULL: the plan's stream) unless stated.
 *   - Outputs are overwritten, never accumulated.
 *
 * Errors.  Every function returns a lens_status.  The status of the last
 * failing call on the calling thread and a one-line message are kept
 * (lens_get_last_error, lens_last_error_message).  No function aborts the
 * process or traps on the GPU.
 */
#ifndef GSLENS_H
#define GSLENS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LENS_OK = 0,
    LENS_ERR_INVALID = 1,   /* bad argument (sizes, spin, NULL pointer, ...) */
    LENS_ERR_DOMAIN = 2,    /* a coordinate is not finite or theta is outside [0, pi] */
    LENS_ERR_PRECISION = 3, /* epsilon not reachable at this precision */
    LENS_ERR_NOMEM = 4,     /* device or host allocation failed */
    LENS_ERR_CUDA = 5,      /* a CUDA runtime call failed */
    LENS_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up */
    LENS_ERR_UNSUPPORTED = 7 /* size outside what this build handles (see message) */
} lens_status;

typedef enum { LENS_FP32 = 0, LENS_FP64 = 1 } lens_prec;

/* Plan flags (lens_plan_create's flags argument, OR-ed). */
typedef enum {
    /* Gradient-only spin-s transforms (Sect. 4: a vanishing curl component,
     * C = 0, e.g. the spin-1 deflection field of Sect. 3 or E-only
     * polarisation).  a_lm buffers then hold G alone, [nmaps][1][nalm]:
     * lens_synthesis takes C = 0 and lens_adjoint returns only G.  The
     * Legendre steps accumulate two sums per degree instead of four.
     * Needs spin > 0 (LENS_ERR_INVALID otherwise). */
    LENS_GRAD_ONLY = 1,
    /* Bit-reproducible adjoints.  The two steps that add with atomics (the
     * spreading of Sect. 3's NUFFT type 1 and the adjoint Legendre step) then
     * accumulate in 64-bit fixed point: each term is scaled by a power of two
     * 2^k and rounded to an integer, and integer additions are exact, so the
     * result does not depend on their order.  k is chosen per call from a
     * bound on the sums (spreading: the most points any grid cell receives
     * times the largest |map value|; adjoint Legendre, per order m: the sum of
     * |Re| + |Im| of the ring coefficients times sqrt((2 lmax + 1)/(4 pi)) and
     * the order weight) so that no sum exceeds 2^62; a term loses what lies
     * below 2^-62 of that bound.  Costs a max-reduction over the map, a sum
     * over the ring coefficients and two conversion passes per adjoint; FP32
     * plans hold int64 copies of the grid and of the a_lm sums.  Maps must be
     * finite (a NaN or infinity makes the whole output NaN).  The forward
     * transform has no atomics and is reproducible without this flag. */
    LENS_DETERMINISTIC = 2
} lens_flags;

typedef struct lens_plan_s *lens_plan;

/* Optional overrides for lens_plan_create_ex; zero fields mean "choose". */
typedef struct {
    double sigma;   /* oversampling factor of the NUFFT grid (1.2 .. 2.5) */
    int W;          /* kernel support in grid cells (4 .. 16) */
    double beta;    /* ES kernel shape parameter (FP32 plans: LENS_ERR_INVALID if the
                       polynomial kernel weights, see lens_kernel_poly, miss the kernel by
                       more than 4 max(e^-beta, 1e-7), e.g. W 4 with beta 16) */
    int ntheta;     /* rings of the equiangular grid (>= lmax + 2) */
    int legendre_rpt_fwd;  /* rings per thread of the Legendre synthesis kernel (1 or 2; also 4
                              for FP32 plans with the restarted FP32 recursion; FP64 plans: for
                              the FP64 and the double-float orders) */
    int legendre_rpt_adj;  /* rings per thread of the adjoint Legendre kernel (as above) */
    int legendre_df32_mmin; /* FP64 plans: orders m >= this value use the double-float Legendre
                               recursion (0 = choose, -1 = never) */
    int fft_cluster;        /* CTAs per FFT vector: 0 = choose (1, or a cluster of 2 or 4 when
                               the vector exceeds one CTA's shared memory), 1, 2 or 4 to force */
    int legendre_tables;    /* FP32 plans: 1 = compute the Legendre values once at plan creation
                               and keep them in device memory (about (2/pi) x n_rings/2 x nalm
                               floats, twice that for spin s: 46 / 93 GB at lmax 4096); the
                               Legendre steps then stream them instead of running the
                               recursion.  0 = recursion (default).  LENS_ERR_NOMEM if the
                               tables do not fit. */
    int legendre_restart;   /* Legendre recursion arithmetic (plans without tables):
                               FP32 plans, 0 = choose: epsilon >= 1e-5 runs the recursion in
                               FP32 and resets it every K = 64 degrees (K doubled while the
                               restart values would exceed 20 GB) to values computed at plan
                               creation (FP64 recursion; 8 or 16 bytes per ring, restart and
                               order: 2.3 / 4.5 GB for spin 0 / spin s at lmax 4096); smaller
                               epsilon runs the double-float recursion.
                               FP64 plans, 0 = choose: epsilon >= 5e-11 runs every order in
                               double-float, reset to the FP64 recursion's values every 16
                               degrees for m < 16 g, 64 for m < 128 g and K = 128 above,
                               g = max(1, lmax / 4096) (K doubled above 40 GB; 16 or 32 bytes
                               per ring, restart and order: 2.6 / 5.2 GB at lmax 4096);
                               smaller epsilon runs the low orders in FP64
                               (legendre_df32_mmin).
                               -1 = no restarts (FP32 plans: the double-float recursion; FP64
                               plans: FP64 low orders as for small epsilon).
                               K > 0 = restart every K degrees (a power of two, 8 .. 4096). */
    int point_weights;      /* FP64 plans: 0 = keep the 2W kernel weights of every point when they
                               take at most 48 GB (16 W bytes per point), else evaluate the taps in
                               every call; -1 = always evaluate them per call (no weight table);
                               1 = always keep them (LENS_ERR_NOMEM if they do not fit). */
    int spread_tile_rows;   /* rows of the grid tiles that sort the points and that the spreading
                               accumulates in shared memory (32 columns): 16, 32 or 64 (0 = 32) */
} lens_plan_params;

typedef struct {
    int lmax, mmax, spin, prec;
    int64_t npoints;
    double epsilon;
    int ntheta;         /* equiangular rings, poles included (Sect. 3 "synthesis") */
    int ntheta_fft;     /* 2 ntheta - 2, length of the doubled theta transform */
    int n1, n2;         /* oversampled torus (theta, phi) */
    int W;              /* kernel support */
    double beta, sigma; /* ES kernel exp(beta (sqrt(1 - (2z/W)^2) - 1)), oversampling */
    int rows_kept;      /* torus rows stored (theta in [0, pi] plus kernel halo) */
    int row_pitch;      /* grid row stride in elements */
    size_t workspace_bytes;    /* per-call work buffers */
    size_t plan_bytes;         /* point tables and coefficient tables */
    unsigned flags;            /* lens_flags the plan was created with */
    int alm_ncomp;             /* components of an a_lm buffer: 1 (spin 0, LENS_GRAD_ONLY) or 2 */
    size_t legendre_table_bytes; /* Legendre tables held by the plan (0: recursion) */
    int legendre_restart;        /* recursion restarted every this many degrees (FP32 plans: FP32
                                    recursion, FP64 plans: double-float; 0: no restarts, or tables) */
    size_t restart_bytes;        /* restart values held by the plan */
    int legendre_df32_mmin;      /* FP64 plans: first order run in double-float (mmax + 1: none) */
    int64_t legendre_triples;    /* restarted recursions: (ring pair, l, m) triples from the first
                                    degree at which |lambda| reaches 2^-40 (FP64 plans: 2^-64) on each
                                    ring (0 if not counted) */
    size_t point_weight_bytes;   /* FP64 plans: kernel weights kept per point (0: evaluated per call) */
} lens_plan_info_t;

/*
 * Create a plan for one geometry (Sect. 3: the geometry is reused by many
 * maps, so everything that depends only on it is prepared here).
 *   out        receives the plan.
 *   lmax, mmax band limit (0 <= mmax <= lmax).
 *   spin       0, or s >= 1 (s <= lmax).
 *   npoints    number of points (>= 0).
 *   theta_d, phi_d   device double[npoints] deflected coordinates.
 *   chi_d      device double[npoints] spin phase, or NULL (ignored for spin 0).
 *   epsilon    target relative accuracy (Sect. 4, eps_eff); FP32 plans accept
 *              epsilon >= 2e-6 (FP32 rounding alone leaves ~1.2e-6 at lmax
 *              4096), FP64 plans epsilon >= 1e-13.  FP64 rounding sets a floor
 *              that grows with lmax: epsilon below ~5e-12 is not reached at lmax
 *              4096-5120 (epsilon 1e-12 or 1e-13 gives an adjoint eps_eff of
 *              3.6e-12 .. 4.2e-12 there).  The orders run in double-float
 *              (m >= legendre_df32_mmin, default 64 / 256 for epsilon >= 1e-9 /
 *              >= 5e-11, scaled by (lmax / 4096)^2 above lmax 4096, none below
 *              5e-11) keep the error of the all-FP64 recursion.
 *   prec       LENS_FP32 or LENS_FP64.
 *   flags      0, or LENS_GRAD_ONLY and / or LENS_DETERMINISTIC (lens_flags);
 *              other bits: LENS_ERR_INVALID.
 *   stream     cudaStream_t (NULL = legacy default stream).
 * Synchronises the stream once (coordinate validation).  LENS_ERR_DOMAIN if a
 * coordinate is not finite or theta is outside [0, pi].
 */
int lens_plan_create(lens_plan *out, int lmax, int mmax, int spin, int64_t npoints,
                     const double *theta_d, const double *phi_d, const double *chi_d,
                     double epsilon, int prec, unsigned flags, void *stream);

/* As lens_plan_create, with explicit kernel / grid parameters (NULL = none). */
int lens_plan_create_ex(lens_plan *out, int lmax, int mmax, int spin, int64_t npoints,
                        const double *theta_d, const double *phi_d, const double *chi_d,
                        double epsilon, int prec, unsigned flags, void *stream,
                        const lens_plan_params *params);

int lens_plan_destroy(lens_plan p);
int lens_plan_info(lens_plan p, lens_plan_info_t *info);

/*
 * Forward lensing (Sect. 2 Eq. "forward" / "forwardpol"; Sect. 3 steps
 * synthesis, doubling, FFT, NUFFT).
 *   alm_d  device [nmaps][ncomp][nalm] complex (ncomp = 1 for spin 0, 2 for spin s)
 *   map_d  device [nmaps][ncomp][npoints] real
 * Entries with l < spin are ignored.  Imaginary parts of m = 0 entries are
 * ignored (real fields).
 * FP32 plans with nmaps >= 2 synthesise the Legendre step of four (then two)
 * maps in one pass that shares the recursion among them; the first such call
 * allocates a workspace of 4 x (ring + a_lm) bytes on the plan (outside a
 * stream capture only; inside one, or if the allocation fails, the maps run
 * one by one).  The result equals the per-map result up to FP32 rounding
 * order (identical arithmetic per map).
 */
int lens_synthesis(lens_plan p, const void *alm_d, void *map_d, int nmaps, void *stream);

/* Synchronises `stream` (NULL: the plan's) and reports whether a kernel of
 * an earlier call on this plan gave up a bounded device-side wait (the bulk
 * copies of the Legendre-table kernels wait at most ~2 s): LENS_ERR_TIMEOUT,
 * and the flag is cleared; else LENS_OK. */
int lens_plan_status(lens_plan p, void *stream);

/* Diagnostic: runs one warp that waits, with a ~10 ms limit, on an mbarrier
 * that no copy completes (nothing else is in flight), through the same
 * bounded wait as the Legendre-table kernels.  LENS_OK when the wait gave up
 * and reported it as those kernels do; LENS_ERR_CUDA otherwise. */
int lens_selftest_bounded_wait(void *stream);

/* Turns the grouped multi-map synthesis above on (on != 0, the default) or off
 * for this plan.  Returns LENS_ERR_INVALID for a NULL plan. */
int lens_plan_set_grouping(lens_plan p, int on);

/*
 * Tensor-core Legendre synthesis (no counterpart in the paper, which runs one
 * map at a time on CPUs).  For spin-0 FP32 plans that run the restarted FP32
 * recursion (lens_plan_params.legendre_restart), lens_synthesis with 16 or more
 * maps computes the Legendre step of up to 64 maps at a time as a dense
 * contraction (Legendre values x coefficients per order m) on the tensor cores
 * (tcgen05, TF32 operands split into high and low parts: three products per
 * term, FP32 accumulation), then the Fourier stages and the interpolation per
 * map.  The first such call allocates its workspace (ring coefficients of 64
 * maps and the coefficient tiles: 18 GB at lmax 4096); inside a stream capture,
 * or if the allocation fails, the maps run on the CUDA-core paths instead.
 * on = 0 turns the tensor-core path off for this plan (default on).
 */
int lens_plan_set_tensor_cores(lens_plan p, int on);

/*
 * Adjoint lensing (Sect. 2 Eq. "adjoint" and its spin-s form; Sect. 3 adjoint
 * steps NUFFT type 1, FFT, undoubling, adjoint synthesis).
 *   map_d  device [nmaps][ncomp][npoints] real
 *   alm_d  device [nmaps][ncomp][nalm] complex (written)
 */
int lens_adjoint(lens_plan p, const void *map_d, void *alm_d, int nmaps, void *stream);

/*
 * Gradients for reverse-mode differentiation (no counterpart in the paper;
 * they follow from the exact adjoint of Sect. 2).  For a real loss L and
 * complex a_lm, gradients are written dL/dRe + i dL/dIm.  lens_synthesis
 * counts each m > 0 coefficient for both +m and -m (real fields), so with the
 * order weight w_0 = 1, w_m = 2 (m > 0):
 *   lens_synthesis_vjp: grad_map_d [nmaps][ncomp][npoints] real = dL/dmap of
 *       lens_synthesis's output; writes grad_alm_d [nmaps][ncomp][nalm]
 *       complex = dL/da_lm = w_m * lens_adjoint(grad_map).
 *   lens_adjoint_vjp: grad_alm_d = dL/da_lm of lens_adjoint's output; writes
 *       grad_map_d = dL/dmap = lens_synthesis(grad_alm / w_m).
 * Imaginary parts at m = 0 receive zero gradient (lens_synthesis ignores
 * them and lens_adjoint returns them as zero).  Same layouts, stream
 * semantics and errors as lens_synthesis / lens_adjoint.
 */
int lens_synthesis_vjp(lens_plan p, const void *grad_map_d, void *grad_alm_d, int nmaps, void *stream);
int lens_adjoint_vjp(lens_plan p, const void *grad_alm_d, void *grad_map_d, int nmaps, void *stream);

/*
 * Deflection field (Sect. 3 Eq. "deflect"): alpha_theta + i alpha_phi =
 * spin-1 forward operator of G_LM = sqrt(L(L+1)) phi_LM, C_LM = 0, i.e. the
 * gradient of phi, at the plan's points.
 *   defl      an FP64 spin-1 plan on the undeflected points (chi NULL).
 *   phi_lm_d  device complex double [nalm] (real-field layout of a_lm).
 *   alpha_d   device double [2][npoints]: alpha_theta then alpha_phi; feed
 *             them to lens_pointing for theta', phi', chi.
 * LENS_ERR_INVALID unless defl is FP64 spin 1.  defl may be LENS_GRAD_ONLY
 * (the deflection has no curl component): the same result with half the
 * Legendre accumulation work.
 */
int lens_deflection(lens_plan defl, const void *phi_lm_d, double *alpha_d, void *stream);

/*
 * Coefficients of eth f (lower = 0) or ethbar f (lower = 1) of a spin-s field
 * f, as a spin s+1 (s-1) field in the convention of Eq. "forwardpol",
 * sf = -sum (G + iC) sY (spin 0: f = sum a Y), with eth sY_lm =
 * sqrt((l-s)(l+s+1)) s+1Y_lm and ethbar sY_lm = -sqrt((l+s)(l-s+1)) s-1Y_lm
 * (no counterpart in the paper; used for gradients at deflected points).
 *   alm_in_d   device complex [ncomp][nalm(lmax, mmax)] (ncomp 1 for s = 0).
 *   alm_out_d  device complex [2][nalm] (G', C').  prec: LENS_FP32 / LENS_FP64.
 * ethbar needs s >= 2 (LENS_ERR_UNSUPPORTED otherwise).
 */
int lens_alm_eth(int lmax, int mmax, int spin, int lower, int prec, const void *alm_in_d, void *alm_out_d,
                 void *stream);

/*
 * Gradient of a real loss L(d) of the lensed map d = A(phi) x with respect to
 * the lensing potential phi_LM (no counterpart in the paper; the chain rule
 * through Eq. "deflect", the pointing formula and chi).  Per point, with
 * g = dL/dQ + i dL/dU (dL/dT for spin 0), P the lensed field, a = |alpha|:
 *   dL/dalpha = J Y + K i alpha/a,  Y = -1/2 [conj(g) A + g conj(B)],
 *   K = -s (1 - cos a)/a Im(conj(g) P),
 * J the derivative of the exponential map, A and B the lensed syntheses of
 * eth x and ethbar x (spin 0: B = conj A); then dL/dphi_LM =
 * sqrt(L(L+1)) * w_m * (G part of the spin-1 adjoint of dL/dalpha), w_0 = 1,
 * w_m = 2 (real-field coefficients).
 *   lensed       plan of spin s (0 or >= 2) on the deflected points, with chi.
 *   lensed_up    plan of spin s+1, same points, chi, band limit, precision.
 *   lensed_down  plan of spin s-1 for s >= 2 (NULL for s = 0).
 *   defl         FP64 spin-1 plan on the undeflected points, band limit of phi
 *                (LENS_GRAD_ONLY or not; the three lensed plans must not be).
 *   alpha_d      device double [2][npoints], the deflection the points came from.
 *   x_alm_d      device complex [ncomp][nalm], lensed's precision.
 *   map_d        lensed map A(phi) x, [ncomp][npoints], or NULL (recomputed).
 *   grad_map_d   dL/dd, [ncomp][npoints], lensed's precision.
 *   grad_phi_d   device complex double [nalm of defl] (written).
 * Scratch comes from the stream-ordered allocator and is released before
 * return (stream order).  LENS_ERR_INVALID if the plans do not match,
 * LENS_ERR_UNSUPPORTED for spin 1.
 */
int lens_phi_gradient(lens_plan lensed, lens_plan lensed_up, lens_plan lensed_down, lens_plan defl,
                      const double *alpha_d, const void *x_alm_d, const void *map_d, const void *grad_map_d,
                      void *grad_phi_d, void *stream);

/*
 * Batched execution (no counterpart in the paper): a list of transforms over
 * any mix of plans, recorded once as a CUDA graph and replayed with one
 * launch.  Items of one plan share its workspace and run in the order they
 * were added, on one branch; plans are spread over up to nbranches concurrent
 * branches, largest estimated cost first, so that small transforms run side by
 * side.
 *   lens_batch_create(&b, device)
 *   lens_batch_add(b, plan, op, in_d, out_d, nmaps)   op 0: lens_synthesis
 *       (in = a_lm, out = map), op 1: lens_adjoint (in = map, out = a_lm);
 *       layouts as for those calls.  The pointers are recorded, not copied:
 *       every launch reads and writes the same buffers.
 *   lens_batch_instantiate(b, nbranches)  records the graph (1 <= nbranches
 *       <= 64); no item may be added afterwards.
 *   lens_batch_launch(b, stream)  one cudaGraphLaunch on stream.
 *   lens_batch_info(b, &nitems, &nbranches, &max_branch_seconds)  the
 *       balancing estimate (any pointer may be NULL).
 *   lens_batch_destroy(b)  the plans stay owned by the caller and must
 *       outlive every launch.
 */
typedef struct lens_batch_s *lens_batch;
int lens_batch_create(lens_batch *out, int device);
int lens_batch_add(lens_batch b, lens_plan p, int op, const void *in_d, void *out_d, int nmaps);
int lens_batch_instantiate(lens_batch b, int nbranches);
int lens_batch_launch(lens_batch b, void *stream);
int lens_batch_info(lens_batch b, int *nitems, int *nbranches, double *max_branch_seconds);
int lens_batch_destroy(lens_batch b);

/*
 * Autotuner (no counterpart in the paper, which picks its kernel parameters
 * with a heuristic): builds candidate plans for the given points and times
 * them on the GPU.  Candidates: oversampling sigma in {1.25, 1.5, 1.75, 2.0,
 * 2.25, 2.5} (W follows from epsilon; candidates outside this build's size
 * limits are skipped), then the Legendre rings per thread (forward, adjoint)
 * in {1, 2}^2 at the best sigma.  Each candidate is timed as reps forward +
 * adjoint pairs after one warm-up pair, with CUDA events on stream.
 * Arguments as for lens_plan_create, plus
 *   reps      timed pairs per candidate (>= 1),
 *   best      receives the fastest parameters (pass to lens_plan_create_ex),
 *   best_ms   milliseconds of one forward + adjoint pair with them (or NULL).
 * Allocates one a_lm and one map buffer for the duration of the call.
 */
int lens_autotune(int lmax, int mmax, int spin, int64_t npoints, const double *theta_d, const double *phi_d,
                  const double *chi_d, double epsilon, int prec, void *stream, int reps, lens_plan_params *best,
                  double *best_ms);

/*
 * Intermediate grids for lensed harmonic coefficients (Sect. 4: remap onto a
 * pixelization, then a standard backward SHT; no counterpart in the paper's
 * interface).  A Gauss-Legendre grid: nrings rings at the roots of P_nrings
 * (theta ascending), nphi equispaced longitudes phi_k = 2 pi k / nphi, point
 * index ring * nphi + k.  weight_d (may be NULL) receives w_j 2 pi / nphi, so
 * that the adjoint transform at the grid points applied to weight * map is the
 * backward SHT, exact for band limits below nrings (and nphi > 2 lmax).
 *   theta_d, phi_d, weight_d  device double [nrings * nphi].
 * Synchronises the stream once (the ring table is computed on the host).
 */
int lens_gl_grid(int nrings, int nphi, double *theta_d, double *phi_d, double *weight_d, void *stream);

/*
 * out[c][i] = weight[i] * in[c][i] for c < ncomp, i < n (quadrature weights,
 * magnification weights).  prec selects float or double values; in_d may equal
 * out_d.
 */
int lens_scale_points(int64_t n, int ncomp, int prec, const double *weight_d, const void *in_d, void *out_d,
                      void *stream);

/*
 * Magnification determinant |A| = |d^2 n' / d^2 n| of the remapping (App. B):
 *   |A| = (sin a / a)((1 - kappa)^2 + omega^2 - |gamma|^2)
 *       + (cos a - sin a / a)(1 - kappa - cos(2 beta) gamma_1 - sin(2 beta) gamma_2),
 * kappa + i omega = ethbar(1alpha)/2, gamma = eth(1alpha)/2; for a deflection
 * that is the gradient of phi, omega = 0, kappa is the spin-0 synthesis of
 * l(l+1)/2 phi_lm and gamma the spin-2 synthesis of G = sqrt((l-1)l(l+1)(l+2))/2
 * phi_lm, C = 0 (Eq. "forwardpol" convention).  Inverse lensing (App. B) is
 * then lens_adjoint of T |A| (times quadrature weights).
 *   p0, p2    FP64 plans of spin 0 and 2 on the observed (undeflected) points,
 *             band limit of phi, no chi.
 *   phi_lm_d  complex double [nalm];  alpha_d  double [2][npoints] (lens_deflection);
 *   det_d     double [npoints] (written).
 */
int lens_magnification(lens_plan p0, lens_plan p2, const void *phi_lm_d, const double *alpha_d, double *det_d,
                       void *stream);

/*
 * The same two operations on host buffers: the inputs are copied to the
 * device, the transform runs, the outputs are copied back; returns after the
 * stream has finished.  Pinned host memory gives full copy bandwidth.
 */
int lens_synthesis_host(lens_plan p, const void *alm_h, void *map_h, int nmaps, void *stream);
int lens_adjoint_host(lens_plan p, const void *map_h, void *alm_h, int nmaps, void *stream);

/*
 * As lens_synthesis_host / lens_adjoint_host, but only enqueued on `stream`:
 * they return once the copies and kernels are queued.  The host buffers must
 * stay valid and unmodified until the stream has been synchronised, and should
 * be page-locked (cudaHostAlloc / pinned): copies from pageable memory go
 * through a CUDA-internal bounce buffer and do not overlap other work.  Calls on one plan share
 * its staging buffers, so they must use one stream; plans on different streams
 * overlap their copies with each other's kernels.
 */
int lens_synthesis_host_async(lens_plan p, const void *alm_h, void *map_h, int nmaps, void *stream);
int lens_adjoint_host_async(lens_plan p, const void *map_h, void *alm_h, int nmaps, void *stream);

/*
 * Forward lensing that allocates nothing (no counterpart in the paper).
 * Callers whose device memory belongs to someone else once they are running
 * (a host framework that owns every device allocation, a service with a
 * memory budget fixed at start-up) cannot call cudaMalloc; this entry
 * point computes exactly what lens_synthesis computes for one map, with its
 * scratch (ring coefficients, torus rows, oversampled grid) taken from a
 * fixed 64 MiB array compiled into the library instead of the plan's
 * workspace, and calls no allocating routine.
 *   alm_d  device [ncomp][nalm] complex;  map_d  device [ncomp][npoints] real.
 * LENS_ERR_UNSUPPORTED if the plan needs more scratch than the array holds
 * (the message gives both sizes; use lens_synthesis then).  The array's
 * device address is looked up on the first call made on each device, which
 * should therefore come before any stream capture.  Every call shares the
 * array: calls that overlap on the GPU race.  The call still uses the plan's
 * own prepared-coefficient buffers (plain and, with the restarted FP32
 * recursion, monic) and status flags (allocated when the plan was created),
 * so it must not overlap any other call on the same plan.
 */
int lens_synthesis_static(lens_plan p, const void *alm_d, void *map_d, void *stream);

/*
 * Measured FMA throughput of the current device's CUDA-core pipes (no
 * counterpart in the paper: the denominator of the ALU rooflines that the
 * benchmark reports for the Legendre recursion, which is not a contraction).
 * Runs independent fma chains on every SM for about 0.25 s and returns the
 * rate in flops per second (2 per fused multiply-add) in *flops_per_s.
 *   prec  LENS_FP32 or LENS_FP64.  Synchronises the stream.
 */
int lens_measure_fma_peak(int prec, double *flops_per_s, void *stream);

/*
 * Legendre step alone (Sect. 3 "synthesis" restricted to the theta direction):
 * ring Fourier coefficients on the plan's equiangular rings
 * theta_j = j pi / (ntheta - 1), j = 0..ntheta-1.
 *   ring_d  device complex [ncol][ntheta], ncol = mmax + 1 (spin 0, column m)
 *           or 2 mmax + 1 (spin s, column m + mmax); spin 0 holds
 *           sum_l a_lm lambda_lm(theta_j), spin s holds
 *           -sum_l (G + iC)_lm s lambda_lm(theta_j) (the sign of Eq. "forwardpol").
 */
int lens_ring_synthesis(lens_plan p, const void *alm_d, void *ring_d, void *stream);

/*
 * Doubling and theta transform alone (Sect. 3 "doubling"): the Fourier
 * coefficients in theta of the doubled ring functions, before the kernel
 * deconvolution and the oversampling.
 *   coef_d  device complex [ncol][2 lmax + 1] (ncol as lens_ring_synthesis;
 *           entry k + lmax is c_k, |k| <= lmax), such that the ring function
 *           of lens_ring_synthesis is F(theta) = sum_k c_k e^{i k theta} at
 *           every theta in [0, pi], not only on the rings (the doubled
 *           function is band-limited to |k| <= lmax).
 * LENS_ERR_UNSUPPORTED when the plan's theta vectors need a CTA cluster.
 * Uses the plan's workspace; stream-ordered like lens_synthesis.
 */
int lens_torus_coefficients(lens_plan p, const void *alm_d, void *coef_d, void *stream);

/* Transpose of lens_ring_synthesis: a_lm (spin 0) or G, C (spin s, with the
 * G/C decomposition of Sect. 2) from ring coefficients of the same layout. */
int lens_ring_adjoint(lens_plan p, const void *ring_d, void *alm_d, void *stream);

/*
 * Pointing (Sect. 3, the unlensed-direction formula; Fig. 1 for chi):
 *   n' = cos(a) n + sin(a)/a (a_theta e_theta + a_phi e_phi),  a = |alpha|,
 *   chi = beta - beta' (angle of the geodesic at n minus its angle at n',
 *   both from e_theta towards e_phi), wrapped to (-pi, pi].
 * All arrays device double[n]; chi_out_d may be NULL.  theta' in [0, pi],
 * phi' in [0, 2 pi).
 */
int lens_pointing(int64_t n, const double *theta_d, const double *phi_d,
                  const double *alpha_theta_d, const double *alpha_phi_d,
                  double *theta_out_d, double *phi_out_d, double *chi_out_d, void *stream);

/*
 * Stage timers.  While enabled, every transform records a CUDA event pair
 * around each of its kernel stages on the stream it launches on; the pairs
 * are resolved by lens_profile_read.  Slots (index = stage + 8 * (spin > 0)
 * + 16 * (prec == LENS_FP64)), stage = 0 Legendre synthesis, 1 theta
 * transform (forward), 2 phi transform (forward), 3 interpolation,
 * 4 spreading, 5 phi transform (adjoint), 6 theta transform (adjoint),
 * 7 adjoint Legendre.  Process-wide; not thread-safe with concurrent calls.
 *   lens_profile_enable(1/0)  start / stop recording (recording keeps totals)
 *   lens_profile_read(ms, counts, n)  synchronises the recorded events, adds
 *       their durations into per-slot totals and copies slots [0, n) out
 *       (ms: double[n] total milliseconds, counts: int64[n] launches; either
 *       may be NULL); n <= 32.
 *   lens_profile_reset()  clears totals and pending events.
 */
int lens_profile_enable(int on);
int lens_profile_read(double *ms, int64_t *counts, int n);
int lens_profile_reset(void);

/* Number of a_lm for (lmax, mmax). */
int64_t lens_nalm(int lmax, int mmax);

/* The polynomial kernel weights FP32 plans evaluate (host only, no device work).
 * The NUFFT steps of Sect. 3 weight tap a (0 <= a < W) of a point by the ES kernel
 * phi(x) = exp(beta (sqrt(1 - x^2) - 1)), x = (frac - a) 2 / W, frac = u - ceil(u - W/2) the
 * point's offset in grid cells.  FP32 plans replace phi by a polynomial of degree W + 1 in
 * t = 2 frac - (W - 1) per tap, fitted at plan creation (interpolation at the W + 2
 * Chebyshev points); this call returns those coefficients as the plan stores them:
 * coef[a (W + 2) + k] multiplies t^k, W (W + 2) floats written (caller-owned).
 * LENS_ERR_INVALID for W outside [4, 16], beta <= 0 or coef NULL. */
int lens_kernel_poly(int W, double beta, float *coef);

const char *lens_status_string(int status);
int lens_get_last_error(void);
const char *lens_last_error_message(void);

/* Library version as major * 10000 + minor * 100 + patch. */
int lens_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GSLENS_H */

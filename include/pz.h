/*
 * pz.h -- C ABI of libpz, the GB300 (sm_103a) spectral-synthesis hot path.
 *
 * The calls follow the paper's statement of the problem (arXiv:2607.24141,
 * "The Payne Zero Project I", Sec. 2.1 Eqs. 1-9, Sec. 6 Eq. 10, Sec. 7):
 *
 *   pz_create          one-time window preparation (Sec. 2.2, Table 1 "Window
 *                      preparation"): copies the atmosphere, grid and line list to
 *                      the device, sorts lines by centre, builds per-tile line ranges.
 *   pz_set_corrections calibration corrections of Eq. 10 (Delta log gf,
 *                      Delta log gamma_6) and abundance offsets.
 *   pz_line_opacity    kappa_line(lambda, d), Eqs. 4-5 summed inside each line's
 *                      fixed window (Sec. 2.2 "Line opacity").
 *   pz_flux            chi = kappa_c + kappa_line (Eq. 3), tau by trapezoid on
 *                      column mass, F_lambda and F_lambda,c from F = 2 pi Int S E_2 dtau
 *                      on piecewise-linear S (Eqs. 6-8, sigma_c = 0 so S = B_lambda).
 *   pz_instrument      f_p = {K S(v_r) B(v_b) F}_p / {K S(v_r) B(v_b) F_c}_p (Sec. 7),
 *                      or f = F/F_c at full resolution (Eq. 9 without K).
 *   pz_loss_chi2       L = sum_p w_p (y_p - f_p)^2 and dL/df (objective of Sec. 6).
 *   pz_backward        reverse pass to per-line Delta log gf, Delta log gamma_6 and
 *                      per-element abundance gradients (Sec. 6).
 *   pz_create_batch    many stars in one context (stars are independent, Sec. 9):
 *                      every stage above runs over all stars in the same launches,
 *                      the line kernels as persistent work queues.
 *   pz_calib_step      one captured calibration step over all stars with shared
 *                      corrections (the joint Sun-Arcturus fit of Sec. 6): forward,
 *                      objective, reverse pass and a gradient update in one CUDA
 *                      graph launch.
 *   pz_group_eval      the four-parameter grouped calibration of Sec. 6 (Eq. 10 with
 *                      linked groups q(l)): objective and group gradients in one
 *                      graph launch, for an optimiser such as L-BFGS.
 *
 * Conventions (every call):
 *  - Return value: PZ_OK or an error code; on error pz_last_error() gives a
 *    message (thread-local).  A call that fails validation launches nothing.
 *  - "host" pointers are read during the call only; the library copies them.
 *    "device" pointers are caller-owned device memory (e.g. torch.empty on
 *    cuda), read or written asynchronously on `stream`.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All work of a call is enqueued on that stream; calls do not synchronise
 *    the host except where stated.
 *  - Arrays are C-contiguous.  [n_depth][n_lambda] means depth-major with the
 *    wavelength index contiguous.  Depth index 0 is the top of the atmosphere.
 *  - A context is not thread-safe: calls on one context must be serialised by
 *    the caller (one stream at a time).
 *  - A context holds S >= 1 stars (S = 1 from pz_create).  Every per-star array
 *    gains a leading [S] dimension: kappa_line [S][n_depth][n_lambda], F and F_c
 *    [S][n_lambda], f, y, w and dL/df [S][n_out].  The corrections and the
 *    gradients are per line of the caller's list and shared by the stars: a
 *    gradient is the sum over the stars that hold the line, and the chi-square
 *    objective is the sum over the stars.
 */
#ifndef PZ_H
#define PZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pz_ctx pz_ctx;

typedef enum {
    PZ_OK = 0,
    PZ_EINVAL = 1,    /* invalid argument (nothing launched) */
    PZ_ENOMEM = 2,    /* device or host allocation failed */
    PZ_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    PZ_ETIMEOUT = 4,  /* a bounded device-side wait gave up (batched scheduler) */
    PZ_ESTATE = 5,    /* call order violated (e.g. pz_flux before pz_line_opacity) */
    PZ_ENUMERIC = 6   /* a device-side iterative solve did not converge (results unreliable) */
} pz_status;

typedef enum {
    PZ_FP64 = 0,   /* plain FP64 GPU form: one thread per (lambda, depth), FP64 Voigt */
    PZ_MIXED = 1   /* FP32 Voigt + compensated FP32 accumulation; FP64 tau and flux */
} pz_precision;

/* Atmosphere and synthesis grid (host pointers, FP64, copied by pz_create).
 * Units: m column mass g cm^-2 (strictly increasing with depth), T K,
 * rho g cm^-3, n_e and n_pert cm^-3, pop = n_s/U_s cm^-3 (partition-normalised
 * number density of species s), mass_amu per species, xi_cms microturbulence
 * cm s^-1, kappa_c continuum absorption cm^2 g^-1 (> 0).
 * Grid (Eq. 1): lambda_i = lambda0_nm (1 + 1/R_grid)^i, i = 0..n_lambda-1. */
typedef struct {
    int32_t n_depth;            /* >= 2 */
    int32_t n_species;          /* >= 1 */
    const double *m;            /* [n_depth] */
    const double *T;            /* [n_depth] */
    const double *rho;          /* [n_depth] */
    const double *n_e;          /* [n_depth] */
    const double *n_pert;       /* [n_depth] */
    const double *pop;          /* [n_species][n_depth] */
    const double *mass_amu;     /* [n_species] */
    double xi_cms;
    const double *kappa_c;      /* [n_depth][n_lambda] */
    double lambda0_nm;
    double R_grid;
    int64_t n_lambda;           /* >= 1 */
} pz_atmos;

/* Line list (host pointers, caller order, copied and sorted by pz_create).
 * log_gamma_rad in log10 s^-1; log_gamma4 and log_gamma6 in log10 cm^3 s^-1
 * per perturber (Eq. 5, no temperature scaling).  species in [0, n_species).
 * half_window W: a line deposits at grid points |i - i_l| <= W where
 * i_l = floor(ln(lambda_l/lambda0)/ln(1 + 1/R) + 1/2) (integer centre
 * placement, Sec. 6); lines whose window misses the grid are dropped. */
typedef struct {
    int64_t n_lines;            /* >= 0 */
    const double *lambda_nm;    /* [n_lines] */
    const float *log_gf;        /* [n_lines] */
    const float *E_low_eV;      /* [n_lines] */
    const float *log_gamma_rad; /* [n_lines] */
    const float *log_gamma4;    /* [n_lines] */
    const float *log_gamma6;    /* [n_lines] */
    const int32_t *species;     /* [n_lines] */
    int32_t half_window;        /* W >= 0 */
} pz_linelist;

/* Allocate a context on the current CUDA device and upload everything.
 * Synchronous (returns when the device copies are complete).
 * Errors: PZ_EINVAL (sizes, non-finite or non-positive inputs, unsorted m,
 * species out of range), PZ_ENOMEM, PZ_ECUDA. */
pz_status pz_create(const pz_atmos *atmos, const pz_linelist *lines, pz_precision precision,
                    pz_ctx **out);

/* Free every device and host resource of the context.  NULL is accepted. */
pz_status pz_destroy(pz_ctx *ctx);

/* Calibration corrections of Eq. 10 and abundance offsets, in caller line order.
 * (gf)' = gf 10^dlog_gf[l]; gamma6' = gamma6 10^dlog_gamma6[l];
 * pop'_{s,d} = pop_{s,d} 10^dabund[elem_of_species[s]].
 * Each pointer may be host or device memory (detected) or NULL (= zeros; for
 * dabund NULL also clears the element map).  elem_of_species is a host array
 * [n_species] with values in [0, n_elem).  Device inputs are read on `stream`.
 * Errors: PZ_EINVAL (n_elem < 0, map out of range), PZ_ECUDA. */
pz_status pz_set_corrections(pz_ctx *ctx, const float *dlog_gf, const float *dlog_gamma6,
                             const float *dabund, const int32_t *elem_of_species, int32_t n_elem,
                             void *stream);

/* Continuum-referenced centre test.  The paper's line opacity rejects weak
 * depth-line pairs against the continuum (Sec. 2.2) and applies its line keep test
 * once per atmosphere with a fixed selection fraction (Sec. 3.2).  Here, with
 * eta > 0, the pair (l, d) is kept when the peak of its term at its centre grid
 * point ic (i_l clipped to the grid), bounded with H(a, 0) <= 1, reaches eta times
 * the continuum there:
 *   (1 - e^{-h nu_ic / k T_d}) A_ld >= eta kappa_c(ic, d),
 *   A_ld = (pi e^2/m_e c) gf n/(rho U) e^{-E/kT} / (sqrt(pi) dnu_D)   (Eq. 4),
 * decided once, in FP64 on the device, with the corrections set at the time of
 * this call; the selection is then fixed until the next call (later corrections
 * change the kept terms' values, not which pairs are kept).  Every later line
 * opacity (both forms) and reverse pass sums only the kept pairs.  eta = 0 turns
 * the test off.  kept_pairs (host, may be NULL): the number of kept (line, depth)
 * pairs, over n_lines x n_depth (synchronises `stream` when not NULL).
 * The forward must run again before pz_flux (PZ_ESTATE otherwise).
 * Errors: PZ_EINVAL for a negative or non-finite eta; PZ_ENOMEM; PZ_ECUDA. */
pz_status pz_set_centre_test(pz_ctx *ctx, double eta, int64_t *kept_pairs, void *stream);

/* Line opacity kappa_line(lambda_i, d) = (1 - e^{-h nu_i/kT_d})
 *   sum_{l : |i - i_l| <= W} (pi e^2/m_e c) gf_l (n_{s,d}/(rho_d U_s)) e^{-E_l/kT_d}
 *   H(a_ld, v_ild) / (sqrt(pi) dnu_D,ld)              (Eqs. 4-5)
 * computed into the context's resident buffer.  If kappa_line is not NULL it
 * also receives a copy: device, FP32, [n_depth][n_lambda]. */
pz_status pz_line_opacity(pz_ctx *ctx, float *kappa_line, void *stream);

/* Emergent flux of the total and continuum branches (Eqs. 6-8):
 * tau_0 = chi_0 m_0, tau_{j+1} = tau_j + (chi_j + chi_{j+1})(m_{j+1} - m_j)/2;
 * F = 2 pi [ sum over layers of Int S E_2 dtau ] with S = B_lambda(T) per nm,
 * linear in tau between layers, the first segment extrapolated to tau = 0 and
 * nothing below the bottom layer.  F, Fc: device FP64 [n_lambda] or NULL
 * (the context keeps its own copy).  Requires pz_line_opacity (PZ_ESTATE). */
pz_status pz_flux(pz_ctx *ctx, double *F, double *Fc, void *stream);

/* Instrument stage and normalisation (Sec. 7):
 *   f_p = sum_i K_pi F_i / sum_i K_pi F_c,i
 * with pixel p at observed wavelength pix_lambda_nm[p] sampling rest wavelength
 * lambda_p / (1 + v_r/c); K_pi a Gaussian in ln(lambda) with
 * sigma^2 = (1/(2 sqrt(2 ln 2) R_lsf))^2 + (v_b/c)^2, truncated at 5 sigma,
 * clipped to the grid and normalised over the in-grid taps.  The weights are
 * rebuilt on the device only when (v_r, v_b, R_lsf, pixels) change.
 * n_pix = 0 (pix_lambda_nm NULL): identity instrument, f_i = F_i / F_c,i on
 * the synthesis grid.  f_norm: device FP32 [n_pix] (or [n_lambda]).
 * pix_lambda_nm: host FP64 [n_pix], strictly increasing.
 * Requires pz_flux (PZ_ESTATE).  Errors: PZ_EINVAL (R_lsf <= 0, a pixel with
 * no in-grid tap, more than 4096 taps per pixel). */
pz_status pz_instrument(pz_ctx *ctx, double v_r_kms, double v_b_kms, double R_lsf,
                        const double *pix_lambda_nm, int64_t n_pix, float *f_norm, void *stream);

/* Chi-square objective on the last pz_instrument output f:
 *   L = sum_p w_p (y_p - f_p)^2,  dL/df_p = -2 w_p (y_p - f_p).
 * y, w: device FP32 [n] (w may be NULL = all ones); n must equal the output
 * size of the last pz_instrument.  loss: device FP64 scalar or NULL;
 * dL_df: device FP32 [n] or NULL.  Requires pz_instrument (PZ_ESTATE). */
pz_status pz_loss_chi2(pz_ctx *ctx, const float *y, const float *w, int64_t n, double *loss,
                       float *dL_df, void *stream);

/* Reverse pass (Sec. 6) for dL/df of the last pz_instrument output:
 * instrument adjoint -> dL/dF -> adjoint of the closed-form flux and of the
 * trapezoid tau -> G = dL/dkappa_line(lambda, d) -> per-line windowed
 * reduction with the Voigt term recomputed (never stored):
 *   g_dlog_gf[l]     = ln10 sum_{i in win, d} G stim kappa-term_l
 *   g_dlog_gamma6[l] = ln10 sum_{i in win, d} G stim A_ld (dH/da) a6_ld
 *   g_dabund[e]      = sum over lines of species in element e of g_dlog_gf
 * dL_df: device FP32 [n_out].  Outputs: device FP32 in caller line order
 * ([n_lines], [n_lines], [n_elem]); any may be NULL.  Lines dropped at
 * pz_create get 0.  Requires pz_instrument since the last forward (PZ_ESTATE).
 * Wavelength derivatives are not provided (integer centre placement, Sec. 6). */
pz_status pz_backward(pz_ctx *ctx, const float *dL_df, float *g_dlog_gf, float *g_dlog_gamma6,
                      float *g_dabund, void *stream);

/* ---- batches of stars ------------------------------------------------------ */

/* A context over n_stars independent stars (Sec. 9: stars are independent, so a
 * batch is the same calculation for each).  atmos: host array [n_stars]; every
 * star must share n_depth, n_species and the wavelength grid (lambda0_nm, R_grid,
 * n_lambda); everything else (T, rho, n_e, n_pert, pop, mass_amu, xi, kappa_c)
 * is per star.  lines: the master line list (caller order), shared.  Star k uses
 * the master lines subset_index[subset_offsets[k] .. subset_offsets[k+1]) (host
 * arrays, [n_stars + 1] int64 starting at 0 and non-decreasing, and int32
 * indices in [0, n_lines); a line may appear in any number of stars).
 * subset_offsets NULL: every star uses every line.  Synchronous like pz_create.
 * Errors: PZ_EINVAL (n_stars outside [1, 512], grids differ, a subset index out
 * of range, anything pz_create rejects), PZ_ENOMEM, PZ_ECUDA. */
pz_status pz_create_batch(int32_t n_stars, const pz_atmos *atmos, const pz_linelist *lines,
                          const int64_t *subset_offsets, const int32_t *subset_index,
                          pz_precision precision, pz_ctx **out);

/* Number of stars of the context (0 for NULL). */
int32_t pz_n_stars(const pz_ctx *ctx);

/* Lines of star k kept at creation (windows intersecting the grid); -1 if k is
 * out of range. */
int64_t pz_star_lines(const pz_ctx *ctx, int32_t star);

/* Current corrections in caller line order (after pz_set_corrections and any
 * pz_calib_step updates): dlog_gf, dlog_gamma6 [n_lines] and dabund [n_elem],
 * FP32, host or device memory, each may be NULL.  Synchronises `stream`. */
pz_status pz_get_corrections(pz_ctx *ctx, float *dlog_gf, float *dlog_gamma6, float *dabund,
                             void *stream);

/* One calibration step on the chi-square objective over all stars (Sec. 6,
 * the shared fit of both standards): corrections applied to the line data,
 * pz_line_opacity, pz_flux and the instrument last configured by pz_instrument,
 * L = sum_stars sum_p w (y - f)^2, the reverse pass, and the plain gradient update
 *   dlog_gf -= lr_gf g_dlog_gf, dlog_gamma6 -= lr_g6 g_dlog_gamma6,
 *   dabund -= lr_ab g_dabund,
 * with the gradients taken before the update.  The paper drives its updates
 * with L-BFGS; this call is the device-side step such a driver repeats.
 * y, w: device FP32 [S][n] (w may be NULL), n the instrument output size.
 * loss: device FP64 scalar or NULL.  g_*: device FP32 outputs (caller order) or
 * NULL.  The whole step is captured once in a CUDA graph and replayed by one
 * graph launch on `stream`; it is re-captured when an argument changes (or after
 * pz_set_tiling, pz_instrument with new settings, or a new element count).
 * Requires one earlier pz_instrument call (PZ_ESTATE).  Errors: PZ_EINVAL (n,
 * non-finite learning rate), PZ_ECUDA. */
pz_status pz_calib_step(pz_ctx *ctx, const float *y, const float *w, int64_t n, float lr_gf,
                        float lr_g6, float lr_ab, double *loss, float *g_dlog_gf,
                        float *g_dlog_gamma6, float *g_dabund, void *stream);

/* ---- continuum scattering (Eq. 6) --------------------------------------------- */

/* Continuum scattering in the formal solution.  With sigma_c set, the extinction is
 * chi = kappa_c + sigma_c + kappa_line and the source function is
 *   S = eps B + (1 - eps) J,   eps = (kappa_c + kappa_line) / chi        (Eq. 6),
 * J the mean intensity of the same plane-parallel slab the flux is taken from (S linear
 * in tau between layers, the first segment extrapolated to tau = 0, nothing below the
 * bottom layer).  The paper iterates the scattering term; its fixed point, the solution
 * of (I - diag(1 - eps) Lambda) S = eps B, is computed directly per wavelength in FP64
 * (one CTA per wavelength and star).  The continuum branch uses
 * eps_c = kappa_c / (kappa_c + sigma_c).  sigma_c: host FP64 [S][n_depth][n_lambda],
 * cm^2/g, finite and >= 0, copied; NULL turns scattering off (S = B).  Synchronous.
 * The forward must run again.  The reverse pass (pz_backward, pz_backward4,
 * pz_calib_step, pz_group_eval) follows the scattering source too: the adjoint of the
 * linear system, M^T mu = dL/dF dF/dS, gives dL/deps = mu (B - J) and the dependence of
 * J = Lambda S on the optical depths, and kappa_line reaches eps through
 * eps = 1 - sigma_c/chi.
 * Errors: PZ_EINVAL (negative or non-finite sigma_c, fewer than two layers), PZ_ENOMEM,
 * PZ_ECUDA. */
pz_status pz_set_scattering(pz_ctx *ctx, const double *sigma_c, void *stream);

/* ---- four-parameter grouped calibration (Sec. 6, Eq. 10) --------------------- */

/* Corrections of the other two damping families of Eq. 10: the radiative and Stark
 * coefficients of line l become gamma_rad,l 10^dlog_gamma_rad[l] and
 * gamma_4,l 10^dlog_gamma4[l].  Arrays [n_lines] in caller order, FP32, host or
 * device memory, NULL = zero.  Applied like pz_set_corrections (the forward must
 * run again).  Errors: PZ_ECUDA. */
pz_status pz_set_damping_corrections(pz_ctx *ctx, const float *dlog_gamma_rad,
                                     const float *dlog_gamma4, void *stream);

/* Current radiative and Stark corrections in caller order (after
 * pz_set_damping_corrections or pz_group_eval): [n_lines] FP32, host or device
 * memory, each may be NULL.  Synchronises `stream`.  Errors: PZ_ECUDA. */
pz_status pz_get_damping_corrections(pz_ctx *ctx, float *dlog_gamma_rad, float *dlog_gamma4,
                                     void *stream);

/* Reverse pass to all four per-line gradients of Eq. 10 -- Delta log gf and the
 * three damping families -- and the per-element abundance gradients:
 *   dL/dDelta log gamma_beta,l = ln10 sum_{i in window, d} G stim A_ld (dH/da) a_beta,ld
 * with a_beta the part of the damping parameter a that family beta contributes
 * (radiative gamma_rad, Stark gamma_4 n_e, van der Waals gamma_6 n_pert, each over
 * 4 pi dnu_D).  The line stage runs once per family (the van der Waals pass also
 * gives the gf sums), so it costs three pz_backward line passes.  Outputs as
 * pz_backward (device FP32, caller order, each may be NULL).  Requirements and
 * errors as pz_backward. */
pz_status pz_backward4(pz_ctx *ctx, const float *dL_df, float *g_dlog_gf, float *g_dlog_gamma_rad,
                       float *g_dlog_gamma4, float *g_dlog_gamma6, float *g_dabund, void *stream);

/* Linked correction groups q(l) (Sec. 6: every component of a group shares the
 * group's four corrections).  group_of_line: host int32 [n_lines] in caller order,
 * values in [0, n_groups) or -1 for a line that takes no correction; n_groups in
 * [0, n_lines], 0 removes the groups.  Synchronous; drops captured graphs.
 * Errors: PZ_EINVAL (n_groups or a group id out of range), PZ_ENOMEM, PZ_ECUDA. */
pz_status pz_set_line_groups(pz_ctx *ctx, const int32_t *group_of_line, int64_t n_groups);

/* One objective and gradient evaluation of the grouped calibration over all stars,
 * captured once in a CUDA graph and replayed by one graph launch (re-captured when
 * an argument changes): delta_l = x[.][q(l)] for the four families, line opacity,
 * flux, the instrument last configured by pz_instrument, L = sum w (y - f)^2, the
 * four-family reverse pass and the group sums
 *   g[.][q] = sum over the members l of q of dL/ddelta_l.
 * x: device FP32 [4][n_groups] rows (Delta log gf, Delta log gamma_rad,
 * Delta log gamma_4, Delta log gamma_6); g: device FP32 [4][n_groups], same rows,
 * or NULL; y, w: device FP32 [S][n] (w may be NULL); loss: device FP64 scalar or
 * NULL.  The corrections of the context are left at the expanded x; abundance
 * offsets stay as last set.  An optimiser (the paper uses L-BFGS) proposes x
 * between calls.  Requires pz_set_line_groups with n_groups > 0 and one earlier
 * pz_instrument (PZ_ESTATE).  Errors: PZ_EINVAL (NULL y or x, n), PZ_ECUDA. */
pz_status pz_group_eval(pz_ctx *ctx, const float *y, const float *w, int64_t n, const float *x,
                        double *loss, float *g, void *stream);

/* Greedy strength-ordered line grouping (Sec. 6), host only: lines are taken from
 * the largest strength down (equal strengths in index order); a line not yet
 * grouped opens the next group (ids from 0 in opening order) and takes every line
 * not yet grouped of the same species (ion stage included) with
 * |E_low,m - E_low,seed| <= dE_eV and |lambda_m - lambda_seed| <= dlam_nm (the
 * paper uses 2.0 cm^-1 and 0.035 nm).  Differences are taken in FP64 (E_low read
 * from FP32).  Inputs host [n]: lambda_nm FP64, E_low_eV FP32, species int32,
 * strength FP32 (any monotone strength proxy, e.g. log gf - theta E_low);
 * group_of_line host int32 [n] output; *n_groups the number of groups.
 * Errors: PZ_EINVAL (NULL pointer, negative or non-finite tolerance, non-finite
 * line data). */
pz_status pz_build_line_groups(int64_t n, const double *lambda_nm, const float *E_low_eV,
                               const int32_t *species, const float *strength, double dE_eV,
                               double dlam_nm, int32_t *group_of_line, int64_t *n_groups);

/* ---- introspection -------------------------------------------------------- */

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *pz_last_error(void);

/* Number of (line, lambda, depth) Voigt evaluations one pz_line_opacity performs
 * (lines in the grid x clipped window points x n_depth). */
int64_t pz_eval_count(const pz_ctx *ctx);

/* Number of kernel launches issued by the most recent pz_* call on this context. */
int32_t pz_last_launch_count(const pz_ctx *ctx);

/* Kernel tiling of the mixed-precision line kernels: lambda points per thread
 * (2 or 4), depths per warp, warps per CTA (1-4), lines per shared-memory chunk
 * (forward and backward) and the minimum number of resident CTAs per SM the
 * kernels are compiled for (a register budget).  Values <= 0 keep the current
 * setting; the next launch uses the new tiling.  Supported (lambda, depth,
 * CTAs) triples: (4,6,1-6) (4,8,1-3) (4,12,1-2) (2,6,4) (2,6,6) (2,8,2-5) (2,12,1-3);
 * depths per warp are even (the far-wing kernels evaluate depth pairs).
 * Errors: PZ_EINVAL for an unsupported combination or a chunk that does not fit
 * in shared memory. */
pz_status pz_set_tiling(pz_ctx *ctx, int32_t lambda_per_thread, int32_t depth_per_warp,
                        int32_t warps_per_cta, int32_t lines_per_chunk, int32_t ctas_per_sm);

/* Autotuner of the mixed-precision line kernels.  The paper sizes its line
 * chunks per device by hand (2,000 / 4,000 / 8,000 lines on V100 / A100 / H100,
 * Sec. 2.3); here the tiling is measured instead.  Starting from the current
 * tiling, a coordinate search times, on this context's own stars, line lists and
 * atmospheres: every compiled (lambda points per thread, depths per warp, CTAs
 * per SM) triple, then warps per CTA 1-4, then lines per chunk 16-128, and runs
 * these three phases twice.  Each
 * candidate gets one untimed pass, then `reps` forward line launches (far wing +
 * near core) and, if with_backward != 0, `reps` backward line launches, timed
 * with CUDA events on `stream`.  The tiling with the smallest forward (+ backward)
 * time per pass is kept.
 *   best:    host int32[6] or NULL: (lambda points per thread, depths per warp,
 *            warps per CTA, lines per chunk, CTAs per SM, candidates timed);
 *   best_ms: host double[2] or NULL: forward and backward line-kernel ms per
 *            pass of the kept tiling (backward 0 without with_backward).
 * The call synchronises `stream`.  It overwrites the line-opacity buffers (and
 * the backward's line accumulators), so pz_line_opacity must run again before
 * pz_flux (PZ_ESTATE otherwise).  The backward timing uses G of the last
 * pz_backward, or zeros if none ran (the kernels' cost does not depend on G).
 * Cost: about 50 candidates x (1 + reps) passes.
 * Errors: PZ_EINVAL for the plain FP64 form (it has no tiling) or reps outside
 * [1, 100]; PZ_ECUDA if a launch fails (the context keeps the last tiling that
 * was applied). */
pz_status pz_autotune(pz_ctx *ctx, int32_t with_backward, int32_t reps, int32_t *best, double *best_ms,
                      void *stream);

/* Device status word of the context, set by kernels that cannot finish normally
 * without a host round trip:
 *   bit 0: a bounded device-side wait gave up (outputs incomplete);
 *   bit 1: the iterative refinement of the scattering source (Eq. 6, pz_set_scattering)
 *          stopped with its last correction above 1e-9 of the solution (stalled,
 *          growing, or out of rounds), in the forward or the reverse pass: the flux or
 *          the gradients of that wavelength rest on an unconverged solve.  Refinement
 *          ends once a correction below 1e-12 of the solution has been applied (what
 *          remains is that times the contraction per round), or where the correction
 *          stops halving per round.
 * This call synchronises `stream`, stores the status word in *flags (host, may be
 * NULL), clears it, and returns PZ_ETIMEOUT if bit 0 was set, PZ_ENUMERIC if bit 1
 * was set, else PZ_OK. */
pz_status pz_sync_status(pz_ctx *ctx, void *stream, int32_t *flags);

/* ---- profiling ------------------------------------------------------------- */

/* Kernel families timed by the built-in CUDA-event profiler. */
typedef enum {
    PZ_K_LINE_FWD = 0,     /* windowed Voigt sum (mixed or FP64 form; mixed: far-wing + near-core) */
    PZ_K_LINE_BWD = 1,     /* per-line windowed gradient reduction (mixed: far-wing + near-core) */
    PZ_K_FLUX = 2,         /* tau + closed-form flux, both branches */
    PZ_K_RT_ADJOINT = 3,   /* adjoint of flux and tau */
    PZ_K_INSTRUMENT = 4,   /* weight build + apply (or identity) */
    PZ_K_INST_ADJOINT = 5, /* transpose of the instrument */
    PZ_K_LOSS = 6,         /* chi-square and its seed */
    PZ_K_OTHER = 7,        /* corrections, finalisation, copies */
    PZ_K_STEP = 8,         /* a whole pz_calib_step graph launch */
    PZ_K_NEAR_FWD = 9,     /* the near-core part of PZ_K_LINE_FWD (mixed form; also counted there) */
    PZ_K_NEAR_BWD = 10,    /* the near-core part of PZ_K_LINE_BWD (mixed form; also counted there) */
    PZ_NK = 11
} pz_kernel_id;

/* enable != 0: every kernel launch of this context is bracketed by CUDA events
 * recorded on the launching stream.  Disabling (or re-enabling) clears the
 * accumulated times.  Host-side overhead: two event records per launch. */
pz_status pz_set_profiling(pz_ctx *ctx, int32_t enable);

/* Accumulated device time (ms) and launch count per kernel family since
 * profiling was enabled, for the first nk families (ms, counts: host arrays
 * [nk]).  Synchronises on the recorded events. */
pz_status pz_kernel_times(pz_ctx *ctx, double *ms, int64_t *counts, int32_t nk);

/* ---- device memory ------------------------------------------------------------ */

/* The library's device buffers (context tables, work queues, outputs it keeps, scratch)
 * come from cudaMalloc and go back through cudaFree unless the caller installs its own
 * allocator here, e.g. a framework that accounts for every byte of device memory in
 * its own pool or caps it.  Not a step of the paper's method: host-side plumbing.
 *   alloc(bytes, user) returns device memory of the current device, aligned to 256
 *     bytes (as cudaMalloc), or NULL on failure; the call that needed it then returns
 *     PZ_ENOMEM and frees what it had taken (misaligned memory is handed back to
 *     free_fn and treated as a failure);
 *   free_fn(ptr, user) releases memory alloc returned;
 *   user is passed through unchanged.
 * Both functions, or neither (NULL, NULL: back to cudaMalloc / cudaFree).  The
 * allocator is process-wide and may change only while no context exists (PZ_ESTATE
 * otherwise), so every buffer is freed by the allocator that made it.  Errors:
 * PZ_EINVAL (exactly one function NULL), PZ_ESTATE. */
typedef void *(*pz_alloc_fn)(size_t bytes, void *user);
typedef void (*pz_free_fn)(void *ptr, void *user);
pz_status pz_set_allocator(pz_alloc_fn alloc, pz_free_fn free_fn, void *user);

/* ---- allocation-free variant -------------------------------------------------- */

/* Per-element abundance gradient from per-line oscillator-strength gradients,
 *   g_dabund[e] = sum over lines l with elem_of_species[species[l]] == e of g_dlog_gf[l],
 * without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc where they need the
 * reduction -- a framework that owns all device memory through its own pool (an
 * outside allocation escapes its accounting or fails under its memory cap), or a
 * tight optimiser loop that cannot accept cudaMalloc's implicit synchronisation.
 * Its FP64 accumulators are a fixed array inside the library (4096 entries,
 * 32 KiB, held on every GPU that loads the library until the process exits).
 * All pointers are device memory: g_dlog_gf [n_lines] FP32 and species [n_lines]
 * int32 (caller line order, e.g. the pz_backward output and the list's
 * species), elem_of_species [n_species] int32, g_dabund [n_elem] FP32 output.
 * Lines whose species or element is out of range are skipped.
 * The first call on each device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call clears and reuses the same array, so calls that overlap
 * on the GPU (unordered streams) race and give wrong sums.
 * Errors: PZ_EINVAL (n_elem outside [1, 4096], NULL pointer), PZ_ECUDA. */
pz_status pz_abundance_grad_noalloc(const float *g_dlog_gf, const int32_t *species,
                                    const int32_t *elem_of_species, int64_t n_lines, int32_t n_species,
                                    int32_t n_elem, float *g_dabund, void *stream);

/* ---- device-function probes (same device code as the hot path) ------------- */

/* FP32 Voigt H(a,v) and dH/da exactly as the mixed-precision kernels evaluate
 * them, for n device-resident (a, v) pairs.  a, v, H: device FP32 [n]; dHda
 * device FP32 [n] or NULL. */
pz_status pz_probe_voigt(const float *a, const float *v, int64_t n, float *H, float *dHda,
                         void *stream);

/* FP64 exponential integrals exactly as the transfer kernels evaluate them.
 * x: device FP64 [n] (x >= 0); out: device FP64 [5][n]: rows 0-2 E_2, E_3, E_4
 * of the flux kernels, rows 3-4 E_2, E_3 of the scattering kernels' layer-pair
 * table (its own Taylor table of E_3; zero above x = 40). */
pz_status pz_probe_expn(const double *x, int64_t n, double *out, void *stream);

/* Measured throughput of the two arithmetic pipes the line kernels are bound by,
 * for the roofline denominators of an ALU-bound path (the paper reports wall
 * times only; Sec. 2.3 notes its line kernels use no tensor cores).
 *   pipe 0: FP32 FMA issued as packed f32x2 fma, counted as 2 FP32 operations
 *           per lane per instruction;
 *   pipe 1: MUFU reciprocal (rcp.approx.ftz.f32 of x + 1, so that the chain cannot
 *           be simplified), 1 operation per lane;
 *   pipe 2: FP64 FMA, 1 operation per lane (the denominator of the FP64 transfer
 *           stage and the scattering solve).
 * 8 CTAs x 256 threads per SM each run 8 independent dependency chains for
 * `iters` rounds; one warm-up launch, then one launch timed with CUDA events on
 * `stream`.  *ops_per_s (host) receives operations per second over the device.
 * Allocates and frees a small device buffer; synchronises `stream`.
 * Errors: PZ_EINVAL for pipe outside {0, 1, 2}, iters outside [1, 2^20] or a NULL
 * ops_per_s. */
pz_status pz_probe_pipe(int32_t pipe, int32_t iters, double *ops_per_s, void *stream);

/* The bounded wait of the far-wing kernels, on a barrier phase that nothing
 * completes: one CTA waits limit_ns (host, in [1, 1e9]) nanoseconds, gives up and
 * sets bit 0 of a status word exactly as the line kernels do; *flags (host)
 * receives that word.  Exercises the failure path without a fault or a hang.
 * Synchronises `stream`; allocates and frees one device word. */
pz_status pz_probe_wait(int64_t limit_ns, int32_t *flags, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PZ_H */

/*
 * pz_oracle.c -- plain FP64 CPU oracle for the synthesis hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the two meet only in the
 * seeded input arrays.
 *
 * Every routine is the plain definition written out in double precision, in
 * the order the paper states it (arXiv:2607.24141, "The Payne Zero Project I"):
 *
 *   grid            Sec. 2.1, Eq. 1        lambda_i = lambda_0 (1 + 1/R)^i
 *   line opacity    Sec. 2.1, Eqs. 4-5     LTE strength x Voigt profile,
 *                                           phi = H(a,v) / (sqrt(pi) dnu_D)
 *   extinction      Sec. 2.1, Eq. 3        chi = kappa_c + sum_l kappa_l (sigma_c = 0)
 *   optical depth   Sec. 2.1 (dtau = chi dm), trapezoid on column mass
 *   source          Sec. 2.1, Eq. 6        eps = 1  =>  S = B_lambda(T)
 *   flux            Sec. 2.1, Eqs. 7-8     F = 2 pi Int S E_2 dtau, closed form
 *                                           on piecewise-linear S
 *   instrument      Sec. 7 (f_p equation) and Eq. 9: shift + broaden + LSF +
 *                                           sampling, applied to F and F_c
 *                                           before the ratio
 *   adjoint         Sec. 6: reverse pass from the pixel loss to per-line
 *                   Delta log gf, Delta log gamma_6 and abundances (Eq. 10)
 *
 * Where the paper is silent (units, window rule, boundary treatment) the
 * reading taken is stated where it is used below.
 *
 * Voigt function: H(a,v) = Re w(v + i a), w the Faddeeva function.
 *   |z| <  7 : H, L = Im w and dH/da from the Fourier representation
 *              H + iL = pi^-1/2 Int_0^inf exp(-a t - t^2/4) exp(i v t) dt,
 *              by composite Gauss-Legendre quadrature (12 panels x 16 nodes
 *              on [0, 12.5]; the integrand there is below 1e-16 of its peak);
 *              for H the a = 0 term, pi^-1/2 Int exp(-t^2/4) cos(v t) dt =
 *              exp(-v^2), is taken in closed form and only the rest is summed.
 *   |z| >= 7 : the Laplace continued fraction
 *              w(z) = (i/sqrt(pi)) / (z - (1/2)/(z - (2/2)/(z - (3/2)/(z - ...)))),
 *              evaluated bottom-up, and dH/da = 2 (v L + a H) - 2/sqrt(pi)
 *              (from w' = -2 z w + 2i/sqrt(pi)).
 * Exponential integrals E_n: the power series (Abramowitz & Stegun 5.1.12)
 * for x <= 1 and the modified-Lentz continued fraction for x > 1.
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- constants: CODATA 2018, cgs -------------------------------------- */
#define O_H      6.62607015e-27      /* erg s */
#define O_KB     1.380649e-16        /* erg K^-1 */
#define O_C      2.99792458e10       /* cm s^-1 */
#define O_E      4.80320471e-10      /* esu */
#define O_ME     9.1093837015e-28    /* g */
#define O_EV     1.602176634e-12     /* erg */
#define O_AMU    1.66053906660e-24   /* g */
#define O_PI     3.14159265358979323846
#define O_SQRTPI 1.77245385090551602730
#define O_LN10   2.30258509299404568402
#define O_EULER  0.57721566490153286061

/* ======================================================================= */
/* Gauss-Legendre nodes by Newton iteration on P_n (plain textbook method). */
/* ======================================================================= */
#define GL_N 16
#define GL_PANELS 12
#define GL_TMAX 12.5
static double gl_x[GL_N], gl_w[GL_N];
static double fq_t[GL_N * GL_PANELS], fq_w[GL_N * GL_PANELS], fq_g[GL_N * GL_PANELS];

static void gl_init(void) {
    int n = GL_N;
    for (int i = 0; i < n; ++i) {
        double x = cos(O_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        double dp = n * (x * p1 - p0) / (x * x - 1.0);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    double h = GL_TMAX / GL_PANELS;
    for (int p = 0; p < GL_PANELS; ++p)
        for (int i = 0; i < n; ++i) {
            double t = p * h + 0.5 * h * (gl_x[i] + 1.0);
            fq_t[p * n + i] = t;
            fq_w[p * n + i] = 0.5 * h * gl_w[i];
            fq_g[p * n + i] = exp(-0.25 * t * t);
        }
}

__attribute__((constructor)) static void oracle_init(void) { gl_init(); }

/* ======================================================================= */
/* Voigt function H(a,v), L = Im w, dH/da                                   */
/* ======================================================================= */
void pzo_voigt(double a, double v, double *H, double *L, double *dHda) {
    double x = fabs(v);
    double sgn = v < 0.0 ? -1.0 : 1.0;
    if (x * x + a * a < 49.0) {
        /* The a = 0 part of the real integral is exp(-v^2) in closed form; only
         * the remainder, with (exp(-a t) - 1) in place of exp(-a t), goes through
         * the quadrature.  Its terms are O(a), so a small H near |z| = 7 is no
         * longer the difference of O(1) terms. */
        double sh = 0.0, sl = 0.0, sd = 0.0;
        for (int k = 0; k < GL_N * GL_PANELS; ++k) {
            double t = fq_t[k];
            double g = fq_w[k] * fq_g[k];
            double e = g * exp(-a * t);
            double s, c;
            sincos(x * t, &s, &c);
            sh += g * expm1(-a * t) * c;
            sl += e * s;
            sd -= t * e * c;
        }
        *H = exp(-x * x) + sh / O_SQRTPI;
        if (L) *L = sgn * sl / O_SQRTPI;
        if (dHda) *dHda = sd / O_SQRTPI;
        return;
    }
    /* bottom-up continued fraction in real arithmetic: r <- (k/2) / (z - r) */
    double r2 = x * x + a * a;
    int depth = r2 < 100.0 ? 24 : (r2 < 900.0 ? 12 : (r2 < 1e4 ? 8 : 6));
    double rr = 0.0, ri = 0.0;
    for (int k = depth; k >= 0; --k) {
        double dr = x - rr, di = a - ri;
        double q = (k > 0 ? 0.5 * k : 1.0) / (dr * dr + di * di);
        rr = q * dr;
        ri = -q * di;
    }
    /* after the k = 0 step, (rr, ri) = 1/(z - r); w = (i/sqrt(pi)) (rr + i ri) */
    double complex w = (-ri + I * rr) / O_SQRTPI;
    *H = creal(w);
    if (L) *L = sgn * cimag(w);
    if (dHda) *dHda = 2.0 * (x * cimag(w) + a * creal(w)) - 2.0 / O_SQRTPI;
}

/* ======================================================================= */
/* Exponential integral E_n(x), n >= 0, x >= 0                              */
/* ======================================================================= */
double pzo_expn(int n, double x) {
    if (n == 0) return exp(-x) / x;
    if (x == 0.0) return n > 1 ? 1.0 / (n - 1) : INFINITY;
    if (x > 1.0) {
        /* modified Lentz evaluation of
           E_n(x) = e^-x ( 1/(x+n-) 1*n/(x+n+2-) 2(n+1)/(x+n+4-) ... )            */
        const double tiny = 1e-300;
        double b = x + n, c = 1.0 / tiny, d = 1.0 / b, h = d;
        for (int i = 1; i < 100000; ++i) {
            double an = -(double)i * (n - 1 + i);
            b += 2.0;
            d = 1.0 / (an * d + b);
            c = b + an / c;
            double del = c * d;
            h *= del;
            if (fabs(del - 1.0) < 1e-16) break;
        }
        return h * exp(-x);
    }
    /* A&S 5.1.12: E_n(x) = (-x)^{n-1}/(n-1)! [-ln x + psi(n)]
                           - sum_{m>=0, m != n-1} (-x)^m / ((m-n+1) m!)        */
    double psi = -O_EULER;
    for (int k = 1; k <= n - 1; ++k) psi += 1.0 / k;
    double sum = 0.0, term = 1.0;  /* term = (-x)^m / m! */
    double lead = 0.0;
    for (int m = 0; m < 200; ++m) {
        if (m > 0) term *= -x / m;
        if (m == n - 1) {
            lead = term * (-log(x) + psi);
        } else {
            double t = term / (m - n + 1);
            sum -= t;
            if (m > n && fabs(t) < 1e-18 * fabs(sum)) break;
        }
    }
    return lead + sum;
}

/* ======================================================================= */
/* Problem description (mirrors the ctypes structure in oracle.py)          */
/* ======================================================================= */
typedef struct {
    int32_t n_depth, n_species;
    const double *m, *T, *rho, *n_e, *n_pert, *pop, *mass_amu;
    double xi_cms;
    const double *kappa_c;          /* [n_depth][n_lambda] */
    double lambda0_nm, R_grid;
    int64_t n_lambda;
    int64_t n_lines;
    const double *lambda_nm;
    const float *log_gf, *E_low_eV, *log_gamma_rad, *log_gamma4, *log_gamma6;
    const int32_t *species;
    int32_t half_window;
    /* optional calibration corrections (Eq. 10); NULL means zero */
    const double *dlog_gf, *dlog_gamma6;   /* [n_lines] */
    const double *dabund;                  /* [n_elem] */
    const int32_t *elem_of_species;        /* [n_species] */
    /* continuum-referenced centre test: selection fraction eta (0 = every pair kept) */
    double centre_eta;
    /* the other two damping families of Eq. 10 (radiative, Stark); NULL means zero */
    const double *dlog_gamma_rad, *dlog_gamma4;   /* [n_lines] */
    /* continuum scattering coefficient sigma_c [n_depth][n_lambda] cm^2/g; NULL: none (S = B) */
    const double *sigma_c;
} pzo_problem;

/* Eq. 1 */
static double grid_lambda_cm(const pzo_problem *P, int64_t i) {
    return P->lambda0_nm * 1e-7 * exp((double)i * log1p(1.0 / P->R_grid));
}

/* fractional centre index x_l and integer placement i_l = floor(x_l + 1/2) */
static double centre_x(const pzo_problem *P, int64_t l) {
    return log(P->lambda_nm[l] / P->lambda0_nm) / log1p(1.0 / P->R_grid);
}

/* Planck function per nanometre, B_lambda(T) = 2hc^2 lambda^-5 / (e^{hc/lambda kT} - 1) x 1e-7 */
static double planck_nm(double lambda_cm, double T) {
    double x = O_H * O_C / (lambda_cm * O_KB * T);
    return 2.0 * O_H * O_C * O_C / pow(lambda_cm, 5.0) / expm1(x) * 1e-7;
}

/* Per (line, depth) quantities of Eqs. 4-5 and the line term at one lambda. */
typedef struct {
    double A;        /* (pi e^2/m_e c) gf n/(rho U) e^{-E/kT} / (sqrt(pi) dnu_D) */
    double a;        /* damping parameter */
    double a6;       /* van der Waals part of a (for d a / d Delta log gamma_6 = ln10 a6) */
    double arad;     /* radiative part of a (d a / d Delta log gamma_rad = ln10 arad) */
    double a4;       /* Stark part of a (d a / d Delta log gamma_4 = ln10 a4) */
    double dvD;      /* Doppler velocity width, cm/s */
} line_depth;

static line_depth line_at_depth(const pzo_problem *P, int64_t l, int d) {
    line_depth q;
    int s = P->species[l];
    double T = P->T[d];
    double lam_cm = P->lambda_nm[l] * 1e-7;
    double dvD = sqrt(2.0 * O_KB * T / (P->mass_amu[s] * O_AMU) + P->xi_cms * P->xi_cms);
    double dnuD = dvD / lam_cm;                           /* nu_l dv_D / c */
    double dgf = P->dlog_gf ? P->dlog_gf[l] : 0.0;
    double dg6 = P->dlog_gamma6 ? P->dlog_gamma6[l] : 0.0;
    double dab = (P->dabund && P->elem_of_species) ? P->dabund[P->elem_of_species[s]] : 0.0;
    double gf = pow(10.0, (double)P->log_gf[l] + dgf);
    double pop = P->pop[(int64_t)s * P->n_depth + d] * pow(10.0, dab);
    double boltz = exp(-(double)P->E_low_eV[l] * O_EV / (O_KB * T));
    double pie2mc = O_PI * O_E * O_E / (O_ME * O_C);
    q.A = pie2mc * gf * (pop / P->rho[d]) * boltz / (O_SQRTPI * dnuD);
    double drad = P->dlog_gamma_rad ? P->dlog_gamma_rad[l] : 0.0;
    double dg4 = P->dlog_gamma4 ? P->dlog_gamma4[l] : 0.0;
    double g_rad = pow(10.0, (double)P->log_gamma_rad[l] + drad);
    double g4 = pow(10.0, (double)P->log_gamma4[l] + dg4);
    double g6 = pow(10.0, (double)P->log_gamma6[l] + dg6);
    q.a = (g_rad + g4 * P->n_e[d] + g6 * P->n_pert[d]) / (4.0 * O_PI * dnuD);
    q.a6 = g6 * P->n_pert[d] / (4.0 * O_PI * dnuD);
    q.arad = g_rad / (4.0 * O_PI * dnuD);
    q.a4 = g4 * P->n_e[d] / (4.0 * O_PI * dnuD);
    q.dvD = dvD;
    return q;
}

/* 1 - exp(-h nu / kT) at the sample frequency (Eq. 4, factored out of the sum) */
static double stim_emission(const pzo_problem *P, int64_t i, int d) {
    return -expm1(-O_H * O_C / (grid_lambda_cm(P, i) * O_KB * P->T[d]));
}

/* Continuum-referenced centre test (Sec. 2.2: weak depth-line pairs are rejected against
 * the continuum; the threshold form follows the selection fraction eta of Sec. 3.2).
 * Reading: the pair (l, d) is kept when the peak of its term at its centre grid point,
 * bounded with H(a, 0) <= 1, reaches eta times the continuum there:
 *   (1 - exp(-h nu_ic / k T_d)) A_ld >= eta kappa_c(ic, d),  ic = i_l clipped to the grid.
 * eta = 0 keeps every pair. */
static int centre_keep(const pzo_problem *P, int64_t il, int d, double A) {
    if (!(P->centre_eta > 0.0)) return 1;
    int64_t ic = il < 0 ? 0 : (il > P->n_lambda - 1 ? P->n_lambda - 1 : il);
    double peak = stim_emission(P, ic, d) * A;
    return peak >= P->centre_eta * P->kappa_c[(int64_t)d * P->n_lambda + ic];
}

/* kappa_line(i, d) for the requested columns; out[d * n_cols + c].
 * Sum over every line whose window |i - i_l| <= W contains column i
 * (window clipped to the grid), over the pairs the centre test keeps. */
void pzo_kappa_line(const pzo_problem *P, int64_t n_cols, const int64_t *cols, double *out) {
    int nd = P->n_depth;
    int64_t nl = P->n_lines;
    int W = P->half_window;
    int64_t *il = (int64_t *)malloc(sizeof(int64_t) * (nl > 0 ? nl : 1));
    double *xl = (double *)malloc(sizeof(double) * (nl > 0 ? nl : 1));
    for (int64_t l = 0; l < nl; ++l) {
        xl[l] = centre_x(P, l);
        il[l] = (int64_t)floor(xl[l] + 0.5);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < n_cols; ++c) {
        int64_t i = cols[c];
        double lam_i = grid_lambda_cm(P, i);
        for (int d = 0; d < nd; ++d) out[(int64_t)d * n_cols + c] = 0.0;
        for (int64_t l = 0; l < nl; ++l) {
            int64_t di = i - il[l];
            if (di < -W || di > W) continue;
            double lam_l = P->lambda_nm[l] * 1e-7;
            for (int d = 0; d < nd; ++d) {
                line_depth q = line_at_depth(P, l, d);
                if (!centre_keep(P, il[l], d, q.A)) continue;
                double v = (lam_l / lam_i - 1.0) * O_C / q.dvD;   /* (nu - nu_l)/dnu_D */
                double H;
                pzo_voigt(q.a, v, &H, NULL, NULL);
                out[(int64_t)d * n_cols + c] += q.A * H;
            }
        }
        for (int d = 0; d < nd; ++d) out[(int64_t)d * n_cols + c] *= stim_emission(P, i, d);
    }
    free(il);
    free(xl);
}

/* ---- formal solution ----------------------------------------------------- */

/* Int_{ta}^{tb} S E_2 dtau for S linear from Sa to Sb:
 *   Sa (E3(ta) - E3(tb)) + s (E4(ta) - E4(tb) - (tb - ta) E3(tb)),  s = (Sb-Sa)/(tb-ta) */
static double interval_integral(double ta, double tb, double Sa, double Sb) {
    double s = (Sb - Sa) / (tb - ta);
    double e3a = pzo_expn(3, ta), e3b = pzo_expn(3, tb);
    double e4a = pzo_expn(4, ta), e4b = pzo_expn(4, tb);
    return Sa * (e3a - e3b) + s * (e4a - e4b - (tb - ta) * e3b);
}

/* tau by the trapezoid on column mass, tau_0 = chi_0 m_0 (constant opacity above layer 0) */
static void optical_depth(int nd, const double *m, const double *chi, double *tau) {
    tau[0] = chi[0] * m[0];
    for (int d = 0; d + 1 < nd; ++d) tau[d + 1] = tau[d] + 0.5 * (chi[d] + chi[d + 1]) * (m[d + 1] - m[d]);
}

/* F_lambda = 2 pi Int_0^{tau_max} S E_2 dtau; S linear in tau between layers, the first
 * segment extrapolated linearly to tau = 0, nothing below the bottom layer. */
static double flux_from(int nd, const double *tau, const double *S) {
    double s0 = (S[1] - S[0]) / (tau[1] - tau[0]);
    double S_top = S[0] - s0 * tau[0];
    double F = interval_integral(0.0, tau[0], S_top, S[0]);
    for (int d = 0; d + 1 < nd; ++d) F += interval_integral(tau[d], tau[d + 1], S[d], S[d + 1]);
    return 2.0 * O_PI * F;
}

/* ---- scattering source function (Eq. 6 with the transfer equation of Sec. 2.3) ----
 * S = eps B + (1 - eps) J, eps = (kappa_c + sum kappa_l)/chi, chi = kappa_c + sigma_c + sum kappa_l,
 * J(tau) = 1/2 Int_0^{tau_max} S(t) E_1(|t - tau|) dt (the mean intensity of the same
 * plane-parallel slab whose emergent flux is taken: S linear between layers, the first segment
 * extrapolated to tau = 0, nothing below the bottom layer).  With S piecewise linear, J at a layer
 * is a linear form in the layer values, J = Lambda S; the paper iterates the scattering term,
 * S <- eps B + (1 - eps) Lambda S, whose fixed point solves (I - diag(1 - eps) Lambda) S = eps B.
 * The oracle solves that system directly (Gaussian elimination with partial pivoting). */

/* 1/2 Int_a^b S(t) E_1(|t - tj|) dt for S linear from Sa (at a) to Sb (at b), as weights
 * (*wa, *wb) of Sa and Sb; [a, b] lies wholly below tj (a >= tj) or above it (b <= tj). */
static void lambda_interval(double tj, double a, double b, double *wa, double *wb) {
    double D = b - a;
    if (a >= tj) {
        /* t = tj + x:  Int (Sa + s(t - a)) E_1(x) = Sa (E2(xa) - E2(xb)) + s (E3(xa) - E3(xb) - D E2(xb)) */
        double xa = a - tj, xb = b - tj;
        double e2a = pzo_expn(2, xa), e2b = pzo_expn(2, xb), e3a = pzo_expn(3, xa), e3b = pzo_expn(3, xb);
        double slope = (e3a - e3b - D * e2b) / D;
        *wa = 0.5 * ((e2a - e2b) - slope);
        *wb = 0.5 * slope;
    } else {
        /* t = tj - y:  Int (Sb - s(b - t)) E_1(y) = Sb (E2(yb) - E2(ya)) - s (E3(yb) - E3(ya) - D E2(ya)) */
        double ya = tj - a, yb = tj - b;
        double e2a = pzo_expn(2, ya), e2b = pzo_expn(2, yb), e3a = pzo_expn(3, ya), e3b = pzo_expn(3, yb);
        double slope = (e3b - e3a - D * e2a) / D;
        *wb = 0.5 * ((e2b - e2a) - slope);
        *wa = 0.5 * slope;
    }
}

/* Lambda [nd][nd]: row j gives J(tau_j) from the layer values of S. */
void pzo_lambda_matrix(int nd, const double *tau, double *Lam) {
    for (int64_t k = 0; k < (int64_t)nd * nd; ++k) Lam[k] = 0.0;
    if (nd < 2) return;
    double D1 = tau[1] - tau[0];
    for (int j = 0; j < nd; ++j) {
        double *row = Lam + (int64_t)j * nd;
        double wa, wb;
        for (int k = 0; k + 1 < nd; ++k) {
            lambda_interval(tau[j], tau[k], tau[k + 1], &wa, &wb);
            row[k] += wa;
            row[k + 1] += wb;
        }
        /* top interval [0, tau_0]: S(0) = S_0 - s_0 tau_0 with s_0 = (S_1 - S_0)/D1 */
        lambda_interval(tau[j], 0.0, tau[0], &wa, &wb);
        row[0] += wa * (1.0 + tau[0] / D1) + wb;
        row[1] += -wa * tau[0] / D1;
    }
}

/* Solve (I - diag(1 - eps) Lambda) S = eps B for S. */
void pzo_scatter_source(int nd, const double *tau, const double *eps, const double *B, double *S) {
    double *A = (double *)malloc(sizeof(double) * (size_t)nd * (nd + 1));
    double *Lam = (double *)malloc(sizeof(double) * (size_t)nd * nd);
    pzo_lambda_matrix(nd, tau, Lam);
    int W = nd + 1;
    for (int j = 0; j < nd; ++j) {
        for (int k = 0; k < nd; ++k) A[(int64_t)j * W + k] = (j == k ? 1.0 : 0.0) - (1.0 - eps[j]) * Lam[(int64_t)j * nd + k];
        A[(int64_t)j * W + nd] = eps[j] * B[j];
    }
    for (int p = 0; p < nd; ++p) {
        int piv = p;
        for (int r = p + 1; r < nd; ++r)
            if (fabs(A[(int64_t)r * W + p]) > fabs(A[(int64_t)piv * W + p])) piv = r;
        if (piv != p)
            for (int k = 0; k < W; ++k) {
                double t = A[(int64_t)p * W + k];
                A[(int64_t)p * W + k] = A[(int64_t)piv * W + k];
                A[(int64_t)piv * W + k] = t;
            }
        for (int r = p + 1; r < nd; ++r) {
            double f = A[(int64_t)r * W + p] / A[(int64_t)p * W + p];
            for (int k = p; k < W; ++k) A[(int64_t)r * W + k] -= f * A[(int64_t)p * W + k];
        }
    }
    for (int p = nd - 1; p >= 0; --p) {
        double v = A[(int64_t)p * W + nd];
        for (int k = p + 1; k < nd; ++k) v -= A[(int64_t)p * W + k] * S[k];
        S[p] = v / A[(int64_t)p * W + p];
    }
    free(Lam);
    free(A);
}

/* F and F_c for the requested columns given kappa_line there (same layout as pzo_kappa_line).
 * Without sigma_c, S = B in both branches; with it, each branch solves its own scattering
 * source (total: eps = (kappa_c + kappa_line)/chi; continuum: eps_c = kappa_c/(kappa_c + sigma_c)). */
void pzo_flux(const pzo_problem *P, int64_t n_cols, const int64_t *cols, const double *kline,
              double *F, double *Fc) {
    int nd = P->n_depth;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n_cols; ++c) {
        int64_t i = cols[c];
        double *chi = (double *)malloc(sizeof(double) * nd * 7);
        double *chic = chi + nd, *tau = chi + 2 * nd, *S = chi + 3 * nd, *B = chi + 4 * nd;
        double *eps = chi + 5 * nd, *Ssc = chi + 6 * nd;
        double lam = grid_lambda_cm(P, i);
        for (int d = 0; d < nd; ++d) {
            int64_t o = (int64_t)d * P->n_lambda + i;
            double sig = P->sigma_c ? P->sigma_c[o] : 0.0;
            double kl = kline[(int64_t)d * n_cols + c];
            chic[d] = P->kappa_c[o] + sig;
            chi[d] = P->kappa_c[o] + kl + sig;
            B[d] = planck_nm(lam, P->T[d]);
            S[d] = B[d];
            eps[d] = (P->kappa_c[o] + kl) / chi[d];
        }
        optical_depth(nd, P->m, chi, tau);
        if (P->sigma_c) {
            pzo_scatter_source(nd, tau, eps, B, Ssc);
            F[c] = flux_from(nd, tau, Ssc);
        } else {
            F[c] = flux_from(nd, tau, S);
        }
        optical_depth(nd, P->m, chic, tau);
        if (P->sigma_c) {
            for (int d = 0; d < nd; ++d) {
                int64_t o = (int64_t)d * P->n_lambda + i;
                eps[d] = P->kappa_c[o] / chic[d];
            }
            pzo_scatter_source(nd, tau, eps, B, Ssc);
            Fc[c] = flux_from(nd, tau, Ssc);
        } else {
            Fc[c] = flux_from(nd, tau, S);
        }
        free(chi);
    }
}

/* ---- instrument (Sec. 7): row-normalised Gaussian taps ------------------- */
/* Pixel p at observed wavelength lambda_p samples rest wavelength
 * lambda_p / (1 + v_r/c).  Gaussian in ln(lambda) with sigma^2 = sigma_LSF^2 + sigma_b^2,
 * sigma_LSF = 1/(2 sqrt(2 ln 2) R_LSF), sigma_b = v_b/c; taps |ln lambda_i - ln lambda'_p| <= 5 sigma
 * clipped to the grid and renormalised over the in-grid taps; point sampling. */
int pzo_instrument_taps(const pzo_problem *P, double v_r_kms, double v_b_kms, double R_lsf,
                        int64_t n_pix, const double *pix_nm, int64_t *tap0, int32_t *ntap,
                        double *weights, int32_t max_taps) {
    double lnr = log1p(1.0 / P->R_grid);
    double sig_lsf = 1.0 / (2.0 * sqrt(2.0 * log(2.0)) * R_lsf);
    double sig_b = v_b_kms * 1e5 / O_C;
    double sig = sqrt(sig_lsf * sig_lsf + sig_b * sig_b) / lnr;   /* grid points */
    for (int64_t p = 0; p < n_pix; ++p) {
        double rest = pix_nm[p] / (1.0 + v_r_kms * 1e5 / O_C);
        double cp = log(rest / P->lambda0_nm) / lnr;
        int64_t i0 = (int64_t)ceil(cp - 5.0 * sig);
        int64_t i1 = (int64_t)floor(cp + 5.0 * sig);
        if (i0 < 0) i0 = 0;
        if (i1 > P->n_lambda - 1) i1 = P->n_lambda - 1;
        if (i1 < i0) return -1;
        if (i1 - i0 + 1 > max_taps) return -2;
        double sum = 0.0;
        for (int64_t i = i0; i <= i1; ++i) {
            double u = ((double)i - cp) / sig;
            double w = exp(-0.5 * u * u);
            weights[p * max_taps + (i - i0)] = w;
            sum += w;
        }
        for (int64_t i = i0; i <= i1; ++i) weights[p * max_taps + (i - i0)] /= sum;
        tap0[p] = i0;
        ntap[p] = (int32_t)(i1 - i0 + 1);
    }
    return 0;
}

/* ---- adjoint (Sec. 6) ------------------------------------------------------ */

/* d/dtau_a and d/dtau_b of the interval integral at fixed Sa, Sb. */
static void interval_partials(double ta, double tb, double Sa, double Sb, double *dta, double *dtb) {
    double D = tb - ta;
    double s = (Sb - Sa) / D;
    double e2a = pzo_expn(2, ta), e2b = pzo_expn(2, tb);
    double e3a = pzo_expn(3, ta), e3b = pzo_expn(3, tb);
    double e4a = pzo_expn(4, ta), e4b = pzo_expn(4, tb);
    double Pd = e3a - e3b;
    double Bq = e4a - e4b - D * e3b;
    *dta = -Sa * e2a + (s / D) * Bq - s * Pd;
    *dtb = Sb * e2b - (s / D) * Bq;
}

/* dF/dtau_j (j = 0..nd-1) of flux_from(). */
static void flux_dtau(int nd, const double *tau, const double *S, double *dF) {
    for (int j = 0; j < nd; ++j) dF[j] = 0.0;
    /* top interval: Sa = S0 - s tau0, s = (S1-S0)/(tau1-tau0) */
    double t0 = tau[0], t1 = tau[1];
    double s = (S[1] - S[0]) / (t1 - t0);
    double sp = s / (t1 - t0);
    double Pt = 0.5 - pzo_expn(3, t0);
    double Bt = 1.0 / 3.0 - pzo_expn(4, t0) - t0 * pzo_expn(3, t0);
    dF[0] += -s * Pt + sp * (Bt - t0 * Pt) + S[0] * pzo_expn(2, t0);
    dF[1] += -sp * (Bt - t0 * Pt);
    for (int d = 0; d + 1 < nd; ++d) {
        double da, db;
        interval_partials(tau[d], tau[d + 1], S[d], S[d + 1], &da, &db);
        dF[d] += da;
        dF[d + 1] += db;
    }
    for (int j = 0; j < nd; ++j) dF[j] *= 2.0 * O_PI;
}

/* dL/dchi(i, d) for every column, given dL/dF_i (total branch; F_c does not depend on
 * line opacity).  G[d * n_lambda + i].  Chain rule written with the explicit Jacobian
 * d tau_j / d chi_d of the trapezoid. */
/* ---- reverse pass through the scattering source ------------------------------- */

/* dF/dS_k of flux_from (F is linear in the layer values of S): 2 pi times each interval's
 * coefficients, the top interval's extrapolated S(0) = S_0 - tau_0 (S_1 - S_0)/D1 chained
 * to S_0 and S_1. */
static void flux_dS(int nd, const double *tau, double *a) {
    for (int k = 0; k < nd; ++k) a[k] = 0.0;
    for (int d = 0; d + 1 < nd; ++d) {
        double ta = tau[d], tb = tau[d + 1], D = tb - ta;
        double q = (pzo_expn(4, ta) - pzo_expn(4, tb) - D * pzo_expn(3, tb)) / D;
        a[d] += (pzo_expn(3, ta) - pzo_expn(3, tb)) - q;
        a[d + 1] += q;
    }
    double t0 = tau[0], D1 = tau[1] - tau[0];
    double q = (1.0 / 3.0 - pzo_expn(4, t0) - t0 * pzo_expn(3, t0)) / t0;
    double a_zero = (0.5 - pzo_expn(3, t0)) - q;   /* coefficient of S(0) */
    a[0] += q + a_zero * (1.0 + t0 / D1);
    a[1] += -a_zero * t0 / D1;
    for (int k = 0; k < nd; ++k) a[k] *= 2.0 * O_PI;
}

/* dJ[j][m] = d J_j / d tau_m at fixed layer values S, J = Lambda S.  Moving layer m with its
 * value fixed reshapes the two segments that meet there: with s the segment slopes and w the
 * layer's Lambda weight from each segment (seen from tau_j), -s_{m-1} w - s_m w; the end
 * terms 1/2 S_m E_1(|tau_m - tau_j|) of the two segments cancel except at the bottom layer,
 * where the slab ends with it.  The top segment's extrapolation adds its own dependence on
 * tau_0 and tau_1.  The layer j itself follows from translation invariance: shifting every
 * layer and the surface together leaves J_j unchanged, so sum_m dJ_j/dtau_m = 1/2 S(0) E_1(tau_j). */
void pzo_lambda_dtau(int nd, const double *tau, const double *S, double *dJ) {
    double D1 = tau[1] - tau[0];
    double s0 = (S[1] - S[0]) / D1;
    double Szero = S[0] - s0 * tau[0];
    for (int j = 0; j < nd; ++j) {
        double *row = dJ + (int64_t)j * nd;
        double tj = tau[j];
        for (int m = 0; m < nd; ++m) row[m] = 0.0;
        /* top segment [0, tau_0]: weights of its values at 0 (lo) and tau_0 (hi) */
        double wlo, whi;
        lambda_interval(tj, 0.0, tau[0], &wlo, &whi);
        row[0] += 0.5 * S[0] * pzo_expn(1, fabs(tau[0] - tj)) - (s0 / D1) * tau[0] * wlo - s0 * (wlo + whi);
        row[1] += (s0 / D1) * tau[0] * wlo;
        /* segments [tau_k, tau_k+1] */
        for (int k = 0; k + 1 < nd; ++k) {
            double wa, wb;
            lambda_interval(tj, tau[k], tau[k + 1], &wa, &wb);
            double sk = (S[k + 1] - S[k]) / (tau[k + 1] - tau[k]);
            row[k] += -sk * wa;          /* its lower end moves */
            row[k + 1] += -sk * wb;      /* its upper end moves */
            /* end terms: +1/2 S E_1 at a moving upper end, -1/2 S E_1 at a moving lower end */
            double e1b = (k + 1 == j) ? 0.0 : pzo_expn(1, fabs(tau[k + 1] - tj));
            double e1a = (k == j) ? 0.0 : pzo_expn(1, fabs(tau[k] - tj));
            row[k + 1] += 0.5 * S[k + 1] * e1b;
            row[k] -= 0.5 * S[k] * e1a;
        }
        /* the layer itself */
        double off = 0.0;
        for (int m = 0; m < nd; ++m)
            if (m != j) off += row[m];
        row[j] = 0.5 * Szero * pzo_expn(1, tj) - off;
    }
}

/* Reverse pass of one column's scattering flux: with S solving (I - diag(1 - eps) Lambda) S
 * = eps B and F = flux_from(tau, S), returns dL/dtau (gtau) and dL/deps (geps) for
 * dL/dF = Fbar.  The adjoint mu solves M^T mu = Fbar dF/dS; then
 *   dL/deps_j = mu_j (B_j - J_j),
 *   dL/dtau_m = Fbar dF/dtau_m (at fixed S) + sum_j mu_j (1 - eps_j) dJ_j/dtau_m. */
void pzo_scatter_adjoint(int nd, const double *tau, const double *eps, const double *B, double Fbar, double *gtau,
                         double *geps) {
    size_t n2 = (size_t)nd * nd;
    double *Lam = (double *)malloc(sizeof(double) * (n2 * 3 + (size_t)nd * (nd + 1) + 6 * nd));
    double *dJ = Lam + n2, *A = dJ + n2, *Mt = A + (size_t)nd * (nd + 1);
    double *S = Mt + n2, *J = S + nd, *a = J + nd, *mu = a + nd, *dF = mu + nd;
    pzo_scatter_source(nd, tau, eps, B, S);
    pzo_lambda_matrix(nd, tau, Lam);
    for (int j = 0; j < nd; ++j) {
        double v = 0.0;
        for (int k = 0; k < nd; ++k) v += Lam[(int64_t)j * nd + k] * S[k];
        J[j] = v;
    }
    flux_dS(nd, tau, a);
    flux_dtau(nd, tau, S, dF);
    /* M^T mu = Fbar a, M = I - diag(1 - eps) Lambda: Gaussian elimination with partial pivoting */
    int W = nd + 1;
    for (int r = 0; r < nd; ++r) {
        for (int c = 0; c < nd; ++c)
            A[(int64_t)r * W + c] = (r == c ? 1.0 : 0.0) - (1.0 - eps[c]) * Lam[(int64_t)c * nd + r];
        A[(int64_t)r * W + nd] = Fbar * a[r];
    }
    for (int p = 0; p < nd; ++p) {
        int piv = p;
        for (int r = p + 1; r < nd; ++r)
            if (fabs(A[(int64_t)r * W + p]) > fabs(A[(int64_t)piv * W + p])) piv = r;
        if (piv != p)
            for (int k = 0; k < W; ++k) {
                double t = A[(int64_t)p * W + k];
                A[(int64_t)p * W + k] = A[(int64_t)piv * W + k];
                A[(int64_t)piv * W + k] = t;
            }
        for (int r = p + 1; r < nd; ++r) {
            double f = A[(int64_t)r * W + p] / A[(int64_t)p * W + p];
            for (int k = p; k < W; ++k) A[(int64_t)r * W + k] -= f * A[(int64_t)p * W + k];
        }
    }
    for (int p = nd - 1; p >= 0; --p) {
        double v = A[(int64_t)p * W + nd];
        for (int k = p + 1; k < nd; ++k) v -= A[(int64_t)p * W + k] * mu[k];
        mu[p] = v / A[(int64_t)p * W + p];
    }
    pzo_lambda_dtau(nd, tau, S, dJ);
    for (int j = 0; j < nd; ++j) geps[j] = mu[j] * (B[j] - J[j]);
    for (int m = 0; m < nd; ++m) {
        double g = Fbar * dF[m];
        for (int j = 0; j < nd; ++j) g += mu[j] * (1.0 - eps[j]) * dJ[(int64_t)j * nd + m];
        gtau[m] = g;
    }
    (void)Mt;
    free(Lam);
}

/* emergent flux of the scattering source on explicit tau, eps, B (for the adjoint pins) */
double pzo_scatter_flux(int nd, const double *tau, const double *eps, const double *B) {
    double *S = (double *)malloc(sizeof(double) * nd);
    pzo_scatter_source(nd, tau, eps, B, S);
    double F = flux_from(nd, tau, S);
    free(S);
    return F;
}

void pzo_rt_adjoint(const pzo_problem *P, const double *kline_full, const double *dLdF, double *G) {
    int nd = P->n_depth;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < P->n_lambda; ++i) {
        double *chi = (double *)malloc(sizeof(double) * nd * 6);
        double *tau = chi + nd, *S = chi + 2 * nd, *dF = chi + 3 * nd, *eps = chi + 4 * nd, *geps = chi + 5 * nd;
        double lam = grid_lambda_cm(P, i);
        for (int d = 0; d < nd; ++d) {
            int64_t o = (int64_t)d * P->n_lambda + i;
            double sig = P->sigma_c ? P->sigma_c[o] : 0.0;
            chi[d] = P->kappa_c[o] + kline_full[o] + sig;
            eps[d] = (P->kappa_c[o] + kline_full[o]) / chi[d];
            S[d] = planck_nm(lam, P->T[d]);
        }
        optical_depth(nd, P->m, chi, tau);
        if (P->sigma_c) {
            /* dF/dtau here is dL/dtau for dL/dF = 1 (S follows tau and eps); the eps part is
             * added per layer below: eps = 1 - sigma/chi, so d eps / d kappa_line = sigma/chi^2 */
            pzo_scatter_adjoint(nd, tau, eps, S, 1.0, dF, geps);
        } else {
            flux_dtau(nd, tau, S, dF);
            for (int d = 0; d < nd; ++d) geps[d] = 0.0;
        }
        for (int d = 0; d < nd; ++d) {
            double g = 0.0;
            for (int j = 0; j < nd; ++j) {
                /* d tau_j / d chi_d */
                double J = 0.0;
                if (d == 0) J += P->m[0];
                for (int k = 0; k < j; ++k) {
                    double hm = 0.5 * (P->m[k + 1] - P->m[k]);
                    if (d == k) J += hm;
                    if (d == k + 1) J += hm;
                }
                g += dF[j] * J;
            }
            if (P->sigma_c) {
                double sig = P->sigma_c[(int64_t)d * P->n_lambda + i];
                g += geps[d] * sig / (chi[d] * chi[d]);
            }
            G[(int64_t)d * P->n_lambda + i] = dLdF[i] * g;
        }
        free(chi);
    }
}

/* Per-line gradients from G = dL/dkappa_line (all columns), Eq. 10 differentiated:
 *   dL/dDelta log gf_l         = ln10 sum_{i in win, d} G stim A H
 *   dL/dDelta log gamma_beta_l = ln10 sum_{i in win, d} G stim A (dH/da) a_beta,
 * a_beta the part of the damping parameter that family beta contributes (van der Waals
 * a6, radiative arad, Stark a4), since 10^delta scales that part alone.  g_rad and g_4
 * may be NULL.  (The abundance gradient is the species-to-element sum of the first.) */
void pzo_line_grad(const pzo_problem *P, const double *G, double *g_gf, double *g_g6, double *g_rad,
                   double *g_4) {
    int nd = P->n_depth;
    int W = P->half_window;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t l = 0; l < P->n_lines; ++l) {
        double x = centre_x(P, l);
        int64_t il = (int64_t)floor(x + 0.5);
        int64_t i0 = il - W, i1 = il + W;
        if (i0 < 0) i0 = 0;
        if (i1 > P->n_lambda - 1) i1 = P->n_lambda - 1;
        double lam_l = P->lambda_nm[l] * 1e-7;
        double sgf = 0.0, sg6 = 0.0, srad = 0.0, sg4 = 0.0;
        for (int d = 0; d < nd; ++d) {
            line_depth q = line_at_depth(P, l, d);
            if (!centre_keep(P, il, d, q.A)) continue;
            for (int64_t i = i0; i <= i1; ++i) {
                double v = (lam_l / grid_lambda_cm(P, i) - 1.0) * O_C / q.dvD;
                double H, dH;
                pzo_voigt(q.a, v, &H, NULL, &dH);
                double gs = G[(int64_t)d * P->n_lambda + i] * stim_emission(P, i, d);
                sgf += gs * q.A * H;
                sg6 += gs * q.A * dH * q.a6;
                srad += gs * q.A * dH * q.arad;
                sg4 += gs * q.A * dH * q.a4;
            }
        }
        g_gf[l] = O_LN10 * sgf;
        g_g6[l] = O_LN10 * sg6;
        if (g_rad) g_rad[l] = O_LN10 * srad;
        if (g_4) g_4[l] = O_LN10 * sg4;
    }
}

/* chi^2 loss L = sum_p w_p (y_p - f_p)^2 and its seed dL/df_p = -2 w_p (y_p - f_p). */
double pzo_chi2(int64_t n, const double *y, const double *w, const double *f, double *dLdf) {
    double L = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        double r = y[p] - f[p];
        L += w[p] * r * r;
        if (dLdf) dLdf[p] = -2.0 * w[p] * r;
    }
    return L;
}

/* ---- vector helpers for the Python wrapper -------------------------------- */
void pzo_voigt_vec(int64_t n, const double *a, const double *v, double *H, double *L, double *dH) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) pzo_voigt(a[k], v[k], &H[k], L ? &L[k] : NULL, dH ? &dH[k] : NULL);
}

void pzo_expn_vec(int n, int64_t cnt, const double *x, double *out) {
    for (int64_t k = 0; k < cnt; ++k) out[k] = pzo_expn(n, x[k]);
}

/* flux of one column from explicit tau/S (for the closed-form pins) */
double pzo_flux_tau(int nd, const double *tau, const double *S) { return flux_from(nd, tau, S); }

/* dF/dtau of one column (for the adjoint pins) */
void pzo_flux_dtau(int nd, const double *tau, const double *S, double *dF) { flux_dtau(nd, tau, S, dF); }

double pzo_planck_nm(double lambda_nm, double T) { return planck_nm(lambda_nm * 1e-7, T); }

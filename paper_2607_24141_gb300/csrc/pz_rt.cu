// pz_rt.cu -- per-wavelength LTE formal solution (Eqs. 6-8), instrument stage
// and normalisation (Sec. 7, Eq. 9), chi-square objective, and their adjoints
// (Sec. 6).  All transfer arithmetic is FP64: optical depths at the top layers
// are ~1e-8 while E_3(0) = 1/2, so the interval integrals are differences of
// nearly equal numbers.
//
// Flux: for every wavelength one thread walks the depth axis, accumulating
// tau by the trapezoid rule on column mass, and sums the closed form
//   Int_{ta}^{tb} S E_2 dtau = Sa (E3(ta) - E3(tb)) + s (E4(ta) - E4(tb) - (tb - ta) E3(tb)),
// s = (Sb - Sa)/(tb - ta), over the layers plus the top interval [0, tau_0]
// (S extrapolated linearly from the first segment).  Nothing is added below
// the bottom layer.  Total and continuum branches share the walk.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "pz_internal.h"

namespace pz {

constexpr double kEuler = 0.57721566490153286061;

// ---------------------------------------------------------------------------
// E_2, E_3, E_4 from a Taylor table of E_4 (FP64).
//
// The FP64 units of this GPU are few, so the exponential integrals (two calls per
// wavelength and layer in the flux, one in its adjoint) must cost few FP64
// instructions and no divides.  E_4 is expanded about table nodes x0,
//   E_4(x0 + t) = sum_k c_k t^k,  c_k = E_4^(k)(x0) / k!,
// and E_3 = -E_4', E_2 = E_4'' come from the same polynomial (Horner with
// derivatives), using E_n' = -E_{n-1}.  The coefficients are exact derivatives:
//   E_4^(k) = (-1)^k E_{4-k} (k <= 4, E_0 = e^-x / x),
//   E_0^(m) = (-1)^m e^-x m! sum_{i=0..m} x^-(i+1) / (m-i)!   (all terms positive).
// Nodes: 2^-40 <= x < 2: eight per binade at the centres of the binade's eighths
// (|t| / x0 <= 1/17, inside the radius of convergence x0 of the logarithmic
// singularity at 0); 2 <= x < 40: spacing 1/8 (|t| <= 1/16).  Fourteen terms
// leave a truncation error below 1e-16 relative in both ranges.  Outside them:
// x < 2^-40 the leading terms of the small-x expansion, x >= 40 the continued
// fraction of E_4 (8 levels), x > 740 zero.
// ---------------------------------------------------------------------------
constexpr int kExpnK = 14;                      // Taylor terms per node
constexpr int kExpnMinExp = -40;                // smallest binade 2^-40
constexpr int kExpnGeo = (1 - kExpnMinExp) * 8; // nodes below 2: binades -40..0
constexpr double kExpnUni0 = 2.0, kExpnUni1 = 40.0;
constexpr int kExpnUni = (int)((kExpnUni1 - kExpnUni0) * 8);   // nodes on [2, 40)
constexpr int kExpnNodes = kExpnGeo + kExpnUni;

__device__ double g_expn_tab[kExpnNodes * kExpnK];
// The same nodes for E_3 (E_3 = p, E_2 = -p'): the scattering kernels need E_2 and E_3 at
// every layer pair, and two Horner chains cost 2/3 of the three E_4 takes.
__device__ double g_expn3_tab[kExpnNodes * kExpnK];

// host: E_1..E_4 at x > 0 in extended precision (series below 2, continued fraction above)
static void expn_host(long double x, long double E[5]) {
    const long double ex = expl(-x);
    if (x <= 2.0L) {
        long double term = 1.0L, s = 0.0L;
        for (int k = 1; k < 200; ++k) {
            term *= -x / k;
            s += term / k;
            if (fabsl(term) < 1e-30L) break;
        }
        E[1] = -(long double)kEuler - logl(x) - s;
        for (int n = 1; n < 4; ++n) E[n + 1] = (ex - x * E[n]) / n;
    } else {
        const int K = 600;
        long double f = x + 4.0L + 2.0L * K;
        for (int k = K; k >= 1; --k) f = x + 4.0L + 2.0L * (k - 1) - (long double)k * (3.0L + k) / f;
        E[4] = ex / f;
        for (int n = 3; n >= 1; --n) E[n] = (ex - n * E[n + 1]) / x;
    }
    E[0] = ex / x;
}

// Taylor coefficients E_n^(k)(x0)/k! of E_n (n = 3 or 4) about x0:
//   E_n^(k) = (-1)^k E_{n-k} (k <= n),  E_n^(k) = (-1)^n E_0^(k-n) (k > n).
static void expn_node_coeffs(long double x0, double *c, int n = 4) {
    long double E[5];
    expn_host(x0, E);
    long double fact = 1.0L;   // k!
    for (int k = 0; k < kExpnK; ++k) {
        if (k > 0) fact *= k;
        long double d;
        if (k <= n) {
            d = ((k & 1) ? -1.0L : 1.0L) * E[n - k];
        } else {
            const int m = k - n;
            long double sum = 0.0L, mf = 1.0L;   // m! / (m - i)! built as a running product
            for (int i = 0; i <= m; ++i) {
                if (i > 0) mf *= (m - i + 1);
                sum += mf * powl(x0, -(long double)(i + 1));
            }
            d = ((n & 1) ? -1.0L : 1.0L) * ((m & 1) ? -1.0L : 1.0L) * expl(-x0) * sum;
        }
        c[k] = (double)(d / fact);
    }
}

static double expn_node_x0(int j) {
    if (j < kExpnGeo) {
        const int e = kExpnMinExp + j / 8, m = j % 8;
        return std::ldexp(1.0 + (m + 0.5) / 8.0, e);
    }
    return kExpnUni0 + (j - kExpnGeo + 0.5) / 8.0;
}

pz_status ensure_expn_table() {
    static std::mutex mu;
    static std::vector<double> tab;
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(PZ_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return PZ_OK;
    static std::vector<double> tab3;
    if (tab.empty()) {
        tab.resize((size_t)kExpnNodes * kExpnK);
        tab3.resize((size_t)kExpnNodes * kExpnK);
        for (int j = 0; j < kExpnNodes; ++j) {
            expn_node_coeffs((long double)expn_node_x0(j), &tab[(size_t)j * kExpnK], 4);
            expn_node_coeffs((long double)expn_node_x0(j), &tab3[(size_t)j * kExpnK], 3);
        }
    }
    e = cudaMemcpyToSymbol(g_expn_tab, tab.data(), sizeof(double) * tab.size());
    if (e != cudaSuccess) return cuda_check(e, "upload E_n table");
    e = cudaMemcpyToSymbol(g_expn3_tab, tab3.data(), sizeof(double) * tab3.size());
    if (e != cudaSuccess) return cuda_check(e, "upload E_3 table");
    done[dev] = true;
    return PZ_OK;
}

// Node of x in [2^-40, 40) and the offset t = x - x0 (exact), from the bits of x alone
// (integer operations: the FP64 pipe is kept for the series).  Below 2, eight nodes per
// binade at the centres of its eighths (x0 keeps three mantissa bits and sets the fourth);
// on [2, 40) nodes every 1/8 at the centres (j - kExpnGeo = floor(8 x) - 16, x0 = x rounded
// down to a multiple of 1/8 plus 1/16).
__device__ __forceinline__ int expn_node(double x, double &t) {
    const long long bits = __double_as_longlong(x);
    const int ex = (int)(bits >> 52) - 1023;           // x > 0
    int j;
    long long x0b;
    if (ex < 1) {
        j = (ex - kExpnMinExp) * 8 + (int)((bits >> 49) & 7);
        x0b = (bits & ~((1LL << 49) - 1)) | (1LL << 48);
    } else {
        const int sh = 49 - ex;                        // mantissa bit of 1/8
        j = kExpnGeo - 16 + (int)(((bits & ((1LL << 52) - 1)) | (1LL << 52)) >> sh);
        x0b = (bits & ~((1LL << sh) - 1)) | (1LL << (sh - 1));
    }
    t = x - __longlong_as_double(x0b);
    return j;
}

// Ranges of x by its bits (x >= 0 orders like its bit pattern)
constexpr long long kBits2m40 = 0x3D70000000000000LL;   // 2^-40
constexpr long long kBits40 = 0x4044000000000000LL;     // 40.0

__device__ __forceinline__ void expn234(double x, double &E2, double &E3, double &E4) {
    const long long xb = __double_as_longlong(x);
    if (xb <= 0) {
        E2 = 1.0;
        E3 = 0.5;
        E4 = 1.0 / 3.0;
        return;
    }
    if (xb < kBits40) {
        if (xb < kBits2m40) {
            // E_2 = 1 + x (ln x + gamma - 1) + O(x^2), E_3 = 1/2 - x + O(x^2 ln x), E_4 = 1/3 - x/2 + O(x^2)
            E2 = 1.0 + x * (log(x) + (kEuler - 1.0));
            E3 = 0.5 - x;
            E4 = 1.0 / 3.0 - 0.5 * x;
            return;
        }
        double t;
        const double *c = g_expn_tab + expn_node(x, t) * kExpnK;
        double p = __ldg(c + kExpnK - 1), d1 = 0.0, d2 = 0.0;
#pragma unroll
        for (int k = kExpnK - 2; k >= 0; --k) {
            d2 = fma(d2, t, d1);
            d1 = fma(d1, t, p);
            p = fma(p, t, __ldg(c + k));
        }
        E4 = p;
        E3 = -d1;
        E2 = 2.0 * d2;
        return;
    }
    if (x > 740.0) {
        E2 = E3 = E4 = 0.0;
        return;
    }
    // E_4(x) = e^-x / (x + 4 - 1*4/(x + 6 - 2*5/(x + 8 - ...))), then downward
    const double ex = exp(-x);
    double f = x + 4.0 + 16.0;
    for (int k = 8; k >= 1; --k) f = x + 4.0 + 2.0 * (k - 1) - (double)k * (3.0 + k) / f;
    E4 = ex / f;
    E3 = (ex - 3.0 * E4) / x;
    E2 = (ex - 2.0 * E3) / x;
}

// E3 and E4 alone (the flux needs no E2): the value and first-derivative chains of the same
// E4 Taylor table, with expn234's branches; identical E3, E4 to expn234's.
__device__ __forceinline__ void expn34(double x, double &E3, double &E4) {
    const long long xb = __double_as_longlong(x);
    if (xb <= 0 || xb >= kBits40 || xb < kBits2m40) {
        double e2;
        expn234(x, e2, E3, E4);
        return;
    }
    double t;
    const double *c = g_expn_tab + expn_node(x, t) * kExpnK;
    double p = __ldg(c + kExpnK - 1), d1 = 0.0;
#pragma unroll
    for (int k = kExpnK - 2; k >= 0; --k) {
        d1 = fma(d1, t, p);
        p = fma(p, t, __ldg(c + k));
    }
    E4 = p;
    E3 = -d1;
}

// Planck function per nanometre
__device__ __forceinline__ double planck_nm(double lamcm, double T) {
    double l2 = lamcm * lamcm;
    return 2.0 * kH * kC * kC / (l2 * l2 * lamcm) / expm1(kC2 / (lamcm * T)) * 1e-7;
}

// B_lambda(T_d) and the stimulated-emission factor 1 - exp(-hc/(lambda k T_d)) at every
// (star, layer, grid point): they depend on the atmosphere and the grid alone, like kappa_c,
// and the flux, its adjoint and the scattering kernels read them (one thread per point).
__global__ void k_planck_tables(int64_t nlam, int64_t ld, int nd, double lam0cm, double lnr, const double *T,
                                double *B, double *stim) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nlam) return;
    const int64_t sd = blockIdx.y;     // star * nd + layer
    const double lam = lam0cm * exp((double)i * lnr);
    const double t = T[sd];
    B[sd * ld + i] = planck_nm(lam, t);
    stim[sd * ld + i] = -expm1(-kC2 / (lam * t));
}

cudaError_t launch_planck_tables(pz_ctx *c, cudaStream_t s) {
    if (c->nlam <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((c->nlam + 255) / 256), (unsigned)((int64_t)c->S * c->nd));
    k_planck_tables<<<grid, 256, 0, s>>>(c->nlam, c->ld, c->nd, c->lambda0_nm * 1e-7, c->lnr, c->d_T, c->d_B, c->d_stim);
    c->launches++;
    return cudaGetLastError();
}

__device__ __forceinline__ double interval(double ta, double tb, double Sa, double Sb, double e3a, double e4a,
                                           double e3b, double e4b) {
    double D = tb - ta;
    double s = (Sb - Sa) / D;
    return Sa * (e3a - e3b) + s * (e4a - e4b - D * e3b);
}

struct FluxArgs {
    int64_t nlam, ld;
    int nd;
    double lam0cm, lnr;
    const double *m, *T, *kc, *B;
    const void *kline;
    double *F, *Fc;
};

// one thread per (lambda, star); star = blockIdx.y
template <typename KT>
__global__ void k_flux(FluxArgs g) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nlam) return;
    {
        const int st = blockIdx.y;
        g.m += (int64_t)st * g.nd;
        g.T += (int64_t)st * g.nd;
        g.kc += (int64_t)st * g.nd * g.ld;
        g.B += (int64_t)st * g.nd * g.ld;
        g.kline = reinterpret_cast<const KT *>(g.kline) + (int64_t)st * g.nd * g.ld;
        g.F += (int64_t)st * g.nlam;
        g.Fc += (int64_t)st * g.nlam;
    }
    const KT *kl = reinterpret_cast<const KT *>(g.kline);
    double chi_p = 0, chic_p = 0, tau_p = 0, tauc_p = 0, S_p = 0, m_p = 0;
    double e3p = 0, e4p = 0, e3cp = 0, e4cp = 0;
    double F = 0.0, Fc = 0.0;
    double tau0 = 0, tauc0 = 0, S0 = 0, e3_0 = 0, e4_0 = 0, e3c_0 = 0, e4c_0 = 0;
    for (int d = 0; d < g.nd; ++d) {
        const int64_t o = (int64_t)d * g.ld + i;
        const double kc = g.kc[o];
        const double chi = kc + (double)kl[o];
        const double md = g.m[d];
        const double S = g.B[o];
        double tau, tauc;
        if (d == 0) {
            tau = chi * md;
            tauc = kc * md;
        } else {
            tau = tau_p + 0.5 * (chi_p + chi) * (md - m_p);
            tauc = tauc_p + 0.5 * (chic_p + kc) * (md - m_p);
        }
        double e3, e4, e3c, e4c;
        expn34(tau, e3, e4);
        expn34(tauc, e3c, e4c);
        if (d == 0) {
            tau0 = tau; tauc0 = tauc; S0 = S;
            e3_0 = e3; e4_0 = e4; e3c_0 = e3c; e4c_0 = e4c;
        } else {
            if (d == 1) {
                // top interval [0, tau_0], S linear through layers 0 and 1
                double s0 = (S - S0) / (tau - tau0);
                F += interval(0.0, tau0, S0 - s0 * tau0, S0, 0.5, 1.0 / 3.0, e3_0, e4_0);
                double sc0 = (S - S0) / (tauc - tauc0);
                Fc += interval(0.0, tauc0, S0 - sc0 * tauc0, S0, 0.5, 1.0 / 3.0, e3c_0, e4c_0);
            }
            F += interval(tau_p, tau, S_p, S, e3p, e4p, e3, e4);
            Fc += interval(tauc_p, tauc, S_p, S, e3cp, e4cp, e3c, e4c);
        }
        chi_p = chi; chic_p = kc; tau_p = tau; tauc_p = tauc; S_p = S; m_p = md;
        e3p = e3; e4p = e4; e3cp = e3c; e4cp = e4c;
    }
    g.F[i] = 2.0 * kPI * F;
    g.Fc[i] = 2.0 * kPI * Fc;
}

cudaError_t launch_flux_scatter(pz_ctx *c, cudaStream_t s);

cudaError_t launch_flux(pz_ctx *c, cudaStream_t s) {
    if (c->d_sigma) return launch_flux_scatter(c, s);
    FluxArgs g;
    g.nlam = c->nlam;
    g.ld = c->ld;
    g.nd = c->nd;
    g.lam0cm = c->lambda0_nm * 1e-7;
    g.lnr = c->lnr;
    g.m = c->d_m;
    g.T = c->d_T;
    g.kc = c->d_kc;
    g.B = c->d_B;
    g.kline = c->d_kline;
    g.F = c->d_F;
    g.Fc = c->d_Fc;
    dim3 nb((unsigned)((c->nlam + 127) / 128), c->S);
    if (c->prec == PZ_MIXED)
        k_flux<float><<<nb, 128, 0, s>>>(g);
    else
        k_flux<double><<<nb, 128, 0, s>>>(g);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Scattering source function (Eq. 6): S = eps B + (1 - eps) J with eps the absorption
// fraction of the extinction and J the mean intensity of the same slab the flux is
// taken from (S linear between layers, first segment extrapolated to tau = 0, nothing
// below the bottom layer).  J = Lambda S is linear in the layer values; the iteration
// of the scattering term converges to the solution of (I - diag(1 - eps) Lambda) S = eps B,
// which is solved here directly, one CTA per (wavelength, star), both branches in turn.
//
// Lambda row j: every segment [a, b] of the source contributes
//   1/2 Int_a^b S E_1(|t - tau_j|) dt = P (Sa + Sb)/2 + Q (Sb - Sa)/2  (segment below tau_j)
// with x = t - tau_j: P = E2(xa) - E2(xb) (the weight of a constant) and
// Q = 2 (E3(xa) - E3(xb) - D E2(xb)) / D - P (the odd part), mirrored for segments above.
// Errors of Q from cancellation at tiny D multiply Sb - Sa, which is small there.
// The matrix is diagonally dominant (row sums of Lambda <= 1, 1 - eps < 1), so Gaussian
// elimination runs without pivoting.
// ---------------------------------------------------------------------------
// d/dtau_a and d/dtau_b of one interval integral at fixed endpoint values (defined with the
// LTE transfer adjoint below)
__device__ __forceinline__ void interval_grad(double ta, double tb, double Sa, double Sb, double e2a, double e3a,
                                              double e4a, double e2b, double e3b, double e4b, double &da,
                                              double &db);

struct ScatArgs {
    int64_t nlam, ld;
    int nd;
    double lam0cm, lnr;
    const double *m, *T, *kc, *sig, *B, *stim;
    const void *kline;
    double *F, *Fc;
    const double *dFbar;   // adjoint: dL/dF [S][nlam]
    void *Gt;              // adjoint: G stim [S][nd][ld]
    int *status;           // context status word: kStatusScatNoConverge if a refinement hit its limit
};

constexpr int kScatThreadsFwd = 256;     // forward CTA: a 16 x 16 grid in the inverse
constexpr int kScatThreadsAdj = 512;     // adjoint CTA: a 16 x 32 grid (one CTA per SM fits its shared memory)
constexpr int kScatTableMaxDepth = 96;    // the adjoint's (E2, E3) pair table fits shared memory up to here
constexpr int kScatMaxRefine = 12;        // iterative-refinement rounds at most
constexpr int kScatVecFwd = 10;           // FP64 vectors of nd: forward kernel
constexpr int kScatVecAdj = 20;           // FP64 vectors of nd: adjoint kernel

// Row stride of the FP32 inverse: odd, so that a warp walking a row or a column of it
// touches 32 different banks.
__host__ __device__ __forceinline__ int scat_ldm(int nd) { return nd | 1; }

// Shared memory of one (wavelength, star) column, by table layout TS:
//   1 (forward): E3 at every layer pair, one FP64 per pair of the packed triangle; the FP32
//     inverse of M takes its space once Lambda is built;
//   2 (adjoint): (E2, E3) at every pair;
//   0 (adjoint above kScatTableMaxDepth layers): no table, E_n evaluated where needed.
// Lambda [nd][nd + 1] (FP64, odd row stride; the adjoint reuses it for dJ/dtau), the FP64
// vectors, the table, one FP64 partial sum per thread, then FP32: the inverse [nd][ldm]
// (TS != 1), one partial sum per thread, the residual and the pivot row and column [4][nd].
static size_t scatter_smem(int nd, int ts, int threads) {
    const size_t W = (size_t)nd + 1;
    size_t n = (size_t)nd * W + threads + (size_t)(ts == 1 ? kScatVecFwd : kScatVecAdj) * nd;
    if (ts == 1) n += (size_t)nd * W / 2;
    if (ts == 2) n += (size_t)nd * W;
    size_t nf = threads + 5 * (size_t)nd;
    if (ts != 1) nf += (size_t)nd * scat_ldm(nd);
    return sizeof(double) * n + sizeof(float) * nf;
}

// E2, E3 at distance x from the E_3 Taylor table (two Horner chains); beyond x = 40 they
// are below e^-40 / 40 and are taken as zero (a weight there is below 1e-19 of the local
// ones)
__device__ __forceinline__ void e23(double x, double &e2, double &e3) {
    const long long xb = __double_as_longlong(x);
    if (xb >= kBits40) {           // the table ends below x = 40
        if (xb > kBits40) {
            e2 = e3 = 0.0;
        } else {
            double e4;
            expn234(x, e2, e3, e4);
        }
        return;
    }
    if (xb <= 0) {
        e2 = 1.0;
        e3 = 0.5;
        return;
    }
    if (xb < kBits2m40) {
        // E_2 = 1 + x (ln x + gamma - 1) + O(x^2), E_3 = 1/2 - x + O(x^2 ln x)
        e2 = 1.0 + x * (log(x) + (kEuler - 1.0));
        e3 = 0.5 - x;
        return;
    }
    double t;
    const double *c = g_expn3_tab + expn_node(x, t) * kExpnK;
    double p = __ldg(c + kExpnK - 1), d1 = 0.0;
#pragma unroll
    for (int k = kExpnK - 2; k >= 0; --k) {
        d1 = fma(d1, t, p);
        p = fma(p, t, __ldg(c + k));
    }
    e3 = p;
    e2 = -d1;
}

// E3 alone (one Horner chain), the same values as e23's
__device__ __forceinline__ double e3only(double x) {
    const long long xb = __double_as_longlong(x);
    if (xb >= kBits40) {
        if (xb > kBits40) return 0.0;
        double e2, e3, e4;
        expn234(x, e2, e3, e4);
        return e3;
    }
    if (xb <= 0) return 0.5;
    if (xb < kBits2m40) return 0.5 - x;
    double t;
    const double *c = g_expn3_tab + expn_node(x, t) * kExpnK;
    double p = __ldg(c + kExpnK - 1);
#pragma unroll
    for (int k = kExpnK - 2; k >= 0; --k) p = fma(p, t, __ldg(c + k));
    return p;
}

// E_1(x), x > 0: the power series -gamma - ln x - sum_k (-x)^k / (k k!) below 1, else
// (e^-x - E_2(x)) / x from the recurrence E_2 = e^-x - x E_1
__device__ __forceinline__ double e1(double x) {
    if (x < 1.0) {
        double term = 1.0, sum = 0.0;
#pragma unroll 1
        for (int k = 1; k <= 20; ++k) {
            term *= -x / k;
            sum += term / k;
        }
        return -kEuler - log(x) - sum;
    }
    if (x > 700.0) return 0.0;
    double e2, e3, e4;
    expn234(x, e2, e3, e4);
    return (exp(-x) - e2) / x;
}

// weights of the near and far ends of a segment (inverse length invD) seen from depth
// tau_j, from E2, E3 at the distances of its near (n) and far (f) ends
__device__ __forceinline__ void seg_weights(double D, double invD, double e2n, double e3n, double e2f, double e3f,
                                            double &wn, double &wf) {
    const double P = e2n - e2f;
    const double Q = 2.0 * (e3n - e3f - D * e2f) * invD - P;
    wn = 0.25 * (P - Q);
    wf = 0.25 * (P + Q);
}

// Shared-memory layout of one (wavelength, star) column.
struct ScatCol {
    int nd, W, ldm;
    double *Lam, *tau, *chi, *eps, *B, *S, *hD, *a, *e3, *e4, *res;   // both kernels
    double *e2, *invD, *mu, *J, *dF, *ge, *wx;                        // adjoint only
    double *e2top, *e3top, *e2bot;   // E2, E3 at tau_j; E2 at tau_{N-1} - tau_j
    double *ET, *p64;
    float *Mi, *p32, *r32, *piv;
};

template <int TS>
__device__ __forceinline__ ScatCol scat_carve(double *sm, int nd) {
    ScatCol c = {};
    c.nd = nd;
    c.W = nd + 1;
    c.ldm = scat_ldm(nd);
    c.Lam = sm;
    double *v = sm + (size_t)nd * c.W;
    if (TS == 1) {
        double **vec[kScatVecFwd] = {&c.tau, &c.chi, &c.eps, &c.B, &c.S, &c.hD, &c.a, &c.e3, &c.e4, &c.res};
        for (int k = 0; k < kScatVecFwd; ++k) *vec[k] = v + (size_t)k * nd;
        v += (size_t)kScatVecFwd * nd;
        // the slab-end E_n are dead before the flux writes e3, e4 and its partial sums
        c.e2top = c.e3;
        c.e3top = c.e4;
        c.e2bot = c.res;
    } else {
        double **vec[kScatVecAdj] = {&c.tau, &c.chi, &c.eps, &c.B, &c.S, &c.hD, &c.a, &c.e3, &c.e4, &c.res,
                                     &c.e2, &c.invD, &c.mu, &c.J, &c.dF, &c.ge, &c.wx, &c.e2top, &c.e3top,
                                     &c.e2bot};
        for (int k = 0; k < kScatVecAdj; ++k) *vec[k] = v + (size_t)k * nd;
        v += (size_t)kScatVecAdj * nd;
    }
    c.ET = v;
    v += TS == 1 ? (size_t)nd * c.W / 2 : (TS == 2 ? (size_t)nd * c.W : 0);
    c.p64 = v;
    float *f = reinterpret_cast<float *>(v + blockDim.x);
    if (TS == 1) {
        c.Mi = reinterpret_cast<float *>(c.ET);
    } else {
        c.Mi = f;
        f += (size_t)nd * c.ldm;
    }
    c.p32 = f;
    c.r32 = f + blockDim.x;
    c.piv = c.r32 + nd;
    return c;
}

__host__ __device__ __forceinline__ size_t pair_idx(int nd, int a, int b) {   // a <= b
    return (size_t)a * nd - (size_t)a * (a - 1) / 2 + (b - a);
}

// The split of an nd x nd product over the CTA: row j = tid % nd, part q = tid / nd of the
// columns [k0, k1); threads with q >= P idle.
struct ScatSplit {
    int P, j, q, k0, k1;
    __device__ __forceinline__ ScatSplit(int nd) {
        P = (int)blockDim.x / nd;
        const int L = (nd + P - 1) / P;
        j = threadIdx.x % nd;
        q = threadIdx.x / nd;
        k0 = min(nd, q * L);
        k1 = min(nd, k0 + L);
    }
};

// chi, eps and tau of one branch (0: total, 1: continuum); hD = 0.5 / tau_0, then 0.5 / D
// of each segment; invD (adjoint); E_n at the layer pairs by the table layout TS, and E2,
// E3 at tau_j and E2 at tau_{N-1} - tau_j.  Ends with a barrier.
template <typename KT, int TS>
__device__ void scat_columns(const ScatArgs &g, const ScatCol &c, int64_t base, const double *m, int branch) {
    const int nd = c.nd, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const KT *kl = reinterpret_cast<const KT *>(g.kline);
    for (int d = tid; d < nd; d += blockDim.x) {
        const int64_t o = base + (int64_t)d * g.ld;
        const double ka = g.kc[o] + (branch == 0 ? (double)kl[o] : 0.0);   // absorption
        c.chi[d] = ka + g.sig[o];
        c.eps[d] = ka / c.chi[d];
    }
    __syncthreads();
    // trapezoid tau: the increments by lane, then an inclusive warp scan per 32 layers
    if (warp == 0) {
        double carry = 0.0;
        for (int b = 0; b < nd; b += 32) {
            const int d = b + lane;
            double v = 0.0;
            if (d < nd) v = d == 0 ? c.chi[0] * m[0] : 0.5 * (c.chi[d - 1] + c.chi[d]) * (m[d] - m[d - 1]);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            v += carry;
            if (d < nd) c.tau[d] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    for (int k = tid; k < nd; k += blockDim.x) {
        const double inv = 1.0 / (k == 0 ? c.tau[0] : c.tau[k] - c.tau[k - 1]);
        c.hD[k] = 0.5 * inv;
        if (TS != 1 && k > 0) c.invD[k - 1] = inv;
    }
    if (TS != 0) {
        // one thread per pair a <= b of the packed triangle, p = pair_idx(nd, a, b); the row
        // a is the root of the quadratic pair_idx(nd, a, a) = p, corrected to the integer
        const int P = nd * (nd + 1) / 2;
        const float b2 = 2.0f * (float)nd + 1.0f;
        for (int p = tid; p < P; p += blockDim.x) {
            int a = (int)((b2 - sqrtf(fmaxf(b2 * b2 - 8.0f * (float)p, 0.0f))) * 0.5f);
            a = max(0, min(a, nd - 1));
            while (a > 0 && (int)pair_idx(nd, a, a) > p) --a;
            while (a + 1 < nd && (int)pair_idx(nd, a + 1, a + 1) <= p) ++a;
            const int b = a + (p - (int)pair_idx(nd, a, a));
            const double x = c.tau[b] - c.tau[a];
            if (TS == 1)
                c.ET[p] = e3only(x);
            else
                e23(x, c.ET[2 * p], c.ET[2 * p + 1]);
        }
    }
    for (int t = tid; t < 2 * nd; t += blockDim.x) {
        const bool top = t < nd;
        double e2, e3;
        e23(top ? c.tau[t] : c.tau[nd - 1] - c.tau[t - nd], e2, e3);
        if (top) {
            c.e2top[t] = e2;
            c.e3top[t] = e3;
        } else {
            c.e2bot[t - nd] = e2;
        }
    }
    __syncthreads();
}

// E3(|tau_k - tau_j|) (table or direct)
template <int TS>
__device__ __forceinline__ double scat_g3(const ScatCol &c, int j, int k) {
    if (TS == 0) return e3only(fabs(c.tau[k] - c.tau[j]));
    const size_t idx = pair_idx(c.nd, min(j, k), max(j, k));
    return TS == 1 ? c.ET[idx] : c.ET[2 * idx + 1];
}

// E2, E3 at |tau_k - tau_j| (adjoint table or direct)
template <int TS>
__device__ __forceinline__ void scat_E(const ScatCol &c, int j, int k, double &e2, double &e3) {
    if (TS == 2) {
        const size_t idx = pair_idx(c.nd, min(j, k), max(j, k));
        e2 = c.ET[2 * idx];
        e3 = c.ET[2 * idx + 1];
    } else {
        e23(fabs(c.tau[k] - c.tau[j]), e2, e3);
    }
}

// Rows of Lambda (J = Lambda S) and the right-hand side a = eps B.
//
// With G(t) = E3(|t - tau_j|)/2 + |t - tau_j|/2, G'' = E1(|t - tau_j|)/2 and G' is
// continuous, so the integral of a hat function against the kernel is the second divided
// difference of G over its three nodes.  With qt_k = (E3(|tau_{k+1} - tau_j|) - E3(|tau_k -
// tau_j|)) / (2 D_k) (the E3 part of G's difference quotient over segment k; qt_{-1} over
// [0, tau_0]) the |t - tau_j| part contributes 1 to the diagonal and nothing else:
//   Lambda_jk = qt_k - qt_{k-1} + [k = j]                          (k < N - 1),
//   Lambda_j,N-1 = G'(tau_{N-1}^-) - qt_{N-2}, G' = -E2(tau_{N-1} - tau_j)/2 (j < N - 1), 1/2 (j = N - 1),
// and the top segment's weight of S(0) is wz = qt_{-1} - E2(tau_j)/2, carried to layers 0
// and 1 by the extrapolation S(0) = S_0 (1 + tau_0/D_0) - S_1 tau_0/D_0.  The same sums the
// segment weights P, Q of the formulation above, three FP64 operations per element.
// Threads over (row, part of the row).  Ends with a barrier.
template <int TS>
__device__ void scat_lambda(const ScatCol &c) {
    const int nd = c.nd, W = c.W;
    const ScatSplit sp(nd);
    if (sp.q < sp.P && sp.k0 < sp.k1) {
        const int j = sp.j;
        double *row = c.Lam + (size_t)j * W;
        double ecur, qprev;   // E3 at node k, qt_{k-1}
        if (sp.k0 == 0) {
            ecur = scat_g3<TS>(c, j, 0);
            qprev = (ecur - c.e3top[j]) * c.hD[0];
        } else {
            const double em = scat_g3<TS>(c, j, sp.k0 - 1);
            ecur = scat_g3<TS>(c, j, sp.k0);
            qprev = (ecur - em) * c.hD[sp.k0];
        }
        for (int k = sp.k0; k < sp.k1; ++k) {
            double v;
            if (k + 1 < nd) {
                const double en = scat_g3<TS>(c, j, k + 1);
                const double qk = (en - ecur) * c.hD[k + 1];
                v = qk - qprev;
                if (k == j) v += 1.0;
                qprev = qk;
                ecur = en;
            } else {
                v = (j + 1 < nd ? -0.5 * c.e2bot[j] : 0.5) - qprev;
            }
            row[k] = v;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nd; j += blockDim.x) {
        double *row = c.Lam + (size_t)j * W;
        const double wz = (scat_g3<TS>(c, j, 0) - c.e3top[j]) * c.hD[0] - 0.5 * c.e2top[j];
        const double r = c.tau[0] / (c.tau[1] - c.tau[0]);
        row[0] += wz * (1.0 + r);
        row[1] -= wz * r;
        c.a[j] = c.eps[j] * c.B[j];
        // the diagonal of M in FP64 before rounding: where the slab is optically thick and
        // eps below the FP32 resolution, 1 - (1 - eps) Lambda_jj is far below FP32's
        // spacing near 1 and would otherwise round to zero
        c.p32[j] = (float)(1.0 - (1.0 - c.eps[j]) * row[j]);
    }
    __syncthreads();
}

// Segment weights of row j: for every segment k (between layers k and k + 1) the weights
// (wa, wb) of its lower and upper layer values, and of the top segment [0, tau_0] the
// weights (wlo, whi) of S(0) and S(tau_0).  f(k, wa, wb) per segment, then top(wlo, whi).
template <int TS, class Seg, class Top>
__device__ __forceinline__ void scat_row_weights(const ScatCol &c, int j, Seg &&seg, Top &&top) {
    const int nd = c.nd;
    double e2p, e3p;
    scat_E<TS>(c, j, 0, e2p, e3p);
    {
        double wn, wf;
        seg_weights(c.tau[0], 1.0 / c.tau[0], e2p, e3p, c.e2top[j], c.e3top[j], wn, wf);   // near: tau_0, far: 0
        top(wf, wn);
    }
    for (int k = 0; k + 1 < nd; ++k) {
        double e2k, e3k, wn, wf;
        scat_E<TS>(c, j, k + 1, e2k, e3k);
        const double D = c.tau[k + 1] - c.tau[k];
        if (k >= j) {          // below tau_j: near end k, far end k + 1
            seg_weights(D, c.invD[k], e2p, e3p, e2k, e3k, wn, wf);
            seg(k, wn, wf);
        } else {               // above: near end k + 1, far end k
            seg_weights(D, c.invD[k], e2k, e3k, e2p, e3p, wn, wf);
            seg(k, wf, wn);
        }
        e2p = e2k;
        e3p = e3k;
    }
}

// FP32 inverse of M = I - diag(1 - eps) Lambda by Gauss-Jordan elimination in place,
// without pivoting (M is diagonally dominant); the diagonal of M comes from scat_lambda
// (FP64, in p32), the off-diagonal elements are formed in FP32.  The CTA is a 16 x TX grid of threads;
// thread (ty, tx) holds the elements of rows ty + 16 i (i < RT) and columns tx + TX jj
// (jj < CT) in registers.  Step p replaces every element by a_rk - f_r g_k with
//   f_r = (a_rp - [r = p]) / a_pp,  g_k = a_pk + [k = p],
// which gives the scaled pivot row a_pk / a_pp, the column -a_rp / a_pp and 1 / a_pp on
// the diagonal in the same fused multiply-add as the rest.  The pivot row and column of
// step p + 1 are copied to double-buffered vectors by their owners, one barrier per
// step.  Ends with the inverse in Mi and a barrier.
template <int RT, int CT, int TX>
__device__ void scat_inverse(const ScatCol &c) {
    const int nd = c.nd, ld = c.ldm, W = c.W, tid = threadIdx.x;
    const int ty = tid / TX, tx = tid - ty * TX;
    float *colb = c.piv, *rowb = c.piv + 2 * nd;
    float a[RT][CT];
#pragma unroll
    for (int i = 0; i < RT; ++i) {
        const int r = ty + 16 * i;
        const float w = r < nd ? (float)(1.0 - c.eps[r]) : 0.0f;
#pragma unroll
        for (int jj = 0; jj < CT; ++jj) {
            const int k = tx + TX * jj;
            a[i][jj] = (r < nd && k < nd) ? (r == k ? c.p32[r] : -w * (float)c.Lam[(size_t)r * W + k]) : 0.0f;
        }
    }
    if (ty == 0) {
#pragma unroll
        for (int jj = 0; jj < CT; ++jj)
            if (tx + TX * jj < nd) rowb[tx + TX * jj] = a[0][jj];
    }
    if (tx == 0) {
#pragma unroll
        for (int i = 0; i < RT; ++i)
            if (ty + 16 * i < nd) colb[ty + 16 * i] = a[i][0];
    }
    __syncthreads();
    for (int p = 0; p < nd; ++p) {
        const int par = p & 1;
        const float *cb = colb + par * nd, *rb = rowb + par * nd;
        float *cn = colb + (par ^ 1) * nd, *rn = rowb + (par ^ 1) * nd;
        // a pivot that rounds to zero (M singular to FP32) skips its step: the result
        // stays finite, and the refinement that cannot converge with it reports
        const float piv = rb[p];
        const float inv = fabsf(piv) >= 1e-30f ? __frcp_rn(piv) : 0.0f;
        float f[RT], g[CT];
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            const int r = ty + 16 * i;
            f[i] = r < nd ? (cb[r] - (r == p ? 1.0f : 0.0f)) * inv : 0.0f;
        }
#pragma unroll
        for (int jj = 0; jj < CT; ++jj) {
            const int k = tx + TX * jj;
            g[jj] = k < nd ? rb[k] + (k == p ? 1.0f : 0.0f) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int jj = 0; jj < CT; ++jj) a[i][jj] = fmaf(-f[i], g[jj], a[i][jj]);
        const int pn = p + 1;
        if (pn < nd) {
            if (ty == (pn & 15)) {
                const int in = pn >> 4;
#pragma unroll
                for (int i = 0; i < RT; ++i)
                    if (i == in) {
#pragma unroll
                        for (int jj = 0; jj < CT; ++jj)
                            if (tx + TX * jj < nd) rn[tx + TX * jj] = a[i][jj];
                    }
            }
            if (tx == pn % TX) {
                const int jn = pn / TX;
#pragma unroll
                for (int jj = 0; jj < CT; ++jj)
                    if (jj == jn) {
#pragma unroll
                        for (int i = 0; i < RT; ++i)
                            if (ty + 16 * i < nd) cn[ty + 16 * i] = a[i][jj];
                    }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int jj = 0; jj < CT; ++jj) {
            const int r = ty + 16 * i, k = tx + TX * jj;
            if (r < nd && k < nd) c.Mi[r * ld + k] = a[i][jj];
        }
    __syncthreads();
}

// out_j = sum_k A[j][k] x_k (TRANS: sum_k A[k][j] x_k) in FP64, A with the row stride of
// Lambda, split over (row, part) and summed over the parts in a fixed order.  Ends with a
// barrier.
template <bool TRANS>
__device__ void scat_matvec(const ScatCol &c, const double *A, const double *x, double *out) {
    const int nd = c.nd, W = c.W;
    const ScatSplit sp(nd);
    if (sp.q < sp.P) {
        double acc = 0.0;
        for (int k = sp.k0; k < sp.k1; ++k)
            acc = fma(TRANS ? A[(size_t)k * W + sp.j] : A[(size_t)sp.j * W + k], x[k], acc);
        c.p64[sp.q * nd + sp.j] = acc;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
        double s = 0.0;
        for (int u = 0; u < sp.P; ++u) s += c.p64[u * nd + d];
        out[d] = s;
    }
    __syncthreads();
}

// Iterative refinement with FP64 residuals of M x = rhs (TRANS false) or M^T x = rhs:
// x += M^-1 (rhs - M x) with the FP32 inverse until the correction is below 1e-12 of x
// (it is applied, so what remains is that times the contraction per round, ~cond(M) 2^-24),
// or until it stops shrinking (at least halving per round after the second), which is
// where FP64 residuals of an ill-conditioned M (eps near 0) leave it.  A solve that
// stops with a last correction above 1e-9 of x (stalled there, growing, or out of
// rounds) sets kStatusScatNoConverge in the context's status word (read by
// pz_sync_status).  Both products are split like scat_matvec.  With TRANS, wx holds
// diag(1 - eps) x of the final x on return.
template <bool TRANS>
__device__ void scat_refine(const ScatCol &c, const double *rhs, double *x, int *s_done, int *status) {
    const int nd = c.nd, W = c.W, ld = c.ldm, tid = threadIdx.x;
    const ScatSplit sp(nd);
    __shared__ double s_dprev;
    for (int d = tid; d < nd; d += blockDim.x) {
        x[d] = 0.0;
        c.r32[d] = (float)rhs[d];
    }
    if (tid == 0) s_dprev = 0.0;
    __syncthreads();
    for (int it = 0; it < kScatMaxRefine; ++it) {
        if (sp.q < sp.P) {       // y = M^-1 r (M^-T r), FP32
            float acc = 0.0f;
            for (int k = sp.k0; k < sp.k1; ++k)
                acc = fmaf(TRANS ? c.Mi[k * ld + sp.j] : c.Mi[sp.j * ld + k], c.r32[k], acc);
            c.p32[sp.q * nd + sp.j] = acc;
        }
        __syncthreads();
        if (tid < 32) {
            double dmax = 0.0, smax = 0.0;
            for (int row = tid; row < nd; row += 32) {
                float y = 0.0f;
                for (int u = 0; u < sp.P; ++u) y += c.p32[u * nd + row];
                const double v = x[row] + (double)y;
                x[row] = v;
                if (TRANS) c.wx[row] = (1.0 - c.eps[row]) * v;
                dmax = fmax(dmax, fabs((double)y));
                smax = fmax(smax, fabs(v));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
                smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
            }
            if (tid == 0) {
                const bool conv = dmax <= 1e-12 * smax;
                const bool stop = conv || (it >= 2 && dmax >= 0.5 * s_dprev) || it + 1 == kScatMaxRefine;
                if (stop && !conv && dmax > 1e-9 * smax && status) atomicOr(status, kStatusScatNoConverge);
                s_dprev = dmax;
                *s_done = stop;
            }
        }
        __syncthreads();
        if (*s_done) break;
        if (sp.q < sp.P) {       // Lambda x (Lambda^T diag(1 - eps) x), FP64
            double acc = 0.0;
            if (!TRANS) {
                const double *row = c.Lam + (size_t)sp.j * W;
                for (int k = sp.k0; k < sp.k1; ++k) acc = fma(row[k], x[k], acc);
            } else {
                for (int k = sp.k0; k < sp.k1; ++k) acc = fma(c.Lam[(size_t)k * W + sp.j], c.wx[k], acc);
            }
            c.p64[sp.q * nd + sp.j] = acc;
        }
        __syncthreads();
        for (int d = tid; d < nd; d += blockDim.x) {
            double lx = 0.0;
            for (int u = 0; u < sp.P; ++u) lx += c.p64[u * nd + d];
            const double r0 = rhs[d] - x[d];
            c.r32[d] = (float)(TRANS ? r0 + lx : fma(1.0 - c.eps[d], lx, r0));
        }
        __syncthreads();
    }
}

// Forward: one CTA per (wavelength, star), both branches in turn; three CTAs fit an SM up
// to 80 layers (RT = 5: rows and columns of the inverse per thread in each direction).
template <typename KT, int RT>
__global__ void __launch_bounds__(kScatThreadsFwd, RT <= 5 ? 3 : 1) k_flux_scatter(ScatArgs g) {
    extern __shared__ double sm[];
    __shared__ int s_done;
    const int nd = g.nd;
    const ScatCol c = scat_carve<1>(sm, nd);
    const int64_t i = blockIdx.x;
    const int st = blockIdx.y;
    const int tid = threadIdx.x;
    const double *m = g.m + (int64_t)st * nd;
    const int64_t base = (int64_t)st * nd * g.ld + i;
    for (int d = tid; d < nd; d += blockDim.x) c.B[d] = g.B[base + (int64_t)d * g.ld];
    for (int branch = 0; branch < 2; ++branch) {
        scat_columns<KT, 1>(g, c, base, m, branch);
        scat_lambda<1>(c);
        scat_inverse<RT, RT, 16>(c);
        scat_refine<false>(c, c.a, c.S, &s_done, g.status);
        // emergent flux of the solved source, the closed form of the LTE kernel
        for (int d = tid; d < nd; d += blockDim.x) expn34(c.tau[d], c.e3[d], c.e4[d]);
        __syncthreads();
        // interval d (layers d, d + 1; for d = 0 also the top one [0, tau_0]) by thread d,
        // summed by warp 0 in a fixed order
        for (int d = tid; d < nd; d += blockDim.x) {
            double v = 0.0;
            if (d + 1 < nd) {   // interval() with the slope from the stored reciprocal 1/D = 2 hD
                const double D = c.tau[d + 1] - c.tau[d];
                const double sl = (c.S[d + 1] - c.S[d]) * (2.0 * c.hD[d + 1]);
                v = c.S[d] * (c.e3[d] - c.e3[d + 1]) + sl * (c.e4[d] - c.e4[d + 1] - D * c.e3[d + 1]);
            }
            if (d == 0) {
                const double s0 = (c.S[1] - c.S[0]) / (c.tau[1] - c.tau[0]);
                v += interval(0.0, c.tau[0], c.S[0] - s0 * c.tau[0], c.S[0], 0.5, 1.0 / 3.0, c.e3[0], c.e4[0]);
            }
            c.res[d] = v;
        }
        __syncthreads();
        if (tid < 32) {
            double F = 0.0;
            for (int d = tid; d < nd; d += 32) F += c.res[d];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) F += __shfl_xor_sync(0xffffffffu, F, o);
            if (tid == 0) (branch == 0 ? g.F : g.Fc)[(int64_t)st * g.nlam + i] = 2.0 * kPI * F;
        }
        __syncthreads();
    }
}

// Reverse pass of the total branch through the scattering source (Eq. 6), one CTA per
// (wavelength, star).  With M S = eps B solved again, dF/dS = a and the explicit dF/dtau
// at fixed S, the adjoint mu solves M^T mu = dL/dF a; then
//   dL/deps_j = mu_j (B_j - J_j),  J = Lambda S,
//   dL/dtau_m = dL/dF dF/dtau_m + sum_j mu_j (1 - eps_j) dJ_j/dtau_m,
// with dJ_j/dtau_m (S fixed) from moving layer m: minus the slope times the layer's
// weight in each adjacent segment, the slab-end term 1/2 S_{N-1} E_1(tau_{N-1} - tau_j) at
// the bottom layer, the top segment's extrapolation terms, and the diagonal from
// translation invariance (the row sums to 1/2 S(0) E_1(tau_j)).  Through the trapezoid and
// eps = 1 - sigma/chi: G_d = dL/dchi_d + dL/deps_d sigma_d / chi_d^2, stored as G stim.
template <typename KT, typename GT, int TS, int RT, int CT>
__global__ void __launch_bounds__(kScatThreadsAdj, 1) k_rt_adjoint_scatter(ScatArgs g) {
    extern __shared__ double sm[];
    __shared__ int s_done;
    const int nd = g.nd, W = nd + 1;
    const ScatCol c = scat_carve<TS>(sm, nd);
    const int64_t i = blockIdx.x;
    const int st = blockIdx.y;
    const int tid = threadIdx.x;
    const double *m = g.m + (int64_t)st * nd;
    const int64_t base = (int64_t)st * nd * g.ld + i;
    const double Fb = g.dFbar[(int64_t)st * g.nlam + i];
    for (int d = tid; d < nd; d += blockDim.x) c.B[d] = g.B[base + (int64_t)d * g.ld];
    scat_columns<KT, TS>(g, c, base, m, 0);
    scat_lambda<TS>(c);
    scat_inverse<RT, CT, 32>(c);
    scat_refine<false>(c, c.a, c.S, &s_done, g.status);
    // J = Lambda S, E_n at the layers
    scat_matvec<false>(c, c.Lam, c.S, c.J);
    for (int j = tid; j < nd; j += blockDim.x) expn234(c.tau[j], c.e2[j], c.e3[j], c.e4[j]);
    __syncthreads();
    // dF/dS (a, times dL/dF) and dF/dtau at fixed S (dF), both with the 2 pi of the flux.
    // Each interval (d, d + 1) once (the terms of interval_grad), its shares of its lower
    // and upper layer kept in vectors that are dead here (e2bot) or not yet written (ge;
    // mu, wx: the transposed solve's).
    const double D1 = c.tau[1] - c.tau[0];
    const double t0 = c.tau[0];
    const double s0 = (c.S[1] - c.S[0]) / D1;
    double *a_lo = c.e2bot, *a_hi = c.ge, *f_lo = c.mu, *f_hi = c.wx;
    for (int d = tid; d + 1 < nd; d += blockDim.x) {
        const double iD = c.invD[d], D = c.tau[d + 1] - c.tau[d];
        const double sl = (c.S[d + 1] - c.S[d]) * iD;
        const double P = c.e3[d] - c.e3[d + 1];
        const double Bq = c.e4[d] - c.e4[d + 1] - D * c.e3[d + 1];
        const double q = Bq * iD;
        a_lo[d] = P - q;
        a_hi[d] = q;
        f_lo[d] = -c.S[d] * c.e2[d] + (sl * iD) * Bq - sl * P;
        f_hi[d] = c.S[d + 1] * c.e2[d + 1] - (sl * iD) * Bq;
    }
    __syncthreads();
    for (int d = tid; d < nd; d += blockDim.x) {
        double a = 0.0, df = 0.0;
        if (d + 1 < nd) {   // interval (d, d + 1), d its lower end
            a += a_lo[d];
            df += f_lo[d];
        }
        if (d >= 1) {       // interval (d - 1, d), d its upper end
            a += a_hi[d - 1];
            df += f_hi[d - 1];
        }
        if (d <= 1) {       // top interval [0, tau_0] with S(0) = S0 - s0 tau_0
            const double qt = (1.0 / 3.0 - c.e4[0] - t0 * c.e3[0]) / t0;
            const double az = (0.5 - c.e3[0]) - qt;      // coefficient of S(0)
            const double sp = s0 / D1;
            const double Pt = 0.5 - c.e3[0];
            const double Bt = 1.0 / 3.0 - c.e4[0] - t0 * c.e3[0];
            if (d == 0) {
                a += qt + az * (1.0 + t0 / D1);
                df += -s0 * Pt + sp * (Bt - t0 * Pt) + c.S[0] * c.e2[0];
            } else {
                a += -az * t0 / D1;
                df += -sp * (Bt - t0 * Pt);
            }
        }
        c.a[d] = 2.0 * kPI * Fb * a;
        c.dF[d] = 2.0 * kPI * Fb * df;
    }
    __syncthreads();
    scat_refine<true>(c, c.a, c.mu, &s_done, g.status);
    // dJ_j/dtau_m into the Lambda area (Lambda is no longer needed), off-diagonal elements
    // by (row, part).  Moving layer k at fixed S_k changes S(t) by -S'(t) times its hat
    // function, so element k is -s_{k-1} wb_{k-1} - s_k wa_k (s the segment slopes, wa/wb
    // the weights of a segment's lower and upper layer).  In the divided-difference form of
    // the Lambda pass (wb_{k-1} = G'_k - Q_{k-1}, wa_k = Q_k - G'_k with G' continuous), for
    // an inner layer k != j the |t - tau_j| parts cancel and
    //   dJ_j/dtau_k = -sgn(k - j) E2(|tau_k - tau_j|)/2 (s_k - s_{k-1}) + s_{k-1} qt_{k-1} - s_k qt_k,
    // qt as in scat_lambda; layers 0 and N - 1 take the segment weights directly, plus the top
    // segment's terms at k <= 1 (S(0) extrapolated) and the slab end at k = N - 1.  Then the
    // diagonal from the row sums.
    const double Szero = c.S[0] - s0 * t0;
    for (int k = tid; k < nd; k += blockDim.x) {   // slopes and their steps (a, e2bot are free here)
        const double sk = k + 1 < nd ? (c.S[k + 1] - c.S[k]) * c.invD[k] : 0.0;
        c.a[k] = sk;
        c.e2bot[k] = (k >= 1 && k + 1 < nd) ? sk - (c.S[k] - c.S[k - 1]) * c.invD[k - 1] : 0.0;
    }
    __syncthreads();
    {
        const double *sl = c.a, *ds = c.e2bot;
        const ScatSplit sp(nd);
        if (sp.q < sp.P && sp.k0 < sp.k1) {
            const int j = sp.j;
            double *row = c.Lam + (size_t)j * W;
            double e3c = scat_g3<TS>(c, j, sp.k0), sqp = 0.0;   // E3 at k, s_{k-1} qt_{k-1}
            if (sp.k0 >= 1) sqp = sl[sp.k0 - 1] * ((e3c - scat_g3<TS>(c, j, sp.k0 - 1)) * c.hD[sp.k0]);
            double off = 0.0;
            for (int k = sp.k0; k < sp.k1; ++k) {
                double e3n = 0.0, sq = 0.0;
                if (k + 1 < nd) {
                    e3n = scat_g3<TS>(c, j, k + 1);
                    sq = sl[k] * ((e3n - e3c) * c.hD[k + 1]);
                }
                if (k != j) {
                    double v;
                    if (k == 0 || k == nd - 1) {   // the end layers: one segment's weight
                        const int kk = k == 0 ? 0 : nd - 2;
                        double e2a, e3a, e2b, e3b, wn, wf;
                        scat_E<TS>(c, j, kk, e2a, e3a);
                        scat_E<TS>(c, j, kk + 1, e2b, e3b);
                        const double D = c.tau[kk + 1] - c.tau[kk];
                        if (kk >= j)
                            seg_weights(D, c.invD[kk], e2a, e3a, e2b, e3b, wn, wf);   // wa = wn, wb = wf
                        else
                            seg_weights(D, c.invD[kk], e2b, e3b, e2a, e3a, wf, wn);   // wa = wn, wb = wf
                        v = -sl[kk] * (k == kk ? wn : wf);
                        if (k == nd - 1) v += 0.5 * c.S[nd - 1] * e1(c.tau[nd - 1] - c.tau[j]);
                    } else {
                        double e2k, e3k;
                        scat_E<TS>(c, j, k, e2k, e3k);
                        v = fma(k > j ? -0.5 * e2k : 0.5 * e2k, ds[k], sqp - sq);
                    }
                    if (k <= 1) {   // the top segment [0, tau_0] with the extrapolated S(0)
                        double e20, e30, whi, wlo;
                        scat_E<TS>(c, j, 0, e20, e30);
                        seg_weights(t0, 1.0 / t0, e20, e30, c.e2top[j], c.e3top[j], whi, wlo);   // near: tau_0, far: 0
                        v += k == 0 ? -(s0 / D1) * t0 * wlo - s0 * (wlo + whi) : (s0 / D1) * t0 * wlo;
                    }
                    row[k] = v;
                    off += v;
                }
                e3c = e3n;
                sqp = sq;
            }
            c.p64[sp.q * nd + j] = off;
        }
        __syncthreads();
        for (int j = tid; j < nd; j += blockDim.x) {
            double off = 0.0;
            for (int u = 0; u < sp.P; ++u) off += c.p64[u * nd + j];
            c.Lam[(size_t)j * W + j] = 0.5 * Szero * e1(c.tau[j]) - off;
        }
        __syncthreads();
    }
    // dL/dtau_m = dF_m + sum_j mu_j (1 - eps_j) dJ_j/dtau_m (wx holds mu (1 - eps)), and dL/deps
    scat_matvec<true>(c, c.Lam, c.wx, c.res);
    for (int mm = tid; mm < nd; mm += blockDim.x) {
        c.res[mm] += c.dF[mm];
        c.ge[mm] = c.mu[mm] * (c.B[mm] - c.J[mm]);
    }
    __syncthreads();
    // through the trapezoid and eps = 1 - sigma/chi: the suffix sums T_d = sum_{k >= d}
    // dL/dtau_k by a warp scan from the bottom layer up (exclusive ones in a, inclusive in
    // e3), then layer d by thread d
    if (tid < 32) {
        double carry = 0.0;
        for (int b = 0; b < nd; b += 32) {
            const int d = nd - 1 - (b + tid);
            double v = d >= 0 ? c.res[d] : 0.0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double u = __shfl_up_sync(0xffffffffu, v, o);
                if (tid >= o) v += u;
            }
            v += carry;
            const double prev = __shfl_up_sync(0xffffffffu, v, 1);
            if (d >= 0) {
                c.a[d] = tid == 0 ? carry : prev;
                c.e3[d] = v;
            }
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    GT *Gt = reinterpret_cast<GT *>(g.Gt) + (int64_t)st * nd * g.ld + i;
    for (int d = tid; d < nd; d += blockDim.x) {
        const double Tn = c.a[d], Td = c.e3[d];
        double gch = 0.0;
        if (d + 1 < nd) gch += 0.5 * (m[d + 1] - m[d]) * Tn;
        if (d >= 1) gch += 0.5 * (m[d] - m[d - 1]) * Td;
        else gch += m[0] * Td;
        const double sig = g.sig[base + (int64_t)d * g.ld];
        gch += c.ge[d] * sig / (c.chi[d] * c.chi[d]);
        Gt[(int64_t)d * g.ld] = (GT)(gch * g.stim[base + (int64_t)d * g.ld]);
    }
}

// Dynamic shared memory granted to a kernel so far, per device.
static cudaError_t scatter_attr(pz_ctx *c, const void *fn, int slot, size_t smem) {
    static std::atomic<size_t> granted[kMaxDevices][10];
    if (c->device < 0 || c->device >= kMaxDevices) return cudaErrorInvalidDevice;
    if (smem <= granted[c->device][slot].load()) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) granted[c->device][slot].store(smem);
    return e;
}

static ScatArgs scatter_args(pz_ctx *c) {
    ScatArgs g;
    g.nlam = c->nlam;
    g.ld = c->ld;
    g.nd = c->nd;
    g.lam0cm = c->lambda0_nm * 1e-7;
    g.lnr = c->lnr;
    g.m = c->d_m;
    g.T = c->d_T;
    g.kc = c->d_kc;
    g.sig = c->d_sigma;
    g.B = c->d_B;
    g.stim = c->d_stim;
    g.kline = c->d_kline;
    g.F = c->d_F;
    g.Fc = c->d_Fc;
    g.dFbar = c->d_dFbar;
    g.Gt = c->prec == PZ_MIXED ? (void *)c->d_Gt : (void *)c->d_Gt64;
    g.status = c->d_status;
    return g;
}

template <typename K>
static cudaError_t launch_scat_kernel(pz_ctx *c, K *fn, int slot, int threads, size_t smem, cudaStream_t s) {
    cudaError_t e = scatter_attr(c, (const void *)fn, slot, smem);
    if (e != cudaSuccess) return e;
    fn<<<dim3((unsigned)c->nlam, c->S), threads, smem, s>>>(scatter_args(c));
    c->launches++;
    return cudaGetLastError();
}

// Instantiations: RT = 5 (16 x 5 = 80 rows of the inverse) up to 80 layers, else 8 (128).
cudaError_t launch_flux_scatter(pz_ctx *c, cudaStream_t s) {
    const size_t smem = scatter_smem(c->nd, 1, kScatThreadsFwd);
    const int T = kScatThreadsFwd;
    if (c->nd <= 80)
        return c->prec == PZ_MIXED ? launch_scat_kernel(c, k_flux_scatter<float, 5>, 0, T, smem, s)
                                   : launch_scat_kernel(c, k_flux_scatter<double, 5>, 1, T, smem, s);
    return c->prec == PZ_MIXED ? launch_scat_kernel(c, k_flux_scatter<float, 8>, 2, T, smem, s)
                               : launch_scat_kernel(c, k_flux_scatter<double, 8>, 3, T, smem, s);
}

cudaError_t launch_rt_adjoint_scatter(pz_ctx *c, cudaStream_t s) {
    const bool mixed = c->prec == PZ_MIXED;
    const int T = kScatThreadsAdj;
    if (c->nd <= 80) {
        const size_t smem = scatter_smem(c->nd, 2, T);
        return mixed ? launch_scat_kernel(c, k_rt_adjoint_scatter<float, float, 2, 5, 3>, 4, T, smem, s)
                     : launch_scat_kernel(c, k_rt_adjoint_scatter<double, double, 2, 5, 3>, 5, T, smem, s);
    }
    if (c->nd <= kScatTableMaxDepth) {
        const size_t smem = scatter_smem(c->nd, 2, T);
        return mixed ? launch_scat_kernel(c, k_rt_adjoint_scatter<float, float, 2, 8, 4>, 6, T, smem, s)
                     : launch_scat_kernel(c, k_rt_adjoint_scatter<double, double, 2, 8, 4>, 7, T, smem, s);
    }
    const size_t smem = scatter_smem(c->nd, 0, T);
    return mixed ? launch_scat_kernel(c, k_rt_adjoint_scatter<float, float, 0, 8, 4>, 8, T, smem, s)
                 : launch_scat_kernel(c, k_rt_adjoint_scatter<double, double, 0, 8, 4>, 9, T, smem, s);
}

// ---------------------------------------------------------------------------
// instrument: banded Gaussian weights, one row per pixel
// ---------------------------------------------------------------------------
__global__ void k_inst_build(int64_t n_pix, const double *pix, double v_r, double v_b, double R_lsf,
                             double lam0nm, double lnr, int64_t nlam, int32_t max_taps, int32_t *tap0,
                             int32_t *ntap, float *w, int32_t *err) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pix) return;
    double sig_lsf = 1.0 / (2.0 * sqrt(2.0 * log(2.0)) * R_lsf);
    double sig_b = v_b * 1e5 / kC;
    double sig = sqrt(sig_lsf * sig_lsf + sig_b * sig_b) / lnr;
    double rest = pix[p] / (1.0 + v_r * 1e5 / kC);
    double cp = log(rest / lam0nm) / lnr;
    int64_t i0 = (int64_t)ceil(cp - 5.0 * sig), i1 = (int64_t)floor(cp + 5.0 * sig);
    if (i0 < 0) i0 = 0;
    if (i1 > nlam - 1) i1 = nlam - 1;
    int64_t n = i1 - i0 + 1;
    if (n <= 0 || n > max_taps) {
        atomicExch(err, 1);
        tap0[p] = 0;
        ntap[p] = 0;
        return;
    }
    double sum = 0.0;
    for (int64_t i = i0; i <= i1; ++i) {
        double u = ((double)i - cp) / sig;
        sum += exp(-0.5 * u * u);
    }
    double inv = 1.0 / sum;
    float *row = w + p * max_taps;
    for (int64_t i = i0; i <= i1; ++i) {
        double u = ((double)i - cp) / sig;
        row[i - i0] = (float)(exp(-0.5 * u * u) * inv);
    }
    tap0[p] = (int32_t)i0;
    ntap[p] = (int32_t)n;
}

cudaError_t launch_inst_build(pz_ctx *c, const double *d_pix, double v_r, double v_b, double R_lsf, int32_t *d_err,
                              cudaStream_t s) {
    k_inst_build<<<(unsigned)((c->n_pix + 127) / 128), 128, 0, s>>>(
        c->n_pix, d_pix, v_r, v_b, R_lsf, c->lambda0_nm, c->lnr, c->nlam, c->max_taps, c->d_tap0, c->d_ntap,
        c->d_tapw, d_err);
    c->launches++;
    return cudaGetLastError();
}

// one warp per (pixel, star): lanes stride over the taps, FP64 sums reduced by shuffles
__global__ void k_inst_apply(int64_t nlam, int64_t n_pix, int32_t max_taps, const int32_t *tap0, const int32_t *ntap,
                             const float *w, const double *F, const double *Fc, double *g, double *gc, float *f) {
    int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (p >= n_pix) return;
    {
        const int64_t st = blockIdx.y;
        F += st * nlam;
        Fc += st * nlam;
        g += st * n_pix;
        gc += st * n_pix;
        if (f) f += st * n_pix;
    }
    int32_t i0 = tap0[p], n = ntap[p];
    const float *row = w + p * max_taps;
    double s = 0.0, sc = 0.0;
    for (int k = lane; k < n; k += 32) {
        double wk = row[k];
        s += wk * F[i0 + k];
        sc += wk * Fc[i0 + k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
    }
    if (lane == 0) {
        g[p] = s;
        gc[p] = sc;
        if (f) f[p] = (float)(s / sc);
    }
}

__global__ void k_identity_apply(int64_t n, const double *F, const double *Fc, double *g, double *gc, float *f) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    g[i] = F[i];
    gc[i] = Fc[i];
    if (f) f[i] = (float)(F[i] / Fc[i]);
}

cudaError_t launch_inst_apply(pz_ctx *c, float *f, cudaStream_t s) {
    if (c->identity_inst) {
        const int64_t n = (int64_t)c->S * c->nlam;
        k_identity_apply<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c->d_F, c->d_Fc, c->d_g, c->d_gc, f);
    } else {
        int64_t threads = c->n_pix * 32;
        dim3 grid((unsigned)((threads + 255) / 256), c->S);
        k_inst_apply<<<grid, 256, 0, s>>>(c->nlam, c->n_pix, c->max_taps, c->d_tap0, c->d_ntap, c->d_tapw, c->d_F,
                                          c->d_Fc, c->d_g, c->d_gc, f);
    }
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// chi-square objective and its seed
// ---------------------------------------------------------------------------
__global__ void k_loss(int64_t n, const double *g, const double *gc, const float *y, const float *w, double *loss,
                       float *dLdf) {
    __shared__ double red[8];
    double acc = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        double f = g[p] / gc[p];
        double wp = w ? (double)w[p] : 1.0;
        double r = (double)y[p] - f;
        acc += wp * r * r;
        if (dLdf) dLdf[p] = (float)(-2.0 * wp * r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && loss) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        atomicAdd(loss, t);
    }
}

cudaError_t launch_loss(pz_ctx *c, const float *y, const float *w, int64_t n, double *loss, float *dLdf,
                        cudaStream_t s) {
    int nb = (int)((n + 255) / 256);
    if (nb > 1024) nb = 1024;
    if (nb < 1) nb = 1;
    k_loss<<<nb, 256, 0, s>>>(n, c->d_g, c->d_gc, y, w, loss, dLdf);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// instrument adjoint: dL/dF_i = sum_p K_pi (dL/df_p) / (K F_c)_p
// one thread per grid point; the pixels whose taps cover i form a contiguous
// range because both tap0_p and tap0_p + ntap_p - 1 are non-decreasing in p.
// ---------------------------------------------------------------------------
__global__ void k_inst_adjoint(int64_t nlam, int64_t n_pix, int32_t max_taps, const int32_t *tap0,
                               const int32_t *ntap, const float *w, const double *gc, const float *dLdf,
                               double *dFbar) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nlam) return;
    {
        const int64_t st = blockIdx.y;
        gc += st * n_pix;
        dLdf += st * n_pix;
        dFbar += st * nlam;
    }
    // first pixel with tap0 + ntap - 1 >= i
    int64_t lo = 0, hi = n_pix;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)tap0[mid] + ntap[mid] - 1 < i) lo = mid + 1; else hi = mid;
    }
    double acc = 0.0;
    for (int64_t p = lo; p < n_pix && tap0[p] <= i; ++p) {
        int64_t k = i - tap0[p];
        if (k < ntap[p]) acc += (double)w[p * max_taps + k] * (double)dLdf[p] / gc[p];
    }
    dFbar[i] = acc;
}

__global__ void k_identity_adjoint(int64_t n, const double *Fc, const float *dLdf, double *dFbar) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dFbar[i] = (double)dLdf[i] / Fc[i];
}

cudaError_t launch_inst_adjoint(pz_ctx *c, const float *dLdf, cudaStream_t s) {
    if (c->identity_inst) {
        const int64_t n = (int64_t)c->S * c->nlam;
        k_identity_adjoint<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c->d_Fc, dLdf, c->d_dFbar);
    } else {
        dim3 nb((unsigned)((c->nlam + 255) / 256), c->S);
        k_inst_adjoint<<<nb, 256, 0, s>>>(c->nlam, c->n_pix, c->max_taps, c->d_tap0, c->d_ntap, c->d_tapw, c->d_gc,
                                          dLdf, c->d_dFbar);
    }
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// transfer adjoint: G(i, d) = dL/dchi(i, d) (total branch), stored as G * stim
// ---------------------------------------------------------------------------
struct RtAdjArgs {
    int64_t nlam, ld;
    int nd;
    double lam0cm, lnr;
    const double *m, *T, *kc, *B, *stim;
    const void *kline;
    const double *dFbar;
    void *Gt;
};

// d/dtau_a and d/dtau_b of the interval integral at fixed endpoint values
__device__ __forceinline__ void interval_grad(double ta, double tb, double Sa, double Sb, double e2a, double e3a,
                                              double e4a, double e2b, double e3b, double e4b, double &da,
                                              double &db) {
    const double D = tb - ta, iD = 1.0 / D;
    const double s = (Sb - Sa) * iD;
    const double P = e3a - e3b;
    const double Bq = e4a - e4b - D * e3b;
    da = -Sa * e2a + (s * iD) * Bq - s * P;
    db = Sb * e2b - (s * iD) * Bq;
}

// one thread per (lambda, star); star = blockIdx.y
template <typename KT, typename GT>
__global__ void k_rt_adjoint(RtAdjArgs g) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nlam) return;
    {
        const int64_t st = blockIdx.y;
        g.m += st * g.nd;
        g.T += st * g.nd;
        g.kc += st * g.nd * g.ld;
        g.B += st * g.nd * g.ld;
        g.stim += st * g.nd * g.ld;
        g.kline = reinterpret_cast<const KT *>(g.kline) + st * g.nd * g.ld;
        g.dFbar += st * g.nlam;
        g.Gt = reinterpret_cast<GT *>(g.Gt) + st * g.nd * g.ld;
    }
    const KT *kl = reinterpret_cast<const KT *>(g.kline);
    GT *Gt = reinterpret_cast<GT *>(g.Gt);
    const double dFb = g.dFbar[i];
    double tau[kMaxDepth], S[kMaxDepth], dF[kMaxDepth];
    double chi_p = 0.0;
    for (int d = 0; d < g.nd; ++d) {
        const int64_t o = (int64_t)d * g.ld + i;
        double chi = g.kc[o] + (double)kl[o];
        tau[d] = d == 0 ? chi * g.m[0] : tau[d - 1] + 0.5 * (chi_p + chi) * (g.m[d] - g.m[d - 1]);
        S[d] = g.B[o];
        dF[d] = 0.0;
        chi_p = chi;
    }
    // dF/dtau_j, walking the intervals with the E_n of both endpoints
    double e2a, e3a, e4a;
    expn234(tau[0], e2a, e3a, e4a);
    {
        // top interval: Sa = S0 - s0 tau0, s0 = (S1 - S0)/(tau1 - tau0)
        double t0 = tau[0], t1 = tau[1];
        double s0 = (S[1] - S[0]) / (t1 - t0);
        double sp = s0 / (t1 - t0);
        double Pt = 0.5 - e3a;
        double Bt = 1.0 / 3.0 - e4a - t0 * e3a;
        dF[0] += -s0 * Pt + sp * (Bt - t0 * Pt) + S[0] * e2a;
        dF[1] += -sp * (Bt - t0 * Pt);
    }
    for (int d = 0; d + 1 < g.nd; ++d) {
        double e2b, e3b, e4b;
        expn234(tau[d + 1], e2b, e3b, e4b);
        double da, db;
        interval_grad(tau[d], tau[d + 1], S[d], S[d + 1], e2a, e3a, e4a, e2b, e3b, e4b, da, db);
        dF[d] += da;
        dF[d + 1] += db;
        e2a = e2b; e3a = e3b; e4a = e4b;
    }
    // reverse cumulative sum through the trapezoid: T_j = sum_{k >= j} dL/dtau_k,
    // dL/dchi_d = [d = 0] m_0 T_0 + (m_{d+1} - m_d)/2 T_{d+1} + (m_d - m_{d-1})/2 T_d
    const double scale = 2.0 * kPI * dFb;
    double Tn = 0.0;   // T_{d+1}
    for (int d = g.nd - 1; d >= 0; --d) {
        double Td = Tn + scale * dF[d];
        double gch = 0.0;
        if (d + 1 < g.nd) gch += 0.5 * (g.m[d + 1] - g.m[d]) * Tn;
        if (d >= 1) gch += 0.5 * (g.m[d] - g.m[d - 1]) * Td;
        else gch += g.m[0] * Td;
        Gt[(int64_t)d * g.ld + i] = (GT)(gch * g.stim[(int64_t)d * g.ld + i]);
        Tn = Td;
    }
}

cudaError_t launch_rt_adjoint(pz_ctx *c, cudaStream_t s) {
    if (c->d_sigma) return launch_rt_adjoint_scatter(c, s);
    RtAdjArgs g;
    g.nlam = c->nlam;
    g.ld = c->ld;
    g.nd = c->nd;
    g.lam0cm = c->lambda0_nm * 1e-7;
    g.lnr = c->lnr;
    g.m = c->d_m;
    g.T = c->d_T;
    g.kc = c->d_kc;
    g.B = c->d_B;
    g.stim = c->d_stim;
    g.kline = c->d_kline;
    g.dFbar = c->d_dFbar;
    dim3 nb((unsigned)((c->nlam + 127) / 128), c->S);
    if (c->prec == PZ_MIXED) {
        g.Gt = c->d_Gt;
        k_rt_adjoint<float, float><<<nb, 128, 0, s>>>(g);
    } else {
        g.Gt = c->d_Gt64;
        k_rt_adjoint<double, double><<<nb, 128, 0, s>>>(g);
    }
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// gradient finalisation: ln10 scale, sum over the stars that hold each caller line,
// species -> element sums
// ---------------------------------------------------------------------------
// Per-line gradients into caller order (a line of several stars' subsets adds once per
// subset) and the abundance gradients: use_ab 1 sums them per block in shared memory
// (n_elem doubles), then one global add per (block, element); use_ab 2 (more elements
// than the shared buffer takes) adds each line's term to the global sum directly.
__global__ void k_grad_finalize(int64_t nl, int64_t nl_caller, const double *gacc, const int32_t *orig,
                                const int32_t *sp, const int32_t *eos, int use_ab, int n_elem, int four,
                                double *gline, double *gab) {
    extern __shared__ double s_ab[];
    if (use_ab == 1) {
        for (int k = threadIdx.x; k < n_elem; k += blockDim.x) s_ab[k] = 0.0;
        __syncthreads();
    }
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l < nl) {
        const double ggf = kLN10 * gacc[l];
        const double gg6 = kLN10 * gacc[nl + l];
        const int32_t o = orig[l];
        atomicAdd(gline + o, ggf);
        atomicAdd(gline + nl_caller + o, gg6);
        if (four) {
            // the second sums of the radiative and Stark passes
            atomicAdd(gline + 2 * nl_caller + o, kLN10 * gacc[3 * nl + l]);
            atomicAdd(gline + 3 * nl_caller + o, kLN10 * gacc[5 * nl + l]);
        }
        if (use_ab) {
            const int e = eos[sp[l]];
            if (e >= 0) atomicAdd(use_ab == 1 ? s_ab + e : gab + e, ggf);
        }
    }
    if (use_ab == 1) {
        __syncthreads();
        for (int k = threadIdx.x; k < n_elem; k += blockDim.x)
            if (s_ab[k] != 0.0) atomicAdd(gab + k, s_ab[k]);
    }
}

__global__ void k_copy_d2f(int64_t n, const double *a, float *b) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) b[k] = (float)a[k];
}

cudaError_t launch_grad_finalize(pz_ctx *c, float *g_gf, float *g_g6, float *g_ab, cudaStream_t s, bool four,
                                 float *g_rad, float *g_g4) {
    constexpr int kMaxBlockElems = 4096;   // 32 KB of shared memory
    const int use_ab = c->n_elem <= 0 ? 0 : (c->n_elem <= kMaxBlockElems ? 1 : 2);
    const int rows = four ? 4 : 2;
    cudaError_t e = cudaMemsetAsync(c->d_gline, 0, sizeof(double) * rows * std::max<int64_t>(c->nl_caller, 1), s);
    if (e != cudaSuccess) return e;
    if (use_ab && (e = cudaMemsetAsync(c->d_gab, 0, sizeof(double) * c->n_elem, s)) != cudaSuccess) return e;
    if (c->L.n > 0) {
        const size_t smem = use_ab == 1 ? sizeof(double) * (size_t)c->n_elem : 0;
        k_grad_finalize<<<(unsigned)((c->L.n + 255) / 256), 256, smem, s>>>(
            c->L.n, c->nl_caller, c->d_gacc, c->L.orig, c->L.sp, c->d_eos, use_ab, (int)c->n_elem, four ? 1 : 0,
            c->d_gline, c->d_gab);
        c->launches++;
    }
    const int64_t n = c->nl_caller;
    if (four && n > 0 && g_rad) {
        k_copy_d2f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c->d_gline + 2 * n, g_rad);
        c->launches++;
    }
    if (four && n > 0 && g_g4) {
        k_copy_d2f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c->d_gline + 3 * n, g_g4);
        c->launches++;
    }
    if (n > 0 && g_gf) {
        k_copy_d2f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c->d_gline, g_gf);
        c->launches++;
    }
    if (n > 0 && g_g6) {
        k_copy_d2f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c->d_gline + n, g_g6);
        c->launches++;
    }
    if (g_ab && use_ab) {
        k_copy_d2f<<<(c->n_elem + 255) / 256, 256, 0, s>>>(c->n_elem, c->d_gab, g_ab);
        c->launches++;
    }
    return cudaGetLastError();
}

// probe: E_2, E_3, E_4 as the flux kernels evaluate them
__global__ void k_probe_expn(const double *x, int64_t n, double *out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double e2, e3, e4;
    expn234(x[k], e2, e3, e4);
    out[k] = e2;
    out[n + k] = e3;
    out[2 * n + k] = e4;
    e23(x[k], e2, e3);
    out[3 * n + k] = e2;
    out[4 * n + k] = e3;
}

cudaError_t launch_probe_expn(const double *x, int64_t n, double *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (ensure_expn_table() != PZ_OK) return cudaErrorInitializationError;
    k_probe_expn<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, out);
    return cudaGetLastError();
}

}  // namespace pz

// pz_api.cu -- the C ABI of include/pz.h: validation, one-time window
// preparation (sorting, per-tile line ranges, device tables) and the
// orchestration of the kernels in pz_line.cu and pz_rt.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "pz_internal.h"

namespace pz {

static thread_local std::string g_err;

pz_status fail(pz_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

pz_status cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return PZ_OK;
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PZ_ENOMEM : PZ_ECUDA;
}

static cudaEvent_t prof_event(pz_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

static void prof_fold(pz_ctx *c) {
    for (auto &m : c->marks) {
        float ms = 0.0f;
        if (cudaEventSynchronize(m.b) == cudaSuccess && cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            c->k_ms[m.kid] += ms;
            c->k_count[m.kid] += 1;
        }
        c->ev_pool.push_back(m.a);
        c->ev_pool.push_back(m.b);
    }
    c->marks.clear();
}

void prof_begin(pz_ctx *c, cudaStream_t s) {
    if (!c->profiling) return;
    cudaEvent_t a = prof_event(c);
    cudaEventRecord(a, s);
    c->pending_begin = a;
}

void prof_end(pz_ctx *c, cudaStream_t s, int kid) {
    if (!c->profiling || !c->pending_begin) return;
    cudaEvent_t b = prof_event(c);
    cudaEventRecord(b, s);
    c->marks.push_back({c->pending_begin, b, kid});
    c->pending_begin = nullptr;
    if (c->marks.size() > 8192) prof_fold(c);
}

template <class Fn>
static cudaError_t timed(pz_ctx *c, cudaStream_t s, int kid, Fn &&fn) {
    prof_begin(c, s);
    cudaError_t e = fn();
    prof_end(c, s, kid);
    return e;
}

#define PZ_TRY(expr)                         \
    do {                                     \
        pz_status _st = (expr);              \
        if (_st != PZ_OK) return _st;        \
    } while (0)
#define PZ_CUDA(expr, what) PZ_TRY(cuda_check((expr), what))

template <typename T>
static pz_status dalloc(T **p, size_t n, const char *what) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cuda_check(cudaMalloc((void **)p, n * sizeof(T)), what);
}

template <typename T>
static pz_status upload(T **p, const std::vector<T> &h, const char *what) {
    PZ_TRY(dalloc(p, h.size(), what));
    if (!h.empty()) PZ_CUDA(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), what);
    return PZ_OK;
}

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

static bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void dfree(void *p) {
    if (p) cudaFree(p);
}

static pz_status build_tiles(pz_ctx *c) {
    int T = c->tiling.lambda_per_tile();
    int nt = (int)((c->nlam + T - 1) / T);
    std::vector<int32_t> lo(nt), hi(nt);
    for (int t = 0; t < nt; ++t) {
        int64_t a = (int64_t)t * T - c->W, b = (int64_t)t * T + T - 1 + c->W;
        lo[t] = (int32_t)(std::lower_bound(c->h_il.begin(), c->h_il.end(), (int32_t)std::max<int64_t>(a, INT32_MIN)) -
                          c->h_il.begin());
        hi[t] = (int32_t)(std::upper_bound(c->h_il.begin(), c->h_il.end(), (int32_t)std::min<int64_t>(b, INT32_MAX)) -
                          c->h_il.begin());
    }
    // near-core line ranges: x_l within 20 Doppler widths (the widest over species and
    // depths) of the tile, plus a margin
    double kmin = 1e300;
    for (float v : c->h_invdv) kmin = std::min(kmin, kC * (double)v);
    const double hw = 20.0 / (kmin * c->lnr) * 1.02 + 4.0;
    std::vector<int32_t> nlo(nt), nhi(nt);
    for (int t = 0; t < nt; ++t) {
        double a = (double)t * T - hw, b = (double)t * T + T - 1 + hw;
        a = std::max(a, (double)INT32_MIN / 2);
        b = std::min(b, (double)INT32_MAX / 2);
        nlo[t] = (int32_t)(std::lower_bound(c->h_il.begin(), c->h_il.end(), (int32_t)std::floor(a)) - c->h_il.begin());
        nhi[t] = (int32_t)(std::upper_bound(c->h_il.begin(), c->h_il.end(), (int32_t)std::ceil(b)) - c->h_il.begin());
    }
    dfree(c->d_tile_lo);
    dfree(c->d_tile_hi);
    dfree(c->d_near_lo);
    dfree(c->d_near_hi);
    c->d_tile_lo = c->d_tile_hi = c->d_near_lo = c->d_near_hi = nullptr;
    PZ_TRY(upload(&c->d_tile_lo, lo, "tile ranges"));
    PZ_TRY(upload(&c->d_tile_hi, hi, "tile ranges"));
    PZ_TRY(upload(&c->d_near_lo, nlo, "tile ranges"));
    PZ_TRY(upload(&c->d_near_hi, nhi, "tile ranges"));
    c->ntiles = nt;
    c->tileT = T;
    return PZ_OK;
}

// Fast-path threshold per (species, depth slab of DS layers): a line whose distance
// from every point of the tile is >= thr (grid units) has |v| >= 20 at every depth of
// the slab, because |v| = |expm1(Delta ln r)| c/dv_D >= |Delta| ln r (1 - |Delta| ln r / 2) c/dv_D.
// Slabs past the last layer (grid padding) get 0.
static pz_status build_thresholds(pz_ctx *c) {
    const int DS = c->tiling.DS, DC = c->tiling.depth_per_cta();
    const int nslab = ((c->nd + DC - 1) / DC) * c->tiling.GW;
    double shrink = 1.0 - 0.5 * (c->W + 1024.0) * c->lnr;
    if (shrink < 0.5) shrink = 0.5;
    std::vector<float> thr((size_t)c->ns * nslab, 0.0f);
    for (int s = 0; s < c->ns; ++s)
        for (int b = 0; b < nslab; ++b) {
            double mn = 1e300;
            for (int d = b * DS; d < std::min(c->nd, (b + 1) * DS); ++d)
                mn = std::min(mn, (double)c->h_invdv[(size_t)s * c->nd + d]);
            if (mn < 1e300) thr[(size_t)s * nslab + b] = (float)(20.0 / (kC * mn * c->lnr * shrink) * (1.0 + 1e-4) + 1e-3);
        }
    dfree(c->d_thr);
    c->d_thr = nullptr;
    PZ_TRY(upload(&c->d_thr, thr, "thresholds"));
    c->nslab = nslab;
    return PZ_OK;
}

static void destroy_ctx(pz_ctx *c) {
    if (!c) return;
    void *ptrs[] = {c->d_m, c->d_T, c->d_beta_hi, c->d_beta_lo, c->d_ne, c->d_npert, c->d_c2T, c->d_ne64,
                    c->d_npert64, c->d_rho64, c->d_R, c->d_Rbase, c->d_invdv, c->d_pop64, c->d_mass64, c->d_thr,
                    c->d_kc, c->d_dab, c->d_eos, c->L.orig, c->L.ilf, c->L.il32, c->L.frac, c->L.sp, c->L.E,
                    c->L.lamcm, c->L.grad, c->L.g4, c->L.g6base, c->L.g6, c->L.Q, c->L.Qbase, c->L.x64,
                    c->L.lg_gf, c->L.lg_rad, c->L.lg_4, c->L.lg_6, c->L.dgf, c->L.dg6, c->d_tile_lo, c->d_tile_hi,
                    c->d_kline, c->d_knear, c->d_near_lo, c->d_near_hi, c->d_F, c->d_Fc, c->d_g, c->d_gc, c->d_tap0, c->d_ntap, c->d_tapw, c->d_dFbar,
                    c->d_Gt, c->d_Gt64, c->d_gacc, c->d_gab};
    for (void *p : ptrs) dfree(p);
    for (auto &m : c->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

static pz_status create_impl(const pz_atmos *at, const pz_linelist *ll, pz_precision prec, pz_ctx **out) {
    if (!out) return fail(PZ_EINVAL, "pz_create: out is NULL");
    *out = nullptr;
    if (!at || !ll) return fail(PZ_EINVAL, "pz_create: atmos or lines is NULL");
    if (prec != PZ_FP64 && prec != PZ_MIXED) return fail(PZ_EINVAL, "pz_create: unknown precision");
    const int nd = at->n_depth, ns = at->n_species;
    if (nd < 2 || nd > kMaxDepth) return fail(PZ_EINVAL, "pz_create: n_depth must be in [2, 128]");
    if (ns < 1) return fail(PZ_EINVAL, "pz_create: n_species must be >= 1");
    if (at->n_lambda < 1 || at->n_lambda > 16000000) return fail(PZ_EINVAL, "pz_create: n_lambda must be in [1, 1.6e7]");
    if (ll->n_lines < 0 || ll->n_lines > 2000000000) return fail(PZ_EINVAL, "pz_create: n_lines out of range");
    if (ll->half_window < 0 || ll->half_window > 500000) return fail(PZ_EINVAL, "pz_create: half_window must be in [0, 5e5]");
    if (!at->m || !at->T || !at->rho || !at->n_e || !at->n_pert || !at->pop || !at->mass_amu || !at->kappa_c)
        return fail(PZ_EINVAL, "pz_create: an atmosphere array is NULL");
    if (!finite_pos(at->lambda0_nm) || !finite_pos(at->R_grid)) return fail(PZ_EINVAL, "pz_create: lambda0 and R_grid must be > 0");
    if (!(std::isfinite(at->xi_cms) && at->xi_cms >= 0)) return fail(PZ_EINVAL, "pz_create: xi must be finite and >= 0");
    for (int d = 0; d < nd; ++d) {
        if (!finite_pos(at->m[d]) || !finite_pos(at->T[d]) || !finite_pos(at->rho[d]))
            return fail(PZ_EINVAL, "pz_create: m, T, rho must be finite and > 0");
        if (!(std::isfinite(at->n_e[d]) && at->n_e[d] >= 0) || !(std::isfinite(at->n_pert[d]) && at->n_pert[d] >= 0))
            return fail(PZ_EINVAL, "pz_create: n_e and n_pert must be finite and >= 0");
        if (d > 0 && !(at->m[d] > at->m[d - 1])) return fail(PZ_EINVAL, "pz_create: m must be strictly increasing");
    }
    for (int s = 0; s < ns; ++s) {
        if (!finite_pos(at->mass_amu[s])) return fail(PZ_EINVAL, "pz_create: mass_amu must be > 0");
        for (int d = 0; d < nd; ++d) {
            double p = at->pop[(size_t)s * nd + d];
            if (!(std::isfinite(p) && p >= 0)) return fail(PZ_EINVAL, "pz_create: pop must be finite and >= 0");
        }
    }
    const int64_t nlam = at->n_lambda;
    for (int64_t k = 0; k < (int64_t)nd * nlam; ++k)
        if (!finite_pos(at->kappa_c[k])) return fail(PZ_EINVAL, "pz_create: kappa_c must be finite and > 0");
    const int64_t nl = ll->n_lines;
    if (nl > 0 && (!ll->lambda_nm || !ll->log_gf || !ll->E_low_eV || !ll->log_gamma_rad || !ll->log_gamma4 ||
                   !ll->log_gamma6 || !ll->species))
        return fail(PZ_EINVAL, "pz_create: a line array is NULL");
    for (int64_t l = 0; l < nl; ++l) {
        if (!finite_pos(ll->lambda_nm[l])) return fail(PZ_EINVAL, "pz_create: lambda_nm must be finite and > 0");
        if (!std::isfinite(ll->log_gf[l]) || !std::isfinite(ll->E_low_eV[l]) || !std::isfinite(ll->log_gamma_rad[l]) ||
            !std::isfinite(ll->log_gamma4[l]) || !std::isfinite(ll->log_gamma6[l]))
            return fail(PZ_EINVAL, "pz_create: non-finite line parameter");
        if (ll->species[l] < 0 || ll->species[l] >= ns) return fail(PZ_EINVAL, "pz_create: species out of range");
    }

    pz_ctx *c = new pz_ctx();
    int dev = 0;
    cudaGetDevice(&dev);
    c->device = dev;
    c->prec = prec;
    c->nd = nd;
    c->ns = ns;
    c->nlam = nlam;
    c->ld = ((nlam + 511) / 512) * 512;
    c->lambda0_nm = at->lambda0_nm;
    c->R = at->R_grid;
    c->lnr = std::log1p(1.0 / at->R_grid);
    c->xi = at->xi_cms;
    c->W = ll->half_window;
    c->nl_caller = nl;

    auto bail = [&](pz_status st) {
        destroy_ctx(c);
        return st;
    };
    if (ensure_device_tables() != PZ_OK) return bail(PZ_ECUDA);

    // ---- lines: centre placement, drop, sort ----
    const double W = c->W;
    std::vector<double> x(nl);
    std::vector<int64_t> keep;
    keep.reserve(nl);
    for (int64_t l = 0; l < nl; ++l) {
        x[l] = std::log(ll->lambda_nm[l] / at->lambda0_nm) / c->lnr;
        double il = std::floor(x[l] + 0.5);
        if (il >= -W && il <= (double)(nlam - 1) + W) keep.push_back(l);
    }
    std::stable_sort(keep.begin(), keep.end(), [&](int64_t a, int64_t b) { return x[a] < x[b]; });
    const int64_t n = (int64_t)keep.size();
    c->L.n = n;
    std::vector<int32_t> orig(n), il32(n), sp(n);
    std::vector<float> ilf(n), frac(n), E(n), lamcm(n), grad(n), g4(n), g6(n), Qf(n), lg_gf(n), lg_rad(n), lg_4(n),
        lg_6(n), zeros(n, 0.0f);
    std::vector<double> Qb(n), x64(n);
    const double C0 = kPI * kE * kE / (kME * kC) / kSQRTPI;
    int64_t evals = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t l = keep[k];
        double il = std::floor(x[l] + 0.5);
        orig[k] = (int32_t)l;
        il32[k] = (int32_t)il;
        ilf[k] = (float)il;
        frac[k] = (float)(x[l] - il);
        sp[k] = ll->species[l];
        E[k] = ll->E_low_eV[l];
        double lc = ll->lambda_nm[l] * 1e-7;
        lamcm[k] = (float)lc;
        grad[k] = (float)std::pow(10.0, (double)ll->log_gamma_rad[l]);
        g4[k] = (float)std::pow(10.0, (double)ll->log_gamma4[l]);
        g6[k] = (float)std::pow(10.0, (double)ll->log_gamma6[l]);
        Qb[k] = C0 * lc * std::pow(10.0, (double)ll->log_gf[l]);
        Qf[k] = (float)Qb[k];
        x64[k] = x[l];
        lg_gf[k] = ll->log_gf[l];
        lg_rad[k] = ll->log_gamma_rad[l];
        lg_4[k] = ll->log_gamma4[l];
        lg_6[k] = ll->log_gamma6[l];
        int64_t i0 = std::max<int64_t>(0, (int64_t)il - c->W), i1 = std::min<int64_t>(nlam - 1, (int64_t)il + c->W);
        evals += (i1 - i0 + 1);
    }
    c->n_evals = evals * nd;
    c->h_il = il32;
    if (upload(&c->L.orig, orig, "lines") || upload(&c->L.il32, il32, "lines") || upload(&c->L.ilf, ilf, "lines") ||
        upload(&c->L.frac, frac, "lines") || upload(&c->L.sp, sp, "lines") || upload(&c->L.E, E, "lines") ||
        upload(&c->L.lamcm, lamcm, "lines") || upload(&c->L.grad, grad, "lines") || upload(&c->L.g4, g4, "lines") ||
        upload(&c->L.g6base, g6, "lines") || upload(&c->L.g6, g6, "lines") || upload(&c->L.Q, Qf, "lines") ||
        upload(&c->L.Qbase, Qb, "lines") || upload(&c->L.x64, x64, "lines") || upload(&c->L.lg_gf, lg_gf, "lines") ||
        upload(&c->L.lg_rad, lg_rad, "lines") || upload(&c->L.lg_4, lg_4, "lines") ||
        upload(&c->L.lg_6, lg_6, "lines") || upload(&c->L.dgf, zeros, "lines") || upload(&c->L.dg6, zeros, "lines"))
        return bail(PZ_ENOMEM);

    // ---- depth and species tables ----
    c->h_m.assign(at->m, at->m + nd);
    c->h_T.assign(at->T, at->T + nd);
    std::vector<float> bh(nd), bl(nd), ne(nd), npert(nd), c2T(nd);
    std::vector<double> ne64(at->n_e, at->n_e + nd), np64(at->n_pert, at->n_pert + nd), rho64(at->rho, at->rho + nd);
    for (int d = 0; d < nd; ++d) {
        double beta = kEV / (kKB * at->T[d]);
        bh[d] = (float)beta;
        bl[d] = (float)(beta - (double)bh[d]);
        ne[d] = (float)at->n_e[d];
        npert[d] = (float)at->n_pert[d];
        c2T[d] = (float)(kC2 / at->T[d]);
    }
    std::vector<float> invdv((size_t)ns * nd), Rf((size_t)ns * nd);
    std::vector<double> Rb((size_t)ns * nd), pop64(at->pop, at->pop + (size_t)ns * nd), mass64(at->mass_amu, at->mass_amu + ns);
    for (int s = 0; s < ns; ++s)
        for (int d = 0; d < nd; ++d) {
            double dv = std::sqrt(2.0 * kKB * at->T[d] / (at->mass_amu[s] * kAMU) + c->xi * c->xi);
            size_t id = (size_t)s * nd + d;
            invdv[id] = (float)(1.0 / dv);
            Rb[id] = (1.0 / dv) * at->pop[id] / at->rho[d];
            Rf[id] = (float)Rb[id];
        }
    c->h_invdv = invdv;
    std::vector<double> dab(1, 0.0);
    std::vector<int32_t> eos(ns, -1);
    if (upload(&c->d_m, c->h_m, "depth") || upload(&c->d_T, c->h_T, "depth") || upload(&c->d_beta_hi, bh, "depth") ||
        upload(&c->d_beta_lo, bl, "depth") || upload(&c->d_ne, ne, "depth") || upload(&c->d_npert, npert, "depth") ||
        upload(&c->d_c2T, c2T, "depth") || upload(&c->d_ne64, ne64, "depth") || upload(&c->d_npert64, np64, "depth") ||
        upload(&c->d_rho64, rho64, "depth") || upload(&c->d_invdv, invdv, "species") || upload(&c->d_R, Rf, "species") ||
        upload(&c->d_Rbase, Rb, "species") || upload(&c->d_pop64, pop64, "species") ||
        upload(&c->d_mass64, mass64, "species") || build_thresholds(c) || upload(&c->d_dab, dab, "abund") ||
        upload(&c->d_eos, eos, "abund"))
        return bail(PZ_ENOMEM);

    // ---- continuum opacity [nd][ld] ----
    if (dalloc(&c->d_kc, (size_t)nd * c->ld, "kappa_c")) return bail(PZ_ENOMEM);
    if (cuda_check(cudaMemset(c->d_kc, 0, sizeof(double) * nd * c->ld), "kappa_c") ||
        cuda_check(cudaMemcpy2D(c->d_kc, c->ld * sizeof(double), at->kappa_c, nlam * sizeof(double),
                                nlam * sizeof(double), nd, cudaMemcpyHostToDevice),
                   "kappa_c"))
        return bail(PZ_ECUDA);

    // ---- resident buffers ----
    size_t ksz = (prec == PZ_MIXED) ? sizeof(float) : sizeof(double);
    if (cuda_check(cudaMalloc(&c->d_kline, ksz * nd * c->ld), "kappa_line buffer") ||
        (prec == PZ_MIXED && dalloc(&c->d_knear, (size_t)nd * c->ld, "kappa_line buffer")) ||
        dalloc(&c->d_F, nlam, "flux") || dalloc(&c->d_Fc, nlam, "flux"))
        return bail(PZ_ENOMEM);
    if (build_tiles(c) != PZ_OK) return bail(PZ_ENOMEM);
    if (cuda_check(cudaDeviceSynchronize(), "pz_create")) return bail(PZ_ECUDA);
    *out = c;
    return PZ_OK;
}

static pz_status ensure_out_buffers(pz_ctx *c, int64_t n) {
    if (c->d_g && c->pix_cap >= n) return PZ_OK;
    dfree(c->d_g);
    dfree(c->d_gc);
    c->d_g = c->d_gc = nullptr;
    PZ_TRY(dalloc(&c->d_g, n, "instrument output"));
    PZ_TRY(dalloc(&c->d_gc, n, "instrument output"));
    c->pix_cap = n;
    return PZ_OK;
}

__global__ void k_gather_f32(int64_t n, const int32_t *orig, const float *src, float *dst) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l < n) dst[l] = src[orig[l]];
}

__global__ void k_f32_to_f64(int n, const float *a, double *b) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) b[k] = (double)a[k];
}

__global__ void k_d2f_2d(int64_t nlam, int64_t ld, int nd, const double *a, float *b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int d = blockIdx.y;
    if (i < nlam) b[(int64_t)d * nlam + i] = (float)a[(int64_t)d * ld + i];
}

}  // namespace pz

using namespace pz;

extern "C" {

pz_status pz_create(const pz_atmos *atmos, const pz_linelist *lines, pz_precision precision, pz_ctx **out) {
    return create_impl(atmos, lines, precision, out);
}

pz_status pz_destroy(pz_ctx *ctx) {
    if (!ctx) return PZ_OK;
    cudaDeviceSynchronize();
    destroy_ctx(ctx);
    return PZ_OK;
}

const char *pz_last_error(void) { return g_err.c_str(); }

int64_t pz_eval_count(const pz_ctx *ctx) { return ctx ? ctx->n_evals : 0; }

int32_t pz_last_launch_count(const pz_ctx *ctx) { return ctx ? ctx->launches : 0; }

pz_status pz_set_tiling(pz_ctx *c, int32_t J, int32_t DS, int32_t GW, int32_t LC, int32_t MINB) {
    if (!c) return fail(PZ_EINVAL, "pz_set_tiling: ctx is NULL");
    Tiling t = c->tiling;
    if (J > 0) t.J = J;
    if (DS > 0) t.DS = DS;
    if (GW > 0) t.GW = GW;
    if (LC > 0) t.LC = LC;
    if (MINB > 0) t.minb = MINB;
    if (!tiling_supported(t.J, t.DS, t.minb))
        return fail(PZ_EINVAL, "pz_set_tiling: unsupported (lambda_per_thread, depth_per_warp, ctas_per_sm)");
    if (t.GW < 1 || t.GW > 4) return fail(PZ_EINVAL, "pz_set_tiling: warps_per_cta must be in [1, 4]");
    if (t.LC < 1 || t.LC > 512) return fail(PZ_EINVAL, "pz_set_tiling: lines_per_chunk must be in [1, 512]");
    if (LC > 0) t.LCB = std::max(1, t.LC / 2);
    size_t gen = (size_t)t.DS * 32 * t.GW * 16;
    size_t smem_fwd = (size_t)t.LC * t.DS * t.GW * 32 + t.LC * 16 + gen;
    size_t smem_bwd = (size_t)t.LCB * t.DS * t.GW * 64 + t.LCB * 16 + (size_t)t.LCB * t.GW * 8;
    if (smem_fwd > 200 * 1024 || smem_bwd > 200 * 1024)
        return fail(PZ_EINVAL, "pz_set_tiling: shared-memory chunk too large");
    bool retile = t.J != c->tiling.J;
    bool reslab = t.DS != c->tiling.DS || t.GW != c->tiling.GW;
    c->tiling = t;
    if (retile) PZ_TRY(build_tiles(c));
    if (reslab) PZ_TRY(build_thresholds(c));
    return PZ_OK;
}

pz_status pz_set_corrections(pz_ctx *c, const float *dgf, const float *dg6, const float *dab,
                             const int32_t *eos, int32_t n_elem, void *stream) {
    if (!c) return fail(PZ_EINVAL, "pz_set_corrections: ctx is NULL");
    if (n_elem < 0) return fail(PZ_EINVAL, "pz_set_corrections: n_elem < 0");
    if (dab && (n_elem == 0 || !eos)) return fail(PZ_EINVAL, "pz_set_corrections: dabund needs n_elem > 0 and elem_of_species");
    if (dab) {
        for (int s = 0; s < c->ns; ++s)
            if (eos[s] < -1 || eos[s] >= n_elem) return fail(PZ_EINVAL, "pz_set_corrections: elem_of_species out of range");
    }
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    const int64_t n = c->L.n;
    std::vector<int32_t> horig;
    auto set_line = [&](const float *src, float *dst, const char *what) -> pz_status {
        if (!src) return cuda_check(cudaMemsetAsync(dst, 0, sizeof(float) * std::max<int64_t>(n, 1), s), what);
        if (n == 0) return PZ_OK;
        if (is_device_ptr(src)) {
            cudaError_t e = timed(c, s, PZ_K_OTHER, [&] {
                k_gather_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c->L.orig, src, dst);
                return cudaGetLastError();
            });
            c->launches++;
            return cuda_check(e, what);
        }
        if (horig.empty()) {
            horig.resize(n);
            PZ_CUDA(cudaMemcpy(horig.data(), c->L.orig, sizeof(int32_t) * n, cudaMemcpyDeviceToHost), what);
        }
        std::vector<float> tmp(n);
        for (int64_t k = 0; k < n; ++k) tmp[k] = src[horig[k]];
        PZ_CUDA(cudaMemcpy(dst, tmp.data(), sizeof(float) * n, cudaMemcpyHostToDevice), what);
        return PZ_OK;
    };
    PZ_TRY(set_line(dgf, c->L.dgf, "dlog_gf"));
    PZ_TRY(set_line(dg6, c->L.dg6, "dlog_gamma6"));
    if (dab) {
        if (n_elem != c->n_elem) {
            dfree(c->d_dab);
            dfree(c->d_gab);
            c->d_dab = nullptr;
            c->d_gab = nullptr;
            PZ_TRY(dalloc(&c->d_dab, n_elem, "dabund"));
        }
        std::vector<int32_t> heos(eos, eos + c->ns);
        PZ_CUDA(cudaMemcpy(c->d_eos, heos.data(), sizeof(int32_t) * c->ns, cudaMemcpyHostToDevice), "elem_of_species");
        if (is_device_ptr(dab)) {
            PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] {
                        k_f32_to_f64<<<(n_elem + 255) / 256, 256, 0, s>>>(n_elem, dab, c->d_dab);
                        return cudaGetLastError();
                    }),
                    "dabund");
            c->launches++;
        } else {
            std::vector<double> h(dab, dab + n_elem);
            PZ_CUDA(cudaMemcpy(c->d_dab, h.data(), sizeof(double) * n_elem, cudaMemcpyHostToDevice), "dabund");
        }
        c->n_elem = n_elem;
    } else {
        c->n_elem = 0;
        std::vector<int32_t> heos(c->ns, -1);
        PZ_CUDA(cudaMemcpy(c->d_eos, heos.data(), sizeof(int32_t) * c->ns, cudaMemcpyHostToDevice), "elem_of_species");
    }
    PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] { return launch_apply_corrections(c, s); }), "apply corrections");
    c->have_kline = c->have_flux = c->have_inst = false;
    return PZ_OK;
}

pz_status pz_line_opacity(pz_ctx *c, float *kappa, void *stream) {
    if (!c) return fail(PZ_EINVAL, "pz_line_opacity: ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    PZ_CUDA(timed(c, s, PZ_K_LINE_FWD,
                  [&] { return c->prec == PZ_MIXED ? launch_line_fwd_mixed(c, s) : launch_line_fwd_fp64(c, s); }),
            "line opacity kernel");
    if (kappa) {
        if (c->prec == PZ_MIXED) {
            PZ_CUDA(cudaMemcpy2DAsync(kappa, c->nlam * sizeof(float), c->d_kline, c->ld * sizeof(float),
                                      c->nlam * sizeof(float), c->nd, cudaMemcpyDeviceToDevice, s),
                    "copy kappa_line");
        } else {
            dim3 grid((unsigned)((c->nlam + 255) / 256), c->nd);
            PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] {
                        k_d2f_2d<<<grid, 256, 0, s>>>(c->nlam, c->ld, c->nd, (const double *)c->d_kline, kappa);
                        return cudaGetLastError();
                    }),
                    "copy kappa_line");
            c->launches++;
        }
    }
    c->have_kline = true;
    c->have_flux = c->have_inst = false;
    return PZ_OK;
}

pz_status pz_flux(pz_ctx *c, double *F, double *Fc, void *stream) {
    if (!c) return fail(PZ_EINVAL, "pz_flux: ctx is NULL");
    if (!c->have_kline) return fail(PZ_ESTATE, "pz_flux: call pz_line_opacity first");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    PZ_CUDA(timed(c, s, PZ_K_FLUX, [&] { return launch_flux(c, s); }), "flux kernel");
    if (F) PZ_CUDA(cudaMemcpyAsync(F, c->d_F, sizeof(double) * c->nlam, cudaMemcpyDeviceToDevice, s), "copy F");
    if (Fc) PZ_CUDA(cudaMemcpyAsync(Fc, c->d_Fc, sizeof(double) * c->nlam, cudaMemcpyDeviceToDevice, s), "copy Fc");
    c->have_flux = true;
    c->have_inst = false;
    return PZ_OK;
}

pz_status pz_instrument(pz_ctx *c, double v_r, double v_b, double R_lsf, const double *pix, int64_t n_pix, float *f,
                        void *stream) {
    if (!c) return fail(PZ_EINVAL, "pz_instrument: ctx is NULL");
    if (!c->have_flux) return fail(PZ_ESTATE, "pz_instrument: call pz_flux first");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    if (n_pix < 0) return fail(PZ_EINVAL, "pz_instrument: n_pix < 0");
    if (n_pix == 0) {
        PZ_TRY(ensure_out_buffers(c, c->nlam));
        c->identity_inst = true;
        c->n_out = c->nlam;
    } else {
        if (!pix) return fail(PZ_EINVAL, "pz_instrument: pix_lambda_nm is NULL");
        if (!finite_pos(R_lsf)) return fail(PZ_EINVAL, "pz_instrument: R_lsf must be > 0");
        if (!(std::isfinite(v_b) && v_b >= 0) || !std::isfinite(v_r) || std::fabs(v_r) > 1e5)
            return fail(PZ_EINVAL, "pz_instrument: v_r, v_b out of range");
        for (int64_t p = 0; p < n_pix; ++p) {
            if (!finite_pos(pix[p])) return fail(PZ_EINVAL, "pz_instrument: pixel wavelengths must be > 0");
            if (p > 0 && !(pix[p] > pix[p - 1])) return fail(PZ_EINVAL, "pz_instrument: pixels must be increasing");
        }
        double sig_lsf = 1.0 / (2.0 * std::sqrt(2.0 * std::log(2.0)) * R_lsf);
        double sig_b = v_b * 1e5 / kC;
        double sig = std::sqrt(sig_lsf * sig_lsf + sig_b * sig_b) / c->lnr;
        int64_t mt = 2 * (int64_t)std::ceil(5.0 * sig) + 2;
        if (mt > kMaxTaps) return fail(PZ_EINVAL, "pz_instrument: instrument kernel wider than 4096 grid points");
        bool same = !c->identity_inst && c->inst_key[0] == v_r && c->inst_key[1] == v_b && c->inst_key[2] == R_lsf &&
                    (int64_t)c->pix_key.size() == n_pix && std::equal(pix, pix + n_pix, c->pix_key.begin());
        if (!same) {
            if (c->n_pix < n_pix || c->max_taps < mt) {
                dfree(c->d_tap0);
                dfree(c->d_ntap);
                dfree(c->d_tapw);
                c->d_tap0 = c->d_ntap = nullptr;
                c->d_tapw = nullptr;
                PZ_TRY(dalloc(&c->d_tap0, n_pix, "instrument"));
                PZ_TRY(dalloc(&c->d_ntap, n_pix, "instrument"));
                PZ_TRY(dalloc(&c->d_tapw, (size_t)n_pix * mt, "instrument"));
            }
            c->n_pix = n_pix;
            c->max_taps = (int32_t)mt;
            double *d_pix = nullptr;
            int32_t *d_err = nullptr;
            PZ_TRY(dalloc(&d_pix, n_pix, "instrument"));
            PZ_TRY(dalloc(&d_err, 1, "instrument"));
            pz_status st = PZ_OK;
            int32_t herr = 0;
            if ((st = cuda_check(cudaMemcpyAsync(d_pix, pix, sizeof(double) * n_pix, cudaMemcpyHostToDevice, s), "pixels")) ==
                    PZ_OK &&
                (st = cuda_check(cudaMemsetAsync(d_err, 0, sizeof(int32_t), s), "pixels")) == PZ_OK &&
                (st = cuda_check(timed(c, s, PZ_K_INSTRUMENT,
                                       [&] { return launch_inst_build(c, d_pix, v_r, v_b, R_lsf, d_err, s); }),
                                 "instrument build")) == PZ_OK &&
                (st = cuda_check(cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "instrument build")) ==
                    PZ_OK)
                st = cuda_check(cudaStreamSynchronize(s), "instrument build");
            dfree(d_pix);
            dfree(d_err);
            if (st != PZ_OK) return st;
            if (herr) {
                c->identity_inst = true;
                c->pix_key.clear();
                return fail(PZ_EINVAL, "pz_instrument: a pixel has no tap inside the synthesis grid");
            }
            c->inst_key[0] = v_r;
            c->inst_key[1] = v_b;
            c->inst_key[2] = R_lsf;
            c->pix_key.assign(pix, pix + n_pix);
        }
        PZ_TRY(ensure_out_buffers(c, n_pix));
        c->identity_inst = false;
        c->n_out = n_pix;
    }
    PZ_CUDA(timed(c, s, PZ_K_INSTRUMENT, [&] { return launch_inst_apply(c, f, s); }), "instrument apply");
    c->have_inst = true;
    return PZ_OK;
}

pz_status pz_loss_chi2(pz_ctx *c, const float *y, const float *w, int64_t n, double *loss, float *dLdf, void *stream) {
    if (!c) return fail(PZ_EINVAL, "pz_loss_chi2: ctx is NULL");
    if (!c->have_inst) return fail(PZ_ESTATE, "pz_loss_chi2: call pz_instrument first");
    if (!y) return fail(PZ_EINVAL, "pz_loss_chi2: y is NULL");
    if (n != c->n_out) return fail(PZ_EINVAL, "pz_loss_chi2: n differs from the instrument output size");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    if (loss) PZ_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s), "loss");
    PZ_CUDA(timed(c, s, PZ_K_LOSS, [&] { return launch_loss(c, y, w, n, loss, dLdf, s); }), "loss kernel");
    return PZ_OK;
}

pz_status pz_backward(pz_ctx *c, const float *dLdf, float *g_gf, float *g_g6, float *g_ab, void *stream) {
    if (!c) return fail(PZ_EINVAL, "pz_backward: ctx is NULL");
    if (!c->have_inst) return fail(PZ_ESTATE, "pz_backward: call pz_instrument first");
    if (!dLdf) return fail(PZ_EINVAL, "pz_backward: dL_df is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    c->launches = 0;
    if (!c->d_dFbar) PZ_TRY(dalloc(&c->d_dFbar, c->nlam, "backward scratch"));
    if (c->prec == PZ_MIXED && !c->d_Gt) PZ_TRY(dalloc(&c->d_Gt, (size_t)c->nd * c->ld, "backward scratch"));
    if (c->prec == PZ_FP64 && !c->d_Gt64) PZ_TRY(dalloc(&c->d_Gt64, (size_t)c->nd * c->ld, "backward scratch"));
    if (!c->d_gacc) PZ_TRY(dalloc(&c->d_gacc, 2 * std::max<int64_t>(c->L.n, 1), "backward scratch"));
    if (c->n_elem > 0 && !c->d_gab) PZ_TRY(dalloc(&c->d_gab, c->n_elem, "backward scratch"));

    PZ_CUDA(timed(c, s, PZ_K_INST_ADJOINT, [&] { return launch_inst_adjoint(c, dLdf, s); }), "instrument adjoint");
    PZ_CUDA(timed(c, s, PZ_K_RT_ADJOINT, [&] { return launch_rt_adjoint(c, s); }), "transfer adjoint");
    PZ_CUDA(cudaMemsetAsync(c->d_gacc, 0, sizeof(double) * 2 * std::max<int64_t>(c->L.n, 1), s), "backward");
    if (c->L.n > 0) {
        PZ_CUDA(timed(c, s, PZ_K_LINE_BWD,
                      [&] { return c->prec == PZ_MIXED ? launch_line_bwd_mixed(c, s) : launch_line_bwd_fp64(c, s); }),
                "line gradient kernel");
    }
    if (g_gf) PZ_CUDA(cudaMemsetAsync(g_gf, 0, sizeof(float) * c->nl_caller, s), "backward");
    if (g_g6) PZ_CUDA(cudaMemsetAsync(g_g6, 0, sizeof(float) * c->nl_caller, s), "backward");
    if (g_ab && c->n_elem > 0) PZ_CUDA(cudaMemsetAsync(c->d_gab, 0, sizeof(double) * c->n_elem, s), "backward");
    PZ_CUDA(timed(c, s, PZ_K_OTHER, [&] { return launch_grad_finalize(c, g_gf, g_g6, g_ab, s); }),
            "gradient finalize");
    return PZ_OK;
}

pz_status pz_set_profiling(pz_ctx *c, int32_t enable) {
    if (!c) return fail(PZ_EINVAL, "pz_set_profiling: ctx is NULL");
    prof_fold(c);
    for (int k = 0; k < PZ_NK; ++k) {
        c->k_ms[k] = 0.0;
        c->k_count[k] = 0;
    }
    c->profiling = enable != 0;
    return PZ_OK;
}

pz_status pz_kernel_times(pz_ctx *c, double *ms, int64_t *counts, int32_t nk) {
    if (!c || nk < 0 || (nk > 0 && (!ms || !counts))) return fail(PZ_EINVAL, "pz_kernel_times: bad arguments");
    prof_fold(c);
    for (int k = 0; k < nk && k < PZ_NK; ++k) {
        ms[k] = c->k_ms[k];
        counts[k] = c->k_count[k];
    }
    for (int k = PZ_NK; k < nk; ++k) {
        ms[k] = 0.0;
        counts[k] = 0;
    }
    return PZ_OK;
}

pz_status pz_probe_voigt(const float *a, const float *v, int64_t n, float *H, float *dH, void *stream) {
    if (n < 0 || (n > 0 && (!a || !v || !H))) return fail(PZ_EINVAL, "pz_probe_voigt: bad arguments");
    PZ_TRY(ensure_device_tables());
    PZ_CUDA(launch_probe_voigt(a, v, n, H, dH, (cudaStream_t)stream), "probe voigt");
    return PZ_OK;
}

pz_status pz_probe_expn(const double *x, int64_t n, double *out, void *stream) {
    if (n < 0 || (n > 0 && (!x || !out))) return fail(PZ_EINVAL, "pz_probe_expn: bad arguments");
    PZ_CUDA(launch_probe_expn(x, n, out, (cudaStream_t)stream), "probe expn");
    return PZ_OK;
}

}  // extern "C"

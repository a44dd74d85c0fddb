// pz_internal.h -- context layout and kernel-launch declarations shared by the
// translation units of libpz.  Not part of the public ABI (see include/pz.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pz.h"

namespace pz {

// ---- physical constants, CODATA 2018, cgs ---------------------------------
constexpr double kH = 6.62607015e-27;       // erg s
constexpr double kKB = 1.380649e-16;        // erg/K
constexpr double kC = 2.99792458e10;        // cm/s
constexpr double kE = 4.80320471e-10;       // esu
constexpr double kME = 9.1093837015e-28;    // g
constexpr double kEV = 1.602176634e-12;     // erg
constexpr double kAMU = 1.66053906660e-24;  // g
constexpr double kPI = 3.14159265358979323846;
constexpr double kSQRTPI = 1.77245385090551602730;
constexpr double kLN10 = 2.30258509299404568402;
constexpr double kC2 = kH * kC / kKB;       // second radiation constant, cm K

// Largest supported depth count (register/local arrays in the flux kernels).
constexpr int kMaxDepth = 128;
// Largest number of instrument taps per pixel.
constexpr int kMaxTaps = 4096;

// Far-wing / mid / core boundaries of the FP32 Voigt (|z|^2 thresholds).
constexpr float kFar2 = 400.0f;   // |z| >= 20: asymptotic series, 2 corrections
constexpr float kMid2 = 36.0f;    // 6 <= |z| < 20: asymptotic series, 8 corrections
// |z| < 6: a < kCoreA -> Dawson-derivative Taylor table; else Weideman rational.
constexpr float kCoreA = 0.5f;
constexpr int kDawsonK = 16;      // Taylor order of the core table
constexpr int kDawsonPerUnit = 16;  // table nodes per unit of x
constexpr int kDawsonNodes = 6 * kDawsonPerUnit + 1;
constexpr int kWeidN = 16;        // Weideman rational order (FP32 core)
constexpr int kWeidN64 = 32;      // Weideman rational order (FP64 plain form)

// Mixed-precision line-kernel tiling.
struct Tiling {
    int J = 4;       // lambda points per thread (contiguous)
    int DS = 9;      // depths per warp
    int GW = 4;      // warps per CTA (each a depth slab)
    int LC = 32;     // lines per shared-memory chunk (forward)
    int LCB = 16;    // lines per shared-memory chunk (backward)
    int minb = 1;    // minimum resident CTAs per SM the kernels are compiled for
    int lambda_per_tile() const { return 32 * J; }
    int depth_per_cta() const { return DS * GW; }
};

// Device copy of the per-line data, sorted by fractional centre index.
struct LineTable {
    int64_t n = 0;              // lines kept (window intersects the grid)
    int32_t *orig = nullptr;    // caller index of each sorted line
    float *ilf = nullptr;       // integer centre i_l as float (exact, |i_l| < 2^24)
    int32_t *il32 = nullptr;    // integer centre i_l
    float *frac = nullptr;      // x_l - i_l in [-1/2, 1/2)
    int32_t *sp = nullptr;      // species
    float *E = nullptr;         // E_low, eV
    float *lamcm = nullptr;     // lambda_l, cm (FP32)
    float *grad = nullptr;      // gamma_rad, s^-1
    float *g4 = nullptr;        // gamma_4
    float *g6base = nullptr;    // 10^log_gamma6 (uncorrected)
    float *g6 = nullptr;        // 10^(log_gamma6 + dlog_gamma6)
    float *Q = nullptr;         // (pi e^2/m_e c)/sqrt(pi) lambda_l gf_l 10^dlog_gf (FP32)
    double *Qbase = nullptr;    // same without the correction, FP64
    double *x64 = nullptr;      // x_l, FP64 (plain FP64 form)
    float *lg_gf = nullptr;     // log10 gf (caller value; FP64 form)
    float *lg_rad = nullptr, *lg_4 = nullptr, *lg_6 = nullptr;
    float *dgf = nullptr, *dg6 = nullptr;  // current corrections (sorted order)
};

struct pz_ctx_impl;

}  // namespace pz

struct pz_ctx {
    int device = 0;
    pz_precision prec = PZ_MIXED;
    int nd = 0, ns = 0;
    int64_t nlam = 0, ld = 0;     // grid points, padded row stride of [nd][ld] buffers
    double lambda0_nm = 0, R = 0, lnr = 0, xi = 0;
    int W = 0;
    int64_t nl_caller = 0;
    int64_t n_evals = 0;
    pz::Tiling tiling;

    // host copies (small)
    std::vector<double> h_m, h_T;
    std::vector<int32_t> h_il;      // sorted integer centres (for tile ranges)

    // device: depth and species tables
    double *d_m = nullptr, *d_T = nullptr;
    float *d_beta_hi = nullptr, *d_beta_lo = nullptr;   // eV/(k T) split hi + lo
    float *d_ne = nullptr, *d_npert = nullptr, *d_c2T = nullptr;
    double *d_ne64 = nullptr, *d_npert64 = nullptr, *d_rho64 = nullptr;
    float *d_R = nullptr;           // [ns][nd] (1/dv_D) (pop/rho) 10^dabund
    double *d_Rbase = nullptr;      // [ns][nd] (1/dv_D)(pop/rho), FP64
    float *d_invdv = nullptr;       // [ns][nd] 1/dv_D (s/cm)
    double *d_pop64 = nullptr, *d_mass64 = nullptr;
    float *d_thr = nullptr;         // [ns][nslab] fast-path distance threshold (grid units)
    int nslab = 0;                  // depth slabs of DS layers covered by the launch grid
    std::vector<float> h_invdv;     // [ns][nd] host copy of 1/dv_D (thresholds)
    double *d_kc = nullptr;         // [nd][ld] continuum opacity FP64
    double *d_dab = nullptr;        // [n_elem_max] current abundance offsets
    int32_t *d_eos = nullptr;       // [ns] element of species (or -1)
    int n_elem = 0;

    pz::LineTable L;
    int32_t *d_tile_lo = nullptr, *d_tile_hi = nullptr;
    int32_t *d_near_lo = nullptr, *d_near_hi = nullptr;   // lines whose near zone can reach a tile
    float *d_knear = nullptr;       // [nd][ld] near-core sums of the forward
    int ntiles = 0, tileT = 0;

    // resident buffers
    void *d_kline = nullptr;        // [nd][ld] float (MIXED) or double (FP64)
    double *d_F = nullptr, *d_Fc = nullptr;
    double *d_g = nullptr, *d_gc = nullptr;   // instrument outputs (n_out)
    int64_t n_out = 0;
    bool identity_inst = true;
    // instrument weights
    int64_t n_pix = 0, pix_cap = 0;
    int32_t max_taps = 0;
    int32_t *d_tap0 = nullptr, *d_ntap = nullptr;
    float *d_tapw = nullptr;        // [n_pix][max_taps]
    double inst_key[3] = {0, 0, 0};
    std::vector<double> pix_key;

    // backward scratch
    double *d_dFbar = nullptr;      // [nlam]
    float *d_Gt = nullptr;          // [nd][ld] G * stim (FP32, MIXED)
    double *d_Gt64 = nullptr;       // [nd][ld] (FP64 form)
    double *d_gacc = nullptr;       // [2][nl]
    double *d_gab = nullptr;        // [n_elem]

    // state
    bool have_kline = false, have_flux = false, have_inst = false;
    int32_t launches = 0;

    // CUDA-event profiler (pz_set_profiling)
    bool profiling = false;
    struct Mark {
        cudaEvent_t a, b;
        int kid;
    };
    std::vector<Mark> marks;          // recorded, not yet folded
    std::vector<cudaEvent_t> ev_pool; // free events
    cudaEvent_t pending_begin = nullptr;
    double k_ms[PZ_NK] = {0};
    int64_t k_count[PZ_NK] = {0};
};

namespace pz {

// profiler brackets around a launch (pz_api.cu); no-ops unless profiling is on
void prof_begin(pz_ctx *c, cudaStream_t s);
void prof_end(pz_ctx *c, cudaStream_t s, int kid);

// error reporting (pz_api.cu)
pz_status fail(pz_status st, const std::string &msg);
pz_status cuda_check(cudaError_t e, const char *what);

// one-time per-device constant tables (pz_line.cu)
pz_status ensure_device_tables();

// launches (return cudaGetLastError() of the launch)
cudaError_t launch_line_fwd_mixed(pz_ctx *c, cudaStream_t s);
cudaError_t launch_line_bwd_mixed(pz_ctx *c, cudaStream_t s);
cudaError_t launch_line_fwd_fp64(pz_ctx *c, cudaStream_t s);
cudaError_t launch_line_bwd_fp64(pz_ctx *c, cudaStream_t s);
cudaError_t launch_apply_corrections(pz_ctx *c, cudaStream_t s);
cudaError_t launch_probe_voigt(const float *a, const float *v, int64_t n, float *H, float *dH,
                               cudaStream_t s);

cudaError_t launch_flux(pz_ctx *c, cudaStream_t s);
cudaError_t launch_inst_build(pz_ctx *c, const double *d_pix, double v_r, double v_b, double R_lsf,
                              int32_t *d_err, cudaStream_t s);
cudaError_t launch_inst_apply(pz_ctx *c, float *f, cudaStream_t s);
cudaError_t launch_loss(pz_ctx *c, const float *y, const float *w, int64_t n, double *loss,
                        float *dLdf, cudaStream_t s);
cudaError_t launch_inst_adjoint(pz_ctx *c, const float *dLdf, cudaStream_t s);
cudaError_t launch_rt_adjoint(pz_ctx *c, cudaStream_t s);
cudaError_t launch_grad_finalize(pz_ctx *c, float *g_gf, float *g_g6, float *g_ab, cudaStream_t s);
cudaError_t launch_probe_expn(const double *x, int64_t n, double *out, cudaStream_t s);
bool tiling_supported(int J, int DS, int minb);

}  // namespace pz

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
constexpr int kNearDepthsFwd = 8;    // layers per work item of the near-core forward
constexpr int kNearDepthsBwd = 6;    // layers per work item of the near-core backward
// Largest number of instrument taps per pixel.
constexpr int kMaxTaps = 4096;
// Device ordinals a context may live on (per-device launch-attribute bookkeeping).
constexpr int kMaxDevices = 64;

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

// Bits of the context's device status word (pz_sync_status).
constexpr int kStatusWaitGaveUp = 1;      // a bounded device-side wait gave up
constexpr int kStatusScatNoConverge = 2;  // the scattering-source refinement hit its round limit

// Scale of the far-wing prefactors and offsets: K = 2^36/k^2 with k = c/dv_D, U = 2^36 u^2.
constexpr float kKScale = 68719476736.0f;

// Mixed-precision line-kernel tiling.
struct Tiling {
    int J = 4;       // lambda points per thread (contiguous)
    int DS = 6;      // depths per warp (even: the far-wing kernels work on depth pairs)
    int GW = 4;      // warps per CTA (each a depth slab)
    int LC = 32;     // lines per shared-memory chunk (forward)
    int LCB = 32;    // lines per shared-memory chunk (backward)
    int minb = 4;    // minimum resident CTAs per SM the kernels are compiled for
    int lambda_per_tile() const { return 32 * J; }
    int depth_per_cta() const { return DS * GW; }
};

// Device copy of the per-line data.  Every star owns a contiguous segment of lines
// sorted by fractional centre index; orig maps a line to its master (caller) index.
struct LineTable {
    int64_t n = 0;              // lines kept over all stars (windows intersect the grid)
    int32_t *orig = nullptr;    // master index of each line
    int32_t *star = nullptr;    // star of each line
    float *ilf = nullptr;       // integer centre i_l as float (exact, |i_l| < 2^24)
    int32_t *il32 = nullptr;    // integer centre i_l
    float *frac = nullptr;      // x_l - i_l in [-1/2, 1/2)
    int32_t *sp = nullptr;      // species
    float *E = nullptr;         // E_low, eV
    float *lamcm = nullptr;     // lambda_l, cm (FP32)
    float *grad = nullptr;      // gamma_rad 10^dlog_gamma_rad, s^-1
    float *g4 = nullptr;        // gamma_4 10^dlog_gamma4
    float *gradbase = nullptr;  // 10^log_gamma_rad (uncorrected)
    float *g4base = nullptr;    // 10^log_gamma4 (uncorrected)
    float *g6base = nullptr;    // 10^log_gamma6 (uncorrected)
    float *g6 = nullptr;        // 10^(log_gamma6 + dlog_gamma6)
    float *Q = nullptr;         // (pi e^2/m_e c)/sqrt(pi) lambda_l gf_l 10^dlog_gf (FP32)
    double *Qbase = nullptr;    // same without the correction, FP64
    double *x64 = nullptr;      // x_l, FP64 (plain FP64 form)
    float *lg_gf = nullptr;     // log10 gf (caller value; FP64 form)
    float *lg_rad = nullptr, *lg_4 = nullptr, *lg_6 = nullptr;
    float *dgf = nullptr, *dg6 = nullptr;  // current corrections (per line)
    float *dgrad = nullptr, *dg4 = nullptr;
};

// A pair of profiler events around one launch and the kernel family it times.
struct ProfMark {
    cudaEvent_t a, b;
    int kid;
};

// Captured corrections + fwd + loss + bwd + update step (pz_calib_step), re-captured
// when any of its arguments changes or profiling is switched.  With profiling on at
// capture, the graph records its own event pairs around each kernel family (marks),
// read after every launch.
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    const void *key[6] = {nullptr};
    float lr[3] = {0.0f, 0.0f, 0.0f};
    int64_t n = -1;
    int32_t launches = 0;
    bool prof = false;
    std::vector<ProfMark> marks;
};

}  // namespace pz

struct pz_ctx {
    int device = 0;
    pz_precision prec = PZ_MIXED;
    int S = 1;                    // stars
    int nd = 0, ns = 0;
    int64_t nlam = 0, ld = 0;     // grid points, padded row stride of [nd][ld] buffers
    double lambda0_nm = 0, R = 0, lnr = 0;
    int W = 0;
    int64_t nl_caller = 0;        // master lines (gradient output size)
    int64_t n_evals = 0;
    pz::Tiling tiling;
    int n_sm = 0;

    // host copies (small)
    std::vector<double> h_m, h_T;          // [S][nd]
    std::vector<int32_t> h_il;             // [L.n] integer centres, sorted within each star
    std::vector<int64_t> h_line_off;       // [S+1] star segments of the line table
    std::vector<float> h_invdv;            // [S][ns][nd] 1/dv_D (thresholds)

    // device: depth and species tables, strided by star
    double *d_m = nullptr, *d_T = nullptr;                      // [S][nd]
    float *d_beta_hi = nullptr, *d_beta_lo = nullptr;           // [S][nd] eV/(k T) split hi + lo
    float *d_ne = nullptr, *d_npert = nullptr, *d_c2T = nullptr; // [S][nd]
    double *d_ne64 = nullptr, *d_npert64 = nullptr, *d_rho64 = nullptr;  // [S][nd]
    float *d_R = nullptr;           // [S][ns][nd] (1/dv_D) (pop/rho) 10^dabund
    double *d_Rbase = nullptr;      // [S][ns][nd] (1/dv_D)(pop/rho), FP64
    float *d_invdv = nullptr;       // [S][ns][nd] 1/dv_D (s/cm)
    float *d_Ksd = nullptr;         // [S][ns][nd] K = 2^36/k^2, k = c/dv_D (far-wing prefactors)
    double *d_pop64 = nullptr;      // [S][ns][nd]
    double *d_mass64 = nullptr;     // [S][ns]
    double *d_xi64 = nullptr;       // [S]
    float *d_thr = nullptr;         // [S][ns][nslab] fast-path distance threshold (grid units)
    int nslab = 0;                  // depth slabs of DS layers covered by the launch grid
    double *d_kc = nullptr;         // [S][nd][ld] continuum opacity FP64
    double *d_B = nullptr;          // [S][nd][ld] Planck function B_lambda(T_d) per nm, FP64
    double *d_stim = nullptr;       // [S][nd][ld] stimulated-emission factor 1 - exp(-hc/(lambda k T_d)), FP64
    double *d_sigma = nullptr;      // [S][nd][ld] continuum scattering FP64, or NULL (S = B)
    double *d_dab = nullptr;        // [n_elem] current abundance offsets
    float *d_mdgf = nullptr, *d_mdg6 = nullptr;   // [nl_caller] current line corrections, caller order
    float *d_mdgrad = nullptr, *d_mdg4 = nullptr; // [nl_caller] radiative and Stark corrections, caller order
    // linked correction groups: group of each caller line (-1: none) and the members of
    // each group as CSR over caller lines
    int32_t *d_grp_of = nullptr;    // [nl_caller]
    int64_t *d_grp_off = nullptr;   // [n_groups + 1]
    int32_t *d_grp_mem = nullptr;   // [members]
    int64_t n_groups = 0;
    int32_t *d_eos = nullptr;       // [ns] element of species (or -1)
    int n_elem = 0;

    pz::LineTable L;
    int64_t *d_line_off = nullptr;  // [S+1]
    // work items (star, tile * groups + group, lo, hi), longest first
    // (far-wing items with many lines are split into pieces of their line range, so that
    // the queue holds several items per resident CTA; see build_items)
    int4 *d_fitems = nullptr;       // far-wing forward pieces
    int4 *d_fext = nullptr;         // per forward piece: (first slot, pieces, item counter, piece)
    int4 *d_bitems = nullptr;       // far-wing backward pieces (those holding lines)
    int4 *d_nitems_f = nullptr;     // near-core forward
    int4 *d_nitems_b = nullptr;     // near-core backward
    int n_fitems = 0, n_bitems = 0, n_nitems_f = 0, n_nitems_b = 0;
    float4 *d_fpart = nullptr;      // compensated partial sums of the split forward items
    size_t fpart_cap = 0;           // bytes allocated at d_fpart
    int *d_fcnt = nullptr;          // [n_fsplit] pieces finished per split forward item
    int n_fsplit = 0;
    int *d_ctr = nullptr;           // [4] work-queue counters
    int ntiles = 0, tileT = 0;
    float *d_knear = nullptr;       // [S][nd][ld] near-core sums of the forward

    // resident buffers
    void *d_kline = nullptr;        // [S][nd][ld] float (MIXED) or double (FP64)
    double *d_F = nullptr, *d_Fc = nullptr;   // [S][nlam]
    double *d_g = nullptr, *d_gc = nullptr;   // [S][n_out] instrument outputs
    int64_t n_out = 0;
    bool identity_inst = true;
    // instrument weights (shared by all stars)
    int64_t n_pix = 0, pix_cap = 0;
    int32_t max_taps = 0;
    int32_t *d_tap0 = nullptr, *d_ntap = nullptr;
    float *d_tapw = nullptr;        // [n_pix][max_taps]
    double inst_key[3] = {0, 0, 0};
    std::vector<double> pix_key;

    // backward scratch
    double *d_dFbar = nullptr;      // [S][nlam]
    float *d_Gt = nullptr;          // [S][nd][ld] G * stim (FP32, MIXED)
    double *d_Gt64 = nullptr;       // [S][nd][ld] (FP64 form)
    double *d_gacc = nullptr;       // [6][L.n] per table line: (gf, vdW) of the first pass, then
                                    // (unused, rad) and (unused, Stark) of the four-family passes
    double *d_gline = nullptr;      // [4][nl_caller] summed over stars, caller order: gf, vdW, rad, Stark
    int bwd_dsel = 0;               // damping family of the line backward pass (0 vdW, 1 rad, 2 Stark)
    int64_t gacc_off = 0;           // its offset into d_gacc
    double *d_gab = nullptr;        // [n_elem]
    float *d_dLdf = nullptr;        // [S][n_out] seed of the captured step

    // state
    bool have_kline = false, have_flux = false, have_inst = false;
    bool have_gt = false;                // G (dL/dkappa_line) holds a reverse pass
    void *d_finfo = nullptr;             // far-wing line records [depth groups][lines]
    size_t finfo_cap = 0;                // its size in bytes
    int32_t *d_status = nullptr;         // device status word (bounded-wait failures), read by pz_sync_status
    uint32_t *d_keep = nullptr;          // centre test: bit d of word [l][d / 32] set if (l, d) is kept; NULL = off
    double centre_eta = 0.0;             // its selection fraction (0 = off)
    int32_t launches = 0;
    pz::StepGraph graph;
    pz::StepGraph ggraph;                // captured group evaluation (pz_group_eval)
    cudaStream_t cap_stream = nullptr;   // private stream the step graph is captured on
    bool capturing = false;              // a step graph is being captured

    // CUDA-event profiler (pz_set_profiling)
    bool profiling = false;
    std::vector<pz::ProfMark> marks;      // recorded, not yet folded
    std::vector<pz::ProfMark> cap_marks;  // recorded into the graph being captured
    std::vector<cudaEvent_t> ev_pool; // free events
    double k_ms[PZ_NK] = {0};
    int64_t k_count[PZ_NK] = {0};
};

namespace pz {

// profiler brackets around a launch (pz_api.cu); no-ops unless profiling is on
cudaEvent_t prof_begin(pz_ctx *c, cudaStream_t s);
void prof_end(pz_ctx *c, cudaStream_t s, int kid, cudaEvent_t begin);

// error reporting (pz_api.cu)
pz_status fail(pz_status st, const std::string &msg);
pz_status cuda_check(cudaError_t e, const char *what);

// one-time per-device constant tables (pz_line.cu: Voigt; pz_rt.cu: E_n)
pz_status ensure_device_tables();
pz_status ensure_expn_table();

// launches (return cudaGetLastError() of the launch)
cudaError_t launch_line_fwd_mixed(pz_ctx *c, cudaStream_t s);
cudaError_t launch_line_bwd_mixed(pz_ctx *c, cudaStream_t s);
cudaError_t launch_line_fwd_fp64(pz_ctx *c, cudaStream_t s);
cudaError_t launch_line_bwd_fp64(pz_ctx *c, cudaStream_t s);
cudaError_t launch_apply_corrections(pz_ctx *c, cudaStream_t s);
cudaError_t launch_probe_voigt(const float *a, const float *v, int64_t n, float *H, float *dH,
                               cudaStream_t s);

cudaError_t launch_flux(pz_ctx *c, cudaStream_t s);
cudaError_t launch_planck_tables(pz_ctx *c, cudaStream_t s);   // fills d_B and d_stim
cudaError_t launch_inst_build(pz_ctx *c, const double *d_pix, double v_r, double v_b, double R_lsf,
                              int32_t *d_err, cudaStream_t s);
cudaError_t launch_inst_apply(pz_ctx *c, float *f, cudaStream_t s);
cudaError_t launch_loss(pz_ctx *c, const float *y, const float *w, int64_t n, double *loss,
                        float *dLdf, cudaStream_t s);
cudaError_t launch_inst_adjoint(pz_ctx *c, const float *dLdf, cudaStream_t s);
cudaError_t launch_rt_adjoint(pz_ctx *c, cudaStream_t s);
cudaError_t launch_grad_finalize(pz_ctx *c, float *g_gf, float *g_g6, float *g_ab, cudaStream_t s, bool four = false,
                                 float *g_rad = nullptr, float *g_g4 = nullptr);
cudaError_t launch_group_gather(pz_ctx *c, const float *x, cudaStream_t s);
cudaError_t launch_group_reduce(pz_ctx *c, float *g, cudaStream_t s);
cudaError_t launch_update(pz_ctx *c, float lr_gf, float lr_g6, float lr_ab, cudaStream_t s);
cudaError_t launch_probe_expn(const double *x, int64_t n, double *out, cudaStream_t s);
constexpr int kProbeThreads = 256;   // threads per CTA of the pipe-throughput probe
cudaError_t launch_probe_pipe(int kind, int iters, int blocks, float *out, cudaStream_t s);
cudaError_t launch_probe_wait(uint64_t limit_ns, int32_t *status, cudaStream_t s);
constexpr int kKeepWords = kMaxDepth / 32;   // centre-test mask words per line
cudaError_t launch_centre_mask(pz_ctx *c, double eta, unsigned long long *d_count, cudaStream_t s);
bool tiling_supported(int J, int DS, int minb);
bool tiling_fits(const Tiling &t);   // both far-wing chunks fit in shared memory
size_t far_info_bytes(const pz_ctx *c);

}  // namespace pz

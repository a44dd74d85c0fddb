// pz_line.cu -- windowed Voigt line-opacity sum (Eqs. 4-5) and its adjoint
// (Sec. 6), FP32-mixed and plain FP64 forms, plus the per-device Voigt tables.
//
// Mixed-precision kernels.  The work is a queue of items (star, lambda tile,
// depth group, line range) built on the host: lines are sorted by centre
// within each star, and an item's range [lo, hi) holds the star's lines whose
// window |i - i_l| <= W touches the tile (binary search).  The kernels are
// persistent: every CTA takes the next item from an atomic counter until the
// queue is empty, and the items are ordered longest first, so stars and tiles
// of very different line counts share one launch.  A far-wing item covers a
// tile of T = 32 J grid points and GW x DS layers; warp w sweeps layers
// [d0 + w DS, d0 + (w+1) DS) and lane l owns the J contiguous points
// t0 + l J + [0, J).  Lines are staged into shared memory LC at a time: the
// CTA first computes the per-(line, depth) prefactors of Eqs. 4-5 (strength A,
// damping a, Doppler factor c/dv_D and the pre-scaled far-wing polynomial
// coefficients) once for the whole tile, then every thread accumulates its
// J x DS (lambda, depth) sums in registers.  Whether a line is entirely inside
// its window and in the far wing (|v| >= 20 at every depth of the warp's slab)
// over the whole tile is decided once per line and warp.  Per-chunk FP32
// partial sums are folded into a compensated (hi, lo) pair (2Sum).  The
// frequency offset is formed in index space: v = expm1((x_l - i) ln r) c/dv_D
// with x_l - i = (i_l - i) + frac_l, the integer part exact, avoiding the
// cancellation of lambda_l/lambda_i - 1.
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "pz_internal.h"
#include "pz_voigt.cuh"

namespace pz {

// ---------------------------------------------------------------------------
// Host construction of the tables (FP64), once per device.
// ---------------------------------------------------------------------------

// Weideman coefficients: Fourier cosine coefficients of psi(t) = (L^2 + t^2) e^{-t^2}
// under t = L tan(theta/2), L = (N/sqrt 2)^(1/2), by the midpoint rule on 8N points.
static void weideman_coeffs(int N, std::vector<double> &a, double &L) {
    L = std::sqrt(N / std::sqrt(2.0));
    int M = 4 * N;
    a.assign(N + 1, 0.0);
    for (int k = 0; k < 2 * M; ++k) {
        double th = kPI * (k - M + 0.5) / M;
        double t = L * std::tan(0.5 * th);
        double psi = (L * L + t * t) * std::exp(-t * t);
        for (int n = 0; n <= N; ++n) a[n] += psi * std::cos(n * th);
    }
    for (int n = 0; n <= N; ++n) a[n] /= 2 * M;
}

// Dawson's integral D(x) = e^{-x^2} Int_0^x e^{t^2} dt = x Int_0^1 e^{-x^2 (1 - s^2)} ds,
// composite 8-point Gauss-Legendre on 256 panels.
static double dawson_quad(double x) {
    static const double gx[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                                 -0.1834346424956498, 0.1834346424956498,  0.5255324099163290,
                                 0.7966664774136267,  0.9602898564975363};
    static const double gw[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                                 0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                                 0.2223810344533745, 0.1012285362903763};
    const int P = 256;
    double sum = 0.0, h = 1.0 / P;
    for (int p = 0; p < P; ++p)
        for (int k = 0; k < 8; ++k) {
            double s = (p + 0.5 * (gx[k] + 1.0)) * h;
            sum += 0.5 * h * gw[k] * std::exp(-x * x * (1.0 - s * s));
        }
    return x * sum;
}

// Node coefficients D^(k)(x_j)/k! from D' = 1 - 2xD, D^(k+1) = -2x D^(k) - 2k D^(k-1),
// stored coefficient-major: tab[k * kDawsonNodes + j].
static void dawson_table(std::vector<float> &tab) {
    tab.assign(kDawsonNodes * (kDawsonK + 1), 0.0f);
    for (int j = 0; j < kDawsonNodes; ++j) {
        double x = (double)j / kDawsonPerUnit;
        double D[kDawsonK + 2];
        D[0] = dawson_quad(x);
        D[1] = 1.0 - 2.0 * x * D[0];
        for (int k = 1; k < kDawsonK; ++k) D[k + 1] = -2.0 * x * D[k] - 2.0 * k * D[k - 1];
        double fact = 1.0;
        for (int k = 0; k <= kDawsonK; ++k) {
            if (k > 0) fact *= k;
            tab[k * kDawsonNodes + j] = (float)(D[k] / fact);
        }
    }
}

pz_status ensure_device_tables() {
    static std::mutex mu;
    static bool host_ready = false;
    static std::vector<float> weid, daw;
    static std::vector<double> weid64;
    static float weidL;
    static double weidL64;
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(mu);
    if (!host_ready) {
        std::vector<double> a;
        double L;
        weideman_coeffs(kWeidN, a, L);
        weid.assign(a.begin(), a.end());
        weidL = (float)L;
        weideman_coeffs(kWeidN64, weid64, weidL64);
        dawson_table(daw);
        host_ready = true;
    }
    if (dev < 0 || dev >= 64) return fail(PZ_EINVAL, "device ordinal out of range");
    if (done[dev]) return PZ_OK;
    if ((e = cudaMemcpyToSymbol(c_weid, weid.data(), sizeof(float) * (kWeidN + 1))) != cudaSuccess ||
        (e = cudaMemcpyToSymbol(c_weidL, &weidL, sizeof(float))) != cudaSuccess ||
        (e = cudaMemcpyToSymbol(c_weid64, weid64.data(), sizeof(double) * (kWeidN64 + 1))) != cudaSuccess ||
        (e = cudaMemcpyToSymbol(c_weidL64, &weidL64, sizeof(double))) != cudaSuccess ||
        (e = cudaMemcpyToSymbol(g_dawson, daw.data(), sizeof(float) * daw.size())) != cudaSuccess)
        return cuda_check(e, "upload Voigt tables");
    done[dev] = true;
    return PZ_OK;
}

// ---------------------------------------------------------------------------
// Mixed-precision kernels
// ---------------------------------------------------------------------------

struct LineInfo;

// Kernel arguments.  Line arrays are indexed by absolute line; the per-star tables
// and buffers point at star 0 and are advanced by star_view().
struct LineArgs {
    int64_t nlam, ld;
    int nd, W;
    float lnr, lam0cm;
    const float *ilf, *frac, *E, *lamcm, *grad, *g4, *g6, *Q;
    const int32_t *sp;
    const float *R, *invdv, *thr;                   // [ns][nd], [ns][nd], [ns][nslab] of the star
    const float *Ksd;                               // [ns][nd] K = 2^36/k^2 of the star
    int nslab;
    const float *beta_hi, *beta_lo, *ne, *npert, *c2T;   // [nd] of the star
    float *kline;                                   // forward output [nd][ld] of the star
    float *knear;                                   // near-core sums [nd][ld] of the star
    const float *Gt;                                // backward input [nd][ld] of the star
    double *gacc;                                   // backward output [2][nl]
    int64_t nl;
    // work queue: items (star, tile * ngroups + group, lo, hi), longest first
    const int4 *items;
    const int4 *fext;                               // forward pieces: (first slot, pieces, counter, piece)
    float4 *fpart;                                  // partial sums of split forward items [slot][DS][threads][2]
    int *fcnt;                                      // pieces finished per split forward item
    int n_items, ngroups;
    int *ctr;
    int64_t sstride, dstride, bstride, tstride;     // per-star strides of the tables above
    float rj[4], rm1j[4];                           // r^-j and r^-j - 1, j = 0..3 (r = 1 + 1/R)
    const int32_t *star;                            // [nl] star of each line
    const LineInfo *finfo;                          // far-wing line records [ngroups][nl] (k_far_info)
    int *status;                                    // device status word (bounded-wait failures)
    const uint32_t *keep;                           // centre-test mask [nl][kKeepWords] or NULL (all kept)
    int dsel;                                       // backward: damping family of the second sum
                                                    // (0 van der Waals, 1 radiative, 2 Stark)
};

// Centre-test decision of the pair (l, d): kept unless a mask is set and its bit is clear.
__device__ __forceinline__ bool pair_kept(const uint32_t *keep, int64_t l, int d) {
    return !keep || ((keep[l * kKeepWords + (d >> 5)] >> (d & 31)) & 1u);
}

__device__ __forceinline__ LineArgs star_view(const LineArgs &g, int s) {
    LineArgs v = g;
    v.R += s * g.sstride;
    v.invdv += s * g.sstride;
    v.Ksd += s * g.sstride;
    v.thr += s * g.tstride;
    v.beta_hi += s * g.dstride;
    v.beta_lo += s * g.dstride;
    v.ne += s * g.dstride;
    v.npert += s * g.dstride;
    v.c2T += s * g.dstride;
    v.kline += s * g.bstride;
    v.knear += s * g.bstride;
    v.Gt += s * g.bstride;
    return v;
}

// Persistent work loop: every CTA takes the next item of the queue until it is empty
// (or until f, if it returns a flag, returns false -- uniformly over the CTA).
template <class F>
__device__ __forceinline__ void for_each_item(const LineArgs &g, F &&f) {
    __shared__ int s_it;
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(g.ctr, 1);
        __syncthreads();
        const int it = s_it;
        __syncthreads();
        if (it >= g.n_items) break;
        const int4 item = g.items[it];
        using R = decltype(f(star_view(g, item.x), 0, 0, 0, 0, 0));
        if constexpr (std::is_same<R, bool>::value) {
            if (!f(star_view(g, item.x), item.y / g.ngroups, item.y % g.ngroups, item.z, item.w, it)) break;
        } else {
            f(star_view(g, item.x), item.y / g.ngroups, item.y % g.ngroups, item.z, item.w, it);
        }
    }
}

// Per-(line, depth) prefactors.  NP = 8 (forward) or 16 (backward):
//  [0] k = c/dv_D   [1] a^2   [2..6] B1..B5 = A a/sqrt(pi) x (1, 1.5, 3.75-2a^2, -15a^2, 12a^4)
//  [7] A            (backward:) [8..13] C1..C6 = A a6/sqrt(pi) x (1, 1.5-2a^2, 3.75-12a^2,
//  12a^4-67.5a^2, 180a^4, -120a^6)   [14] A a6   [15] a
// where a6 is the part of a that the selected damping family contributes (Eq. 10 scales
// one family by 10^delta, so d a / d delta = ln10 a6): van der Waals gamma6 n_pert,
// radiative gamma_rad or Stark gamma4 n_e, over 4 pi dnu_D.
// Per-line scalars of the prefactors (one load per line, shared by its depths).
struct LineScalars {
    int sp;
    float E, Q, lamcm, g4, grad, g6;
};
__device__ __forceinline__ LineScalars load_line(const LineArgs &g, int64_t l) {
    LineScalars L;
    L.sp = g.sp[l];
    L.E = g.E[l];
    L.Q = g.Q[l];
    L.lamcm = g.lamcm[l];
    L.g4 = g.g4[l];
    L.grad = g.grad[l];
    L.g6 = g.g6[l];
    return L;
}

// The damping products are rounded explicitly (no contraction), so that every kernel
// that classifies a cell by |v|^2 + a^2 -- the far-wing and near-core passes -- forms
// k and a^2 with identical roundings.
template <int NP>
__device__ __forceinline__ void depth_params(const LineArgs &g, const LineScalars &L, int d, float *out) {
    if (d >= g.nd) {
#pragma unroll
        for (int k = 0; k < NP; ++k) out[k] = 0.0f;
        out[1] = 1.0f;
        return;
    }
    const int id = L.sp * g.nd + d;
    const float invdv = __ldg(g.invdv + id);
    const float bh = __ldg(g.beta_hi + d), bl = __ldg(g.beta_lo + d);
    const float p = L.E * bh;
    const float r = fmaf(L.E, bh, -p) + L.E * bl;      // E beta = p + r
    const float boltz = expf(-p) * (1.0f - r);
    const float A = L.Q * __ldg(g.R + id) * boltz;
    const float lw = __fmul_rn(__fmul_rn(L.lamcm, invdv), (float)(1.0 / (4.0 * kPI)));
    const float g6n = __fmul_rn(L.g6, __ldg(g.npert + d));
    const float a = __fmul_rn(fmaf(L.g4, __ldg(g.ne + d), __fadd_rn(L.grad, g6n)), lw);
    const float a2 = __fmul_rn(a, a);
    const float B1 = A * a * kInvSqrtPiF;
    out[0] = __fmul_rn((float)kC, invdv);
    out[1] = a2;
    out[2] = B1;
    out[3] = 1.5f * B1;
    out[4] = fmaf(-2.0f, a2, 3.75f) * B1;
    out[5] = -15.0f * a2 * B1;
    out[6] = 12.0f * a2 * a2 * B1;
    out[7] = A;
    if (NP == 16) {
        const float gb = g.dsel == 0 ? g6n : (g.dsel == 1 ? L.grad : __fmul_rn(L.g4, __ldg(g.ne + d)));
        const float Aa6 = A * gb * lw;
        const float C1 = Aa6 * kInvSqrtPiF;
        out[8] = C1;
        out[9] = fmaf(-2.0f, a2, 1.5f) * C1;
        out[10] = fmaf(-12.0f, a2, 3.75f) * C1;
        out[11] = a2 * fmaf(12.0f, a2, -67.5f) * C1;
        out[12] = 180.0f * a2 * a2 * C1;
        out[13] = -120.0f * a2 * a2 * a2 * C1;
        out[14] = Aa6;
        out[15] = a;
    }
}

template <int NP>
__device__ __forceinline__ void line_params(const LineArgs &g, int64_t l, int d, float *out) {
    depth_params<NP>(g, load_line(g, l), d, out);
}

// index-space frequency offset u = lambda_l/lambda_i - 1 = expm1(Delta ln r)
__device__ __forceinline__ float offset_u(float delta, float lnr) {
    float y = delta * lnr;
    return fmaf(y * y, fmaf(y, 0.16666667f, 0.5f), y);
}

// Line record of the far-wing tables: centre, species and the per-slab reduced-form
// mask of the line's depth group.
struct alignas(16) LineInfo {
    float ilf, frac;
    int sp, amask;
};

// ---- packed FP32 pairs ------------------------------------------------------
// The far-wing kernels evaluate two depths of one (line, lambda) cell with one
// instruction: a register pair {value at depth d, value at depth d + 1} and the
// f32x2 forms of mul and fma (each half rounded exactly as the scalar op).  This
// halves the FP32 issue slots of the inner loop; the two reciprocals stay scalar.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// reciprocal of both halves (rcp.approx.ftz, as rcp_approx)
__device__ __forceinline__ f2_t f2_rcp(f2_t a) {
    f2_t r;
    asm("{\n\t.reg .f32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\trcp.approx.ftz.f32 lo, lo;\n\t"
        "rcp.approx.ftz.f32 hi, hi;\n\tmov.b64 %0, {lo, hi};\n\t}"
        : "=l"(r) : "l"(a));
    return r;
}
__device__ __forceinline__ f2_t f2_splat(float v) { return f2_pack(v, v); }
__device__ __forceinline__ float f2_lo(f2_t v) {
    float lo, hi;
    f2_unpack(v, lo, hi);
    return lo;
}
__device__ __forceinline__ float f2_hi(f2_t v) {
    float lo, hi;
    f2_unpack(v, lo, hi);
    return hi;
}

// ---- far-wing prefactors ------------------------------------------------------
// A far-wing CTA stages LC lines at a time.  For each line of the chunk and each of
// the (DC/2) depth pairs of its group it forms NQ quads, quad q holding
// {p_2q(d), p_2q(d + 1), p_2q+1(d), p_2q+1(d + 1)} (one 16-byte shared-memory load
// returns the packed depth pairs of two parameters):
//   forward  (NQ = 2): (K, a^2) (B1 K, B2' K^2)
//   backward (NQ = 3): (K, a^2) (B1 K, B2' K^2) (C1 K, C2' K^2)
// with k = c/dv_D, K = 2^36/k^2 (the power of two keeps every product of the
// prefactors and of the offsets far from the FP32 exponent limits), B2' = B2 - B1 a^2
// = B1 (1.5 - a^2) and C2' = C2 - C1 a^2 = C1 (1.5 - 3a^2).  The far kernels take the
// squared offsets scaled alike, U = 2^36 u^2, so that with s = 1/U
//   reduced form:  H sqrt(pi)/A = (B1 K) s + (B2' K^2) s^2   (p = K s exactly, see below)
//   full form:     r = 1/(U + a^2 K) and t = 1/|z|^2 = K r, so B1 t (...) = (B1 K) r (...)
// and the masked lines recover B1 = (B1 K) k^2 2^-36 (and C1 alike) per depth pair.
// Each warp stages the quads of its own slab, par[li][pair][q] in its part of shared
// memory; the rest of the far polynomial (B3..B5, C3..C6) follows from a^2 and B1 K
// (C1 K) in registers.  Lane li computes line li's quads from the line data and the
// star's per-(species, depth) tables (Eqs. 4-5, with the roundings of depth_params), so
// no per-(line, depth) array exists in device memory: the quads are recomputed for each
// tile the line's window reaches.  The only per-line device array of the far kernels is
// the 16-byte line record of each depth group (k_far_info).
constexpr int kNQF = 2, kNQB = 3;
constexpr int kBwdBatch = 16;   // lines per transposed partial-sum batch of the far-wing backward (2 lanes per line)
constexpr float kUScale = 262144.0f;              // 2^18: scaled offset u 2^18
constexpr float kKUnscale = 1.4551915228366852e-11f;   // 2^-36

// Reduced far-wing form.  Far from the core the polynomial in t = 1/|z|^2 is cut
// after its t^2 term: H sqrt(pi)/(A a) = t (1 + 1.5 t) and, for dH/da, C1 t (1 +
// (1.5 - 2a^2) t).  With |v| >= 100 (t <= 1e-4) and a^2 <= 1.5 (s = a^2 t <= 1.5e-4)
// the dropped terms, (3.75 t^2 + 2 s t + 15 s t^2 + 12 s^2 t^2) relative for H, stay
// below 7e-8 (about one FP32 rounding) and below 2.2e-7 for dH/da.
// In the same region t is expanded about p = 1/(u k)^2 = (1/U) K:
// t = p/(1 + a^2 p) = p - a^2 p^2 + O((a^2 p)^2 p), so that
//   H sqrt(pi)/A = B1 p + B2' p^2 = (B1 K) s + (B2' K^2) s^2,   s = 1/U,
// and dH/da sqrt(pi)/(A a6) = (C1 K) s + (C2' K^2) s^2, with B2' = B1 (1.5 - a^2),
// C2' = C1 (1.5 - 3a^2); the further dropped terms, (a^2 p)^2 and 3 a^2 p^2 relative,
// stay below 5e-8.  s and s^2 depend on the line and the point only, so one MUFU
// reciprocal serves all the depths of a warp, and the forward adds two products per
// cell.  In the backward the sums over the cells of one depth factor:
//   sum_i G_i [(B1 K) s_i + (B2' K^2) s_i^2] = (B1 K) X1 + (B2' K^2) X2,
//   X1 = sum_i G_i s_i,  X2 = sum_i G_i s_i^2,
// and X1, X2 serve both gradients (the C coefficients multiply the same sums).
constexpr float kFast2V = 5.0f;      // distance threshold factor: |v| >= 5 x 20
// Three-term reduced form, for the lines between 30 and 100 Doppler widths from the tile:
// the same expansion one order further,
//   H sqrt(pi)/A = (B1 K) s + (B2' K^2) s^2 + (B3' K^3) s^3,  B3' = B1 (3.75 - 5a^2 + a^4),
//   dH/da sqrt(pi)/(A a6) = (C1 K) s + (C2' K^2) s^2 + (C3' K^3) s^3,  C3' = C1 (3.75 - 15a^2 + 5a^4),
// (the t^3 terms of the far polynomial and the p^3 terms of t and t^2 in p).  Against the
// five-term polynomial the dropped p^4 terms stay below 2.6e-8 relative for H and 4.6e-8 for
// dH/da at |v| >= 30 and a^2 <= 1.5 (evaluated on a dense (a^2, v) lattice).  B3' K^3 and
// C3' K^3 are formed per depth pair from K, a^2, B1 K and C1 K.
constexpr float kFast3V = 1.5f;      // distance threshold factor: |v| >= 1.5 x 20
constexpr float kFast2A2 = 1.5f;     // a^2 bound

// One thread per (group, line): the line record, whose amask has bit w set when
// a^2 <= kFast2A2 at every layer of slab w (DS layers) of the group, and bit 8 + w when
// the centre test rejects every layer of slab w (its warp skips the line).
__global__ void k_far_info(LineArgs gq, int DC, int DS, int ngroups, LineInfo *info) {
    const int64_t n = (int64_t)ngroups * gq.nl;
    for (int64_t gl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gl < n; gl += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = gl % gq.nl;
        const int grp = (int)(gl / gq.nl);
        const LineArgs g = star_view(gq, gq.star[l]);
        const LineScalars L = load_line(g, l);
        int amask = 0;
        for (int w = 0; w < DC / DS; ++w) {
            bool ok = true, none = true;
            for (int dd = grp * DC + w * DS; dd < min(grp * DC + (w + 1) * DS, g.nd); ++dd) {
                float q[16];
                depth_params<8>(g, L, dd, q);
                ok = ok && q[1] <= kFast2A2;
                none = none && !pair_kept(g.keep, l, dd);
            }
            amask |= (ok ? 1 << w : 0) | (none ? 1 << (8 + w) : 0);
        }
        LineInfo r;
        r.ilf = g.ilf[l];
        r.frac = g.frac[l];
        r.sp = L.sp;
        r.amask = amask;
        info[gl] = r;
    }
}

// Prefactors of line l at layer d (one half of a depth pair), with the roundings of
// depth_params for k and a^2 (the cells' near / far classification depends on them):
// K = 2^36/k^2, a^2, B1 K, B2' K^2 and (NQ = kNQB) C1 K, C2' K^2.  dc holds the layer's
// {beta_hi, beta_lo, n_e, n_pert}.  Layers past the last one get K = 0, a^2 = 1 and zero
// coefficients, pairs rejected by the centre test zero coefficients.
template <int NQ>
__device__ __forceinline__ void far_depth_prefactors(const LineArgs &g, const LineScalars &L, int64_t l, int d,
                                                     const float4 dc, float &K, float &a2, float &b1, float &b2,
                                                     float &c1, float &c2) {
    if (d >= g.nd) {
        K = 0.0f;
        a2 = 1.0f;
        b1 = b2 = c1 = c2 = 0.0f;
        return;
    }
    const int id = L.sp * g.nd + d;
    const float invdv = __ldg(g.invdv + id);
    const float p = L.E * dc.x;
    const float r = fmaf(L.E, dc.x, -p) + L.E * dc.y;      // E beta = p + r
    const float boltz = expf(-p) * (1.0f - r);
    const float A = L.Q * __ldg(g.R + id) * boltz;
    const float lw = __fmul_rn(__fmul_rn(L.lamcm, invdv), (float)(1.0 / (4.0 * kPI)));
    const float g6n = __fmul_rn(L.g6, dc.w);
    const float a = __fmul_rn(fmaf(L.g4, dc.z, __fadd_rn(L.grad, g6n)), lw);
    a2 = __fmul_rn(a, a);
    K = __ldg(g.Ksd + id);
    const float KK = K * K;
    const bool kept = pair_kept(g.keep, l, d);
    const float B1 = kept ? A * a * kInvSqrtPiF : 0.0f;
    b1 = B1 * K;
    b2 = fmaf(-B1, a2, 1.5f * B1) * KK;
    if (NQ == kNQB) {
        const float gb = g.dsel == 0 ? g6n : (g.dsel == 1 ? L.grad : __fmul_rn(L.g4, dc.z));
        const float C1 = kept ? A * gb * lw * kInvSqrtPiF : 0.0f;
        c1 = C1 * K;
        c2 = fmaf(-C1, a2, fmaf(-2.0f, a2, 1.5f) * C1) * KK;
    } else {
        c1 = c2 = 0.0f;
    }
}

// Per-warp staging of a chunk of lines.  Each warp keeps, in its own part of shared
// memory, the layer constants of its slab (dc: DS x {beta_hi, beta_lo, n_e, n_pert}),
// and for the chunk's lines their records and the prefactor quads of its DP depth pairs
// (par: [LC][DP][NQ]).  Lane li fills line li (li + 32, ... for chunks over 32 lines); a
// warp barrier publishes the chunk, and the next fill waits on a warp barrier so that
// no lane still reads the previous chunk.  No CTA-wide barrier is involved.
struct WarpStage {
    float4 *dc;          // [DS]
    float4 *par;         // [LC][DP * NQ]
    LineInfo *info;      // [LC]
    int *idx;            // [LC] line of each staged slot (forward: gathered by warp_gather)
};

__host__ __device__ constexpr size_t warp_stage_quads(int LC, int DS, int NQ) {
    return (size_t)DS + (size_t)LC * (DS / 2) * NQ + (size_t)LC + ((size_t)LC + 3) / 4;
}
__device__ __forceinline__ WarpStage make_stage(float4 *mine, int LC, int DS, int NQ) {
    LineInfo *info = reinterpret_cast<LineInfo *>(mine + DS + (size_t)LC * (DS / 2) * NQ);
    return WarpStage{mine, mine + DS, info, reinterpret_cast<int *>(info + LC)};
}

template <int DS>
__device__ __forceinline__ void warp_stage_depths(const LineArgs &g, const WarpStage &ws, int dfirst, int lane) {
    __syncwarp();
    if (lane < DS) {
        const int d = dfirst + lane;
        ws.dc[lane] = d < g.nd ? make_float4(__ldg(g.beta_hi + d), __ldg(g.beta_lo + d), __ldg(g.ne + d),
                                              __ldg(g.npert + d))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
}

// The forward's next chunk: up to LC lines from cur on that slab w has to sweep (all lines
// without the centre test; with it, those with a layer of the slab kept), their indices in
// ws.idx in line order.  Returns the count and leaves cur after the last line looked at.
__device__ __forceinline__ int warp_gather(const WarpStage &ws, const LineInfo *ginfo, int &cur, int hi, int LC,
                                           int w, int lane) {
    int count = 0;
    __syncwarp();
    while (count < LC && cur < hi) {
        const int l = cur + lane;
        const bool need = l < hi && !((ginfo[l].amask >> (8 + w)) & 1);
        const unsigned m = __ballot_sync(0xffffffffu, need);
        const int n = __popc(m);
        const int take = min(n, LC - count);
        const int slot = count + __popc(m & ((1u << lane) - 1u));
        if (need && slot < LC) ws.idx[slot] = l;
        cur += take < n ? __fns(m, 0, take) + 1 : 32;   // after the last line taken
        count += take;
    }
    __syncwarp();
    return count;
}

template <int NQ, int DS>
__device__ __forceinline__ void warp_fill(const LineArgs &g, const WarpStage &ws, const LineInfo *ginfo,
                                          int64_t first, int nl, int dfirst, int lane, bool listed = false) {
    constexpr int DP = DS / 2;
    __syncwarp();
    for (int li = lane; li < nl; li += 32) {
        const int64_t l = listed ? (int64_t)ws.idx[li] : first + li;
        ws.info[li] = ginfo[l];
        const LineScalars L = load_line(g, l);
        float4 *dst = ws.par + (size_t)li * DP * NQ;
#pragma unroll
        for (int dp = 0; dp < DP; ++dp) {
            float K0, K1, a0, a1, b10, b11, b20, b21, c10, c11, c20, c21;
            far_depth_prefactors<NQ>(g, L, l, dfirst + 2 * dp, ws.dc[2 * dp], K0, a0, b10, b20, c10, c20);
            far_depth_prefactors<NQ>(g, L, l, dfirst + 2 * dp + 1, ws.dc[2 * dp + 1], K1, a1, b11, b21, c11, c21);
            dst[NQ * dp] = make_float4(K0, K1, a0, a1);
            dst[NQ * dp + 1] = make_float4(b10, b11, b20, b21);
            if (NQ == kNQB) dst[NQ * dp + 2] = make_float4(c10, c11, c20, c21);
        }
    }
    __syncwarp();
}

// ---- mbarrier waits (the bounded-wait probe) ---------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the barrier to complete; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}


// Per-warp flags of a line over the tile (4: every layer of the slab rejected by the
// centre test, nothing to evaluate): bit 0 if the line's window covers the tile
// and every cell of the warp's slab is in the far wing (|v| >= 20); bit 1 if every
// cell of the slab has |v| >= 100 and a^2 <= kFast2A2 at every layer (reduced form),
// whether or not the window covers the tile: the reduced form masks the window per
// point at no cost per cell (a zero reciprocal s = 1/U); bit 3 if instead every cell
// has |v| >= 30 with the same a^2 bound (three-term reduced form).
__device__ __forceinline__ int far_flags(const LineArgs &g, const LineInfo &info, float t0f, float tendf, int slab,
                                         int w) {
    const float dlo = info.ilf - t0f + info.frac;      // x_l - t0
    const float dhi = info.ilf - tendf + info.frac;    // x_l - (t0 + T - 1)
    const float dmin = fmaxf(0.0f, fmaxf(-dlo, dhi));
    const bool full = (info.ilf - (float)g.W <= t0f) && (info.ilf + (float)g.W >= tendf);
    if ((info.amask >> (8 + w)) & 1) return 4;        // the centre test rejects the whole slab
    const float thr = __ldg(g.thr + info.sp * g.nslab + slab);
    const bool fast = full && dmin >= thr;
    const bool amask = (info.amask >> w) & 1;
    const bool red = dmin >= kFast2V * thr && amask;
    const bool red3 = !red && dmin >= kFast3V * thr && amask;
    return (fast ? 1 : 0) | (red ? 2 : 0) | (red3 ? 8 : 0);
}

// k = c/dv_D of the warp's depth pairs, rounded exactly as depth_params forms it, for the
// masked lines, whose cells are classified near / far with the near-core kernels' own
// arithmetic (x = u k, |z|^2 = x^2 + a^2).  Layers past the last one get 0.
template <int DP>
__device__ __forceinline__ void far_kpairs(const LineArgs &g, int sp, int dfirst, f2_t (&kp)[DP]) {
#pragma unroll
    for (int dp = 0; dp < DP; ++dp) {
        const int da = dfirst + 2 * dp, db = da + 1;
        const float ka = da < g.nd ? __fmul_rn((float)kC, __ldg(g.invdv + sp * g.nd + da)) : 0.0f;
        const float kb = db < g.nd ? __fmul_rn((float)kC, __ldg(g.invdv + sp * g.nd + db)) : 0.0f;
        kp[dp] = f2_pack(ka, kb);
    }
}

// Compensated-sum slots of depth dd of thread tid: the (hi, lo) quads of its J points, hi
// at quad 2 dd nthr + tid and lo at quad (2 dd + 1) nthr + tid, so that the threads of a
// warp touch consecutive quads (16-byte accesses without bank conflicts).  They live in
// shared memory and are touched once per line chunk.
__device__ __forceinline__ float4 *comp_hi(float *s_comp, int dd, int tid, int nthr) {
    return reinterpret_cast<float4 *>(s_comp) + (size_t)(2 * dd) * nthr + tid;
}
__device__ __forceinline__ float4 *comp_lo(float *s_comp, int dd, int tid, int nthr) {
    return reinterpret_cast<float4 *>(s_comp) + (size_t)(2 * dd + 1) * nthr + tid;
}

// Higher far-wing coefficients from a^2 and B1 (as depth_params forms them):
// B3 = (3.75 - 2a^2) B1, B4 = -15 a^2 B1, B5 = 12 a^4 B1.
__device__ __forceinline__ void far_b345(f2_t a2, f2_t B1, f2_t &B3, f2_t &B4, f2_t &B5) {
    B3 = f2_mul(f2_fma(a2, f2_splat(-2.0f), f2_splat(3.75f)), B1);
    B4 = f2_mul(f2_mul(a2, f2_splat(-15.0f)), B1);
    B5 = f2_mul(f2_mul(f2_mul(a2, f2_splat(12.0f)), a2), B1);
}
// C3 = (3.75 - 12 a^2) C1, C4 = a^2 (12 a^2 - 67.5) C1, C5 = 180 a^4 C1, C6 = -120 a^6 C1.
__device__ __forceinline__ void far_c3456(f2_t a2, f2_t C1, f2_t &C3, f2_t &C4, f2_t &C5, f2_t &C6) {
    C3 = f2_mul(f2_fma(a2, f2_splat(-12.0f), f2_splat(3.75f)), C1);
    C4 = f2_mul(f2_mul(a2, f2_fma(a2, f2_splat(12.0f), f2_splat(-67.5f))), C1);
    const f2_t a4 = f2_mul(a2, a2);
    C5 = f2_mul(f2_mul(a4, f2_splat(180.0f)), C1);
    C6 = f2_mul(f2_mul(f2_mul(a4, f2_splat(-120.0f)), a2), C1);
}

// Reciprocals s_j = 1/U_j of the squared scaled offsets of one line at the thread's J
// points (and their squares), for the reduced forms: offsets from the first point's,
// u_j = u_0 r^-j + (r^-j - 1) scaled by 2^18; points outside the line's window get
// s = 0 unless the window covers the tile (full).
template <int J>
__device__ __forceinline__ void far_scaled_u2(const LineArgs &g, const LineInfo &info, float lamf, float (&U)[J]) {
    // scalar chain: the offsets depend on the line and the point only, not on the depth
    const float u0 = offset_u((info.ilf - lamf) + info.frac, g.lnr) * kUScale;
    U[0] = u0 * u0;
#pragma unroll
    for (int j = 1; j < J; ++j) {
        const float u = fmaf(u0, g.rj[j], g.rm1j[j] * kUScale);
        U[j] = u * u;
    }
}

template <int J>
__device__ __forceinline__ void far_reduced_s(const LineArgs &g, const LineInfo &info, bool full, float lamf,
                                              int lam_thr, f2_t (&sp)[J], f2_t (&sq)[J]) {
    float U[J];
    far_scaled_u2<J>(g, info, lamf, U);
    if (full) {
#pragma unroll
        for (int j = 0; j < J; ++j) sp[j] = f2_splat(rcp_approx(U[j]));
    } else {
        const int il = (int)info.ilf;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int di = lam_thr + j - il;
            sp[j] = f2_splat(di >= -g.W && di <= g.W ? rcp_approx(U[j]) : 0.0f);
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) sq[j] = f2_mul(sp[j], sp[j]);
}

// Far-wing kernel (forward).  Every cell with |v|^2 + a^2 >= 400 inside its window is
// evaluated here with the far polynomial; the near-core cells are summed by
// k_line_near_fwd into knear, which this kernel adds before applying stim.
// Returns false if a chunk never arrived (the kernel stops).
template <int J, int DS, bool GATHER>
__device__ __forceinline__ bool far_fwd_item(const LineArgs &g, const int tile, const int group, const int lo,
                                             const int hi, const int GW, const int LC, const WarpStage &ws,
                                             float *s_comp, const int4 ext) {
    static_assert(J == 2 || J == 4, "J must be 2 or 4");
    static_assert(DS % 2 == 0, "DS must be even (depth pairs)");
    constexpr int DP = DS / 2;          // depth pairs per warp
    constexpr int NQ = kNQF;
    const int T = 32 * J;
    const int DC = GW * DS;
    const int nthr = blockDim.x;
    const LineInfo *ginfo = g.finfo + (int64_t)group * g.nl;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int d0 = group * DC;
    const int slab = group * GW + warp;
    const int t0 = tile * T;
    const float t0f = (float)t0, tendf = (float)(t0 + T - 1);
    const int lam_thr = t0 + lane * J;
    const float lamf = (float)lam_thr;

    f2_t acc[DP][J];
#pragma unroll
    for (int dp = 0; dp < DP; ++dp)
#pragma unroll
        for (int j = 0; j < J; ++j) acc[dp][j] = 0ull;
#pragma unroll
    for (int dd = 0; dd < DS; ++dd) {
        *comp_hi(s_comp, dd, tid, nthr) = make_float4(0.f, 0.f, 0.f, 0.f);
        *comp_lo(s_comp, dd, tid, nthr) = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    warp_stage_depths<DS>(g, ws, d0 + warp * DS, lane);
    // chunks of LC lines; with GATHER (a centre test is set) of the lines this warp's slab
    // sweeps, so that lines whose slab the test rejects entirely are neither staged nor visited
    // one chunk of nl staged lines: the cells, then the fold into the compensated sums
    auto chunk = [&](const int nl) {
        const ulonglong2 *s_par = reinterpret_cast<const ulonglong2 *>(ws.par);
        const LineInfo *s_line = ws.info;
        unsigned m_fast = 0u, m_red = 0u, m_red3 = 0u, m_skip = 0u;   // this warp's flags of 32 lines, one per lane
        for (int li = 0; li < nl; ++li) {
            if ((li & 31) == 0) {
                const int lj = li + lane;
                const int f = lj < nl ? far_flags(g, s_line[lj], t0f, tendf, slab, warp) : 0;
                m_fast = __ballot_sync(0xffffffffu, f & 1);
                m_red = __ballot_sync(0xffffffffu, (f & 2) != 0);
                m_red3 = __ballot_sync(0xffffffffu, (f & 8) != 0);
                m_skip = __ballot_sync(0xffffffffu, (f & 4) != 0);
            }
            const unsigned b = li & 31;
            if (b < 31 && li + 1 < nl && ((m_red >> b) & 3u) == 3u && ((m_skip >> b) & 3u) == 0u) {
                // two consecutive two-term lines: their offsets and reciprocals are independent
                // chains, formed together; the sums take line li's terms, then line li + 1's
                f2_t spa[J], sqa[J], spb[J], sqb[J];
                far_reduced_s<J>(g, s_line[li], (m_fast >> b) & 1u, lamf, lam_thr, spa, sqa);
                far_reduced_s<J>(g, s_line[li + 1], (m_fast >> (b + 1)) & 1u, lamf, lam_thr, spb, sqb);
                const ulonglong2 *pa = s_par + (size_t)li * DP * NQ, *pb = pa + DP * NQ;
#pragma unroll
                for (int dp = 0; dp < DP; ++dp) {
                    const ulonglong2 qa = pa[NQ * dp + 1], qb = pb[NQ * dp + 1];
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        acc[dp][j] = f2_fma(sqa[j], qa.y, f2_fma(spa[j], qa.x, acc[dp][j]));
                        acc[dp][j] = f2_fma(sqb[j], qb.y, f2_fma(spb[j], qb.x, acc[dp][j]));
                    }
                }
                ++li;
                continue;
            }
            const LineInfo info = s_line[li];
            const int fl = (int)((m_fast >> b) & 1u) | (int)(((m_red >> b) & 1u) << 1) | (int)(((m_red3 >> b) & 1u) << 2);
            if ((m_skip >> b) & 1u) continue;        // every layer rejected by the centre test
            const ulonglong2 *par = s_par + (size_t)li * DP * NQ;
            // the whole tile in the line's far wing (fl != 0): offsets from the first point's,
            // u_j = u_0 r^-j + (r^-j - 1), scaled by 2^18, and their squares U = 2^36 u^2
            float U[J];
            if (fl != 0) far_scaled_u2<J>(g, info, lamf, U);
            if (fl & 6) {
                // reduced forms (B1 K) s + (B2' K^2) s^2 [+ (B3' K^3) s^3] with s = 1/U; points
                // outside the window (lines whose window edge crosses the tile) get s = 0
                f2_t sp[J], sq[J];
                if (fl & 1) {
#pragma unroll
                    for (int j = 0; j < J; ++j) sp[j] = f2_splat(rcp_approx(U[j]));
                } else {
                    const int il = (int)info.ilf;
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const int di = lam_thr + j - il;
                        sp[j] = f2_splat(di >= -g.W && di <= g.W ? rcp_approx(U[j]) : 0.0f);
                    }
                }
#pragma unroll
                for (int j = 0; j < J; ++j) sq[j] = f2_mul(sp[j], sp[j]);
                if (fl & 2) {
#pragma unroll
                    for (int dp = 0; dp < DP; ++dp) {
                        // q1 = (B1 K, B2' K^2)
                        const ulonglong2 q1 = par[NQ * dp + 1];
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            acc[dp][j] = f2_fma(sq[j], q1.y, f2_fma(sp[j], q1.x, acc[dp][j]));
                    }
                } else {
                    f2_t sc[J];
#pragma unroll
                    for (int j = 0; j < J; ++j) sc[j] = f2_mul(sq[j], sp[j]);
#pragma unroll
                    for (int dp = 0; dp < DP; ++dp) {
                        // q0 = (K, a^2), q1 = (B1 K, B2' K^2); B3' K^3 = (B1 K) K^2 (3.75 - 5a^2 + a^4)
                        const ulonglong2 q0 = par[NQ * dp], q1 = par[NQ * dp + 1];
                        const f2_t b3 = f2_mul(f2_mul(q1.x, f2_mul(q0.x, q0.x)),
                                               f2_fma(q0.y, f2_fma(q0.y, f2_splat(1.0f), f2_splat(-5.0f)),
                                                      f2_splat(3.75f)));
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            acc[dp][j] = f2_fma(sc[j], b3, f2_fma(sq[j], q1.y, f2_fma(sp[j], q1.x, acc[dp][j])));
                    }
                }
            } else if (fl & 1) {
                f2_t u2[J];
#pragma unroll
                for (int j = 0; j < J; ++j) u2[j] = f2_splat(U[j]);
#pragma unroll
                for (int dp = 0; dp < DP; ++dp) {
                    // q0 = (K, a^2), q1 = (B1 K, B2' K^2): the polynomial in t with every
                    // coefficient times K, applied to r = t/K
                    const ulonglong2 q0 = par[NQ * dp], q1 = par[NQ * dp + 1];
                    f2_t B3, B4, B5;
                    far_b345(q0.y, q1.x, B3, B4, B5);
                    const f2_t B2 = f2_mul(q1.x, f2_splat(1.5f));
                    const f2_t ak = f2_mul(q0.y, q0.x);          // a^2 K
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        // r = 1/(U + a^2 K) = 2^-36/(u^2 + a^2/k^2), t = 1/(u^2 k^2 + a^2) = K r
                        const f2_t r = f2_rcp(f2_fma(u2[j], f2_splat(1.0f), ak));
                        const f2_t t = f2_mul(q0.x, r);
                        f2_t h = f2_fma(t, B5, B4);
                        h = f2_fma(t, h, B3);
                        h = f2_fma(t, h, B2);
                        h = f2_fma(t, h, q1.x);
                        acc[dp][j] = f2_fma(r, h, acc[dp][j]);
                    }
                }
            } else {
                // line near the tile or partly outside its window: far cells inside the window
                // only, classified near / far exactly as the near-core kernel does
                f2_t u2[J];
#pragma unroll
                for (int j = 0; j < J; ++j) u2[j] = f2_splat(offset_u((info.ilf - (lamf + (float)j)) + info.frac, g.lnr));
                const int il = (int)info.ilf;
                bool inwin[J];
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int di = lam_thr + j - il;
                    inwin[j] = di >= -g.W && di <= g.W;
                }
                f2_t kp[DP];
                far_kpairs<DP>(g, info.sp, d0 + warp * DS, kp);
#pragma unroll
                for (int dp = 0; dp < DP; ++dp) {
                    const ulonglong2 q0 = par[NQ * dp], q1 = par[NQ * dp + 1];
                    // B1 = (B1 K) k^2 2^-36
                    const f2_t B1 = f2_mul(q1.x, f2_mul(f2_mul(kp[dp], kp[dp]), f2_splat(kKUnscale)));
                    f2_t B3, B4, B5;
                    far_b345(q0.y, B1, B3, B4, B5);
                    const f2_t B2 = f2_mul(B1, f2_splat(1.5f));
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const f2_t x = f2_mul(u2[j], kp[dp]);
                        const f2_t r2 = f2_fma(x, x, q0.y);
                        const f2_t t = f2_rcp(r2);
                        f2_t h = f2_fma(t, B5, B4);
                        h = f2_fma(t, h, B3);
                        h = f2_fma(t, h, B2);
                        h = f2_fma(t, h, B1);
                        const f2_t r = f2_fma(t, h, acc[dp][j]);
                        float r2a, r2b, ra, rb, aa, ab;
                        f2_unpack(r2, r2a, r2b);
                        f2_unpack(r, ra, rb);
                        f2_unpack(acc[dp][j], aa, ab);
                        aa = (inwin[j] && r2a >= kFar2) ? ra : aa;
                        ab = (inwin[j] && r2b >= kFar2) ? rb : ab;
                        acc[dp][j] = f2_pack(aa, ab);
                    }
                }
            }
        }
        // fold the chunk partials into the compensated sums (2Sum; the rounding
        // terms accumulate in this thread's shared-memory slots)
#pragma unroll
        for (int dp = 0; dp < DP; ++dp) {
            float pa[J], pb[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                f2_unpack(acc[dp][j], pa[j], pb[j]);
                acc[dp][j] = 0ull;
            }
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int dd = 2 * dp + h2;
                float4 *ch = comp_hi(s_comp, dd, tid, nthr), *cl = comp_lo(s_comp, dd, tid, nthr);
                const float4 hsum = *ch, lsum = *cl;
                float hj[4] = {hsum.x, hsum.y, hsum.z, hsum.w};
                float lj[4] = {lsum.x, lsum.y, lsum.z, lsum.w};
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    float p = h2 ? pb[j] : pa[j], h = hj[j];
                    float s = h + p;
                    float bp = s - h;
                    float e = (h - (s - bp)) + (p - bp);
                    hj[j] = s;
                    lj[j] += e;
                }
                *ch = make_float4(hj[0], hj[1], hj[2], hj[3]);
                *cl = make_float4(lj[0], lj[1], lj[2], lj[3]);
            }
        }
    };
    if (GATHER) {
        for (int cur = lo; cur < hi;) {
            const int nl = warp_gather(ws, ginfo, cur, hi, LC, warp, lane);
            if (nl == 0) break;
            warp_fill<NQ, DS>(g, ws, ginfo, 0, nl, d0 + warp * DS, lane, true);
            chunk(nl);
        }
    } else {
        const int nch = (hi - lo + LC - 1) / LC;
        for (int c = 0; c < nch; ++c) {
            const int nl = min(LC, hi - (lo + c * LC));
            warp_fill<NQ, DS>(g, ws, ginfo, lo + c * LC, nl, d0 + warp * DS, lane);
            chunk(nl);
        }
    }

    if (ext.y > 1) {
        // one of ext.y pieces of a split item (slots ext.x.., counter ext.z, piece ext.w):
        // store this piece's compensated sums; the piece that completes the item adds
        // all pieces' sums in piece order and finishes the cells below
        __shared__ int s_last;
        const size_t slot = (size_t)DS * nthr * 2;
        float4 *mine = g.fpart + (size_t)(ext.x + ext.w) * slot;
#pragma unroll
        for (int dd = 0; dd < DS; ++dd) {
            mine[((size_t)dd * nthr + tid) * 2] = *comp_hi(s_comp, dd, tid, nthr);
            mine[((size_t)dd * nthr + tid) * 2 + 1] = *comp_lo(s_comp, dd, tid, nthr);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = atomicAdd(g.fcnt + ext.z, 1) == ext.y - 1;
        __syncthreads();
        if (!s_last) return true;
        __threadfence();
#pragma unroll
        for (int dd = 0; dd < DS; ++dd) {
            float hj[4] = {0.f, 0.f, 0.f, 0.f}, lj[4] = {0.f, 0.f, 0.f, 0.f};
            for (int q = 0; q < ext.y; ++q) {
                const float4 *src = g.fpart + (size_t)(ext.x + q) * slot + ((size_t)dd * nthr + tid) * 2;
                const float4 h4 = __ldcg(src), l4 = __ldcg(src + 1);
                const float hq[4] = {h4.x, h4.y, h4.z, h4.w}, lq[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float h = hj[j], p = hq[j];
                    const float sum = h + p;
                    const float bp = sum - h;
                    const float e = (h - (sum - bp)) + (p - bp);
                    hj[j] = sum;
                    lj[j] += lq[j] + e;
                }
            }
            *comp_hi(s_comp, dd, tid, nthr) = make_float4(hj[0], hj[1], hj[2], hj[3]);
            *comp_lo(s_comp, dd, tid, nthr) = make_float4(lj[0], lj[1], lj[2], lj[3]);
        }
    }

    // epilogue: near-core sums, stimulated-emission factor at the sample frequency, vector store
#pragma unroll
    for (int dd = 0; dd < DS; ++dd) {
        int d = d0 + warp * DS + dd;
        if (d >= g.nd) continue;
        float c2T = __ldg(g.c2T + d);
        const float4 hsum = *comp_hi(s_comp, dd, tid, nthr), lsum = *comp_lo(s_comp, dd, tid, nthr);
        const float hj[4] = {hsum.x, hsum.y, hsum.z, hsum.w};
        const float lj[4] = {lsum.x, lsum.y, lsum.z, lsum.w};
        const float *nrow = g.knear + (int64_t)d * g.ld + lam_thr;
        float v[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            float lam = g.lam0cm * expf((float)(lam_thr + j) * g.lnr);
            float stim = -expm1f(-c2T / lam);
            float hi2 = hj[j], nj = nrow[j];
            float s = hi2 + nj;                    // 2Sum of the near-core sum into the total
            float bp = s - hi2;
            float e = (hi2 - (s - bp)) + (nj - bp);
            v[j] = stim * (s + (lj[j] + e));
        }
        float *row = g.kline + (int64_t)d * g.ld + lam_thr;
        if (J == 4)
            *reinterpret_cast<float4 *>(row) = make_float4(v[0], v[1 % J], v[2 % J], v[3 % J]);
        else
            *reinterpret_cast<float2 *>(row) = make_float2(v[0], v[1 % J]);
    }
    return true;
}

// Shared memory of the far-wing kernels: each warp's stage (warp_stage_quads), then
// (forward) the compensated sums of every thread [DS][threads][8] or (backward) the
// per-line sums of the warps, double-buffered by chunk [2][LC][GW], and each warp's
// per-lane partial sums of a batch of kBwdBatch lines [kBwdBatch][32] (lane l of line k at
// column l ^ k, so that both the row writes and the column reads avoid bank conflicts).
template <int J, int DS, int MINB, bool GATHER>
__global__ void __launch_bounds__(128, MINB) k_line_fwd(LineArgs g, int GW, int LC) {
    extern __shared__ float4 smem4[];
    const int warp = threadIdx.x >> 5;
    const size_t wq = warp_stage_quads(LC, DS, kNQF);
    float4 *mine = smem4 + (size_t)warp * wq;
    const WarpStage ws = make_stage(mine, LC, DS, kNQF);
    float *s_comp = reinterpret_cast<float *>(smem4 + (size_t)GW * wq);
    for_each_item(g, [&](const LineArgs &v, int tile, int group, int lo, int hi, int it) {
        return far_fwd_item<J, DS, GATHER>(v, tile, group, lo, hi, GW, LC, ws, s_comp,
                                           g.fext ? g.fext[it] : make_int4(-1, 1, -1, 0));
    });
}

// Reduced far-wing backward forms (lines flagged for them): H and dH/da polynomials cut
// after their t^2 terms (THREE: t^3).  par: the warp's depth pairs, (K, a^2) (B1 K, B2' K^2)
// (C1 K, C2' K^2); usq: the scaled squared offsets U = 2^36 u^2 of the thread's points.
template <int J, int DP, bool THREE>
__device__ __forceinline__ void far_bwd_line_reduced(const ulonglong2 *par, const float (&usq)[J],
                                                     const f2_t (&gv)[DP][J], bool full, int di0, int W, f2_t &S1,
                                                     f2_t &S2) {
    // reduced forms with s = 1/U: per depth pair X1 = sum_j G s_j and X2 = sum_j G s_j^2,
    // then S1 += (B1 K) X1 + (B2' K^2) X2 and S2 += (C1 K) X1 + (C2' K^2) X2 (THREE: also
    // X3 = sum_j G s_j^3 with B3' K^3 and C3' K^3); points outside the window
    // (di0 + j = i - i_l) get s = 0 unless it covers the tile
    f2_t sp[J], sq[J];
    if (full) {
#pragma unroll
        for (int j = 0; j < J; ++j) sp[j] = f2_splat(rcp_approx(usq[j]));
    } else {
#pragma unroll
        for (int j = 0; j < J; ++j)
            sp[j] = f2_splat(di0 + j >= -W && di0 + j <= W ? rcp_approx(usq[j]) : 0.0f);
    }
#pragma unroll
    for (int j = 0; j < J; ++j) sq[j] = f2_mul(sp[j], sp[j]);
    if (THREE) {
        f2_t sc[J];
#pragma unroll
        for (int j = 0; j < J; ++j) sc[j] = f2_mul(sq[j], sp[j]);
#pragma unroll
        for (int dp = 0; dp < DP; ++dp) {
            const ulonglong2 q0 = par[kNQB * dp], q1 = par[kNQB * dp + 1], q2 = par[kNQB * dp + 2];
            f2_t X1 = f2_mul(gv[dp][0], sp[0]), X2 = f2_mul(gv[dp][0], sq[0]), X3 = f2_mul(gv[dp][0], sc[0]);
#pragma unroll
            for (int j = 1; j < J; ++j) {
                X1 = f2_fma(gv[dp][j], sp[j], X1);
                X2 = f2_fma(gv[dp][j], sq[j], X2);
                X3 = f2_fma(gv[dp][j], sc[j], X3);
            }
            // B3' K^3 = (B1 K) K^2 (3.75 - 5a^2 + a^4), C3' K^3 = (C1 K) K^2 (3.75 - 15a^2 + 5a^4)
            const f2_t K2 = f2_mul(q0.x, q0.x);
            const f2_t b3 = f2_mul(f2_mul(q1.x, K2),
                                   f2_fma(q0.y, f2_fma(q0.y, f2_splat(1.0f), f2_splat(-5.0f)), f2_splat(3.75f)));
            const f2_t c3 = f2_mul(f2_mul(q2.x, K2),
                                   f2_fma(q0.y, f2_fma(q0.y, f2_splat(5.0f), f2_splat(-15.0f)), f2_splat(3.75f)));
            S1 = f2_fma(b3, X3, f2_fma(q1.y, X2, f2_fma(q1.x, X1, S1)));
            S2 = f2_fma(c3, X3, f2_fma(q2.y, X2, f2_fma(q2.x, X1, S2)));
        }
    } else {
#pragma unroll
        for (int dp = 0; dp < DP; ++dp) {
            const ulonglong2 q1 = par[kNQB * dp + 1], q2 = par[kNQB * dp + 2];
            f2_t X1 = f2_mul(gv[dp][0], sp[0]), X2 = f2_mul(gv[dp][0], sq[0]);
#pragma unroll
            for (int j = 1; j < J; ++j) {
                X1 = f2_fma(gv[dp][j], sp[j], X1);
                X2 = f2_fma(gv[dp][j], sq[j], X2);
            }
            S1 = f2_fma(q1.y, X2, f2_fma(q1.x, X1, S1));
            S2 = f2_fma(q2.y, X2, f2_fma(q2.x, X1, S2));
        }
    }
}

// Two-term reduced backward sums of one line from the reciprocals s_j of its points
// (far_reduced_s): per depth pair X1 = sum_j G s_j and X2 = sum_j G s_j^2, then
// S1 += (B1 K) X1 + (B2' K^2) X2 and S2 += (C1 K) X1 + (C2' K^2) X2.
template <int J, int DP>
__device__ __forceinline__ void far_bwd_two_term(const ulonglong2 *par, const f2_t (&sp)[J], const f2_t (&sq)[J],
                                                 const f2_t (&gv)[DP][J], f2_t &S1, f2_t &S2) {
#pragma unroll
    for (int dp = 0; dp < DP; ++dp) {
        const ulonglong2 q1 = par[kNQB * dp + 1], q2 = par[kNQB * dp + 2];
        f2_t X1 = f2_mul(gv[dp][0], sp[0]), X2 = f2_mul(gv[dp][0], sq[0]);
#pragma unroll
        for (int j = 1; j < J; ++j) {
            X1 = f2_fma(gv[dp][j], sp[j], X1);
            X2 = f2_fma(gv[dp][j], sq[j], X2);
        }
        S1 = f2_fma(q1.y, X2, f2_fma(q1.x, X1, S1));
        S2 = f2_fma(q2.y, X2, f2_fma(q2.x, X1, S2));
    }
}

// One line's far-wing backward sums over a warp's J x DS cells (depth pairs):
// S1 += G stim A H, S2 += G stim A a6 dH/da.  Without MASK, w holds the scaled squared
// offsets U = 2^36 u^2; with MASK, w holds the offsets u and kp the depth pairs' k, and
// only the far cells inside the window (inwin per lambda point) are kept.
template <int J, int DP, bool MASK>
__device__ __forceinline__ void far_bwd_line(const ulonglong2 *par, const f2_t (&w)[J], const f2_t (&gv)[DP][J],
                                             const bool *inwin, const f2_t *kp, f2_t &S1, f2_t &S2) {
#pragma unroll
    for (int dp = 0; dp < DP; ++dp) {
        // (K, a^2) (B1 K, B2' K^2) (C1 K, C2' K^2); the other coefficients from a^2, B1 K and C1 K
        const ulonglong2 q0 = par[kNQB * dp], q1 = par[kNQB * dp + 1], q2 = par[kNQB * dp + 2];
        f2_t B1 = q1.x, C1 = q2.x;
        if (MASK) {
            // the masked cells use t = 1/|z|^2 itself: B1 = (B1 K) k^2 2^-36, C1 alike
            const f2_t kk = f2_mul(f2_mul(kp[dp], kp[dp]), f2_splat(kKUnscale));
            B1 = f2_mul(B1, kk);
            C1 = f2_mul(C1, kk);
        }
        f2_t B3, B4, B5, C3, C4, C5, C6;
        far_b345(q0.y, B1, B3, B4, B5);
        far_c3456(q0.y, C1, C3, C4, C5, C6);
        const f2_t B2 = f2_mul(B1, f2_splat(1.5f));
        const f2_t C2 = f2_mul(f2_fma(q0.y, f2_splat(-2.0f), f2_splat(1.5f)), C1);
        const f2_t ak = f2_mul(q0.y, q0.x);          // a^2 K
#pragma unroll
        for (int j = 0; j < J; ++j) {
            f2_t r2, t, m;
            if (MASK) {
                const f2_t x = f2_mul(w[j], kp[dp]);
                r2 = f2_fma(x, x, q0.y);
                t = f2_rcp(r2);
                m = t;
            } else {
                // r = 1/(U + a^2 K), t = K r; the coefficients carry K, so the sums take r
                m = f2_rcp(f2_fma(w[j], f2_splat(1.0f), ak));
                t = f2_mul(q0.x, m);
            }
            f2_t h = f2_fma(t, B5, B4);
            h = f2_fma(t, h, B3);
            h = f2_fma(t, h, B2);
            h = f2_fma(t, h, B1);
            f2_t q = f2_fma(t, C6, C5);
            q = f2_fma(t, q, C4);
            q = f2_fma(t, q, C3);
            q = f2_fma(t, q, C2);
            q = f2_fma(t, q, C1);
            f2_t gt = f2_mul(gv[dp][j], m);
            if (MASK) {
                float r2a, r2b, ga, gb;
                f2_unpack(r2, r2a, r2b);
                f2_unpack(gt, ga, gb);
                ga = (inwin[j] && r2a >= kFar2) ? ga : 0.0f;
                gb = (inwin[j] && r2b >= kFar2) ? gb : 0.0f;
                gt = f2_pack(ga, gb);
            }
            S1 = f2_fma(gt, h, S1);
            S2 = f2_fma(gt, q, S2);
        }
    }
}

// Far-wing kernel (backward): the per-line sums over the tile's far cells of
// G stim A H and G stim A a6 dH/da, reduced over the CTA and added to gacc.
template <int J, int DS>
__device__ __forceinline__ bool far_bwd_item(const LineArgs &g, const int tile, const int group, const int lo,
                                             const int hi, const int GW, const int LC, const WarpStage &ws,
                                             float2 *s_part, float2 *s_red2, unsigned &cc) {
    static_assert(J == 2 || J == 4, "J must be 2 or 4");
    static_assert(DS % 2 == 0, "DS must be even (depth pairs)");
    constexpr int DP = DS / 2;
    constexpr int NQ = kNQB;
    const int T = 32 * J;
    const int DC = GW * DS;
    const int nthr = blockDim.x;
    const LineInfo *ginfo = g.finfo + (int64_t)group * g.nl;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int d0 = group * DC;
    const int slab = group * GW + warp;
    const int t0 = tile * T;
    const float t0f = (float)t0, tendf = (float)(t0 + T - 1);
    const int lam_thr = t0 + lane * J;
    const float lamf = (float)lam_thr;

    // G * stim of the thread's cells as depth pairs; zero outside the grid
    f2_t gv[DP][J];
#pragma unroll
    for (int dp = 0; dp < DP; ++dp) {
        const int da = d0 + warp * DS + 2 * dp, db = da + 1;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const bool inl = lam_thr + j < g.nlam;
            const float ga = (da < g.nd && inl) ? g.Gt[(int64_t)da * g.ld + lam_thr + j] : 0.0f;
            const float gb = (db < g.nd && inl) ? g.Gt[(int64_t)db * g.ld + lam_thr + j] : 0.0f;
            gv[dp][j] = f2_pack(ga, gb);
        }
    }

    warp_stage_depths<DS>(g, ws, d0 + warp * DS, lane);
    const int nch = (hi - lo + LC - 1) / LC;
    for (int c = 0; c < nch; ++c) {
        const int c0 = lo + c * LC;
        const int nl = min(LC, hi - c0);
        // per-line sums of this chunk go to buffer cc & 1: its previous readers (the
        // reduction two chunks back) are past the CTA barrier of the previous chunk
        float2 *s_red = s_red2 + (size_t)((cc + c) & 1) * LC * GW;
        warp_fill<NQ, DS>(g, ws, ginfo, c0, nl, d0 + warp * DS, lane);
        const ulonglong2 *s_par = reinterpret_cast<const ulonglong2 *>(ws.par);
        const LineInfo *s_line = ws.info;
        unsigned m_fast = 0u, m_red = 0u, m_red3 = 0u, m_skip = 0u;   // this warp's flags of 32 lines, one per lane
        for (int li = 0; li < nl;) {
            const unsigned b = li & 31;
            if (b == 0) {
                const int lj = li + lane;
                const int f = lj < nl ? far_flags(g, s_line[lj], t0f, tendf, slab, warp) : 0;
                m_fast = __ballot_sync(0xffffffffu, f & 1);
                m_red = __ballot_sync(0xffffffffu, (f & 2) != 0);
                m_red3 = __ballot_sync(0xffffffffu, (f & 8) != 0);
                m_skip = __ballot_sync(0xffffffffu, (f & 4) != 0);
            }
            if ((b & (kBwdBatch - 1)) != kBwdBatch - 1 && li + 1 < nl && ((m_red >> b) & 3u) == 3u &&
                ((m_skip >> b) & 3u) == 0u) {
                // two consecutive two-term lines of one batch: independent offset and
                // reciprocal chains, formed together
                f2_t spa[J], sqa[J], spb[J], sqb[J];
                far_reduced_s<J>(g, s_line[li], (m_fast >> b) & 1u, lamf, lam_thr, spa, sqa);
                far_reduced_s<J>(g, s_line[li + 1], (m_fast >> (b + 1)) & 1u, lamf, lam_thr, spb, sqb);
                const ulonglong2 *pa = s_par + (size_t)li * DP * NQ;
                f2_t S1a = 0ull, S2a = 0ull, S1b = 0ull, S2b = 0ull;
                far_bwd_two_term<J, DP>(pa, spa, sqa, gv, S1a, S2a);
                far_bwd_two_term<J, DP>(pa + DP * NQ, spb, sqb, gv, S1b, S2b);
                const int r = b & (kBwdBatch - 1);
                s_part[r * 32 + (lane ^ r)] = make_float2(f2_lo(S1a) + f2_hi(S1a), f2_lo(S2a) + f2_hi(S2a));
                s_part[(r + 1) * 32 + (lane ^ (r + 1))] = make_float2(f2_lo(S1b) + f2_hi(S1b), f2_lo(S2b) + f2_hi(S2b));
                li += 2;
            } else {
                const LineInfo info = s_line[li];
                const int fl = (int)((m_fast >> b) & 1u) | (int)(((m_red >> b) & 1u) << 1) | (int)(((m_red3 >> b) & 1u) << 2);
                const ulonglong2 *par = s_par + (size_t)li * DP * NQ;
                f2_t S1 = 0ull, S2 = 0ull;
                // (a slab whose every layer the centre test rejects keeps zero sums)
                if (!((m_skip >> b) & 1u)) {
                    float U[J];
                    if (fl != 0) far_scaled_u2<J>(g, info, lamf, U);
                    if (fl & 2) {
                        far_bwd_line_reduced<J, DP, false>(par, U, gv, (fl & 1) != 0, lam_thr - (int)info.ilf, g.W,
                                                           S1, S2);
                    } else if (fl & 4) {
                        far_bwd_line_reduced<J, DP, true>(par, U, gv, (fl & 1) != 0, lam_thr - (int)info.ilf, g.W,
                                                          S1, S2);
                    } else if (fl & 1) {
                        f2_t u2[J];
#pragma unroll
                        for (int j = 0; j < J; ++j) u2[j] = f2_splat(U[j]);
                        far_bwd_line<J, DP, false>(par, u2, gv, nullptr, nullptr, S1, S2);
                    } else {
                        // line near the tile or partly outside its window: far cells inside the window only
                        f2_t u2[J];
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            u2[j] = f2_splat(offset_u((info.ilf - (lamf + (float)j)) + info.frac, g.lnr));
                        bool inwin[J];
                        const int il = (int)info.ilf;
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            const int di = lam_thr + j - il;
                            inwin[j] = di >= -g.W && di <= g.W;
                        }
                        f2_t kp[DP];
                        far_kpairs<DP>(g, info.sp, d0 + warp * DS, kp);
                        far_bwd_line<J, DP, true>(par, u2, gv, inwin, kp, S1, S2);
                    }
                }
                const int r = b & (kBwdBatch - 1);
                s_part[r * 32 + (lane ^ r)] = make_float2(f2_lo(S1) + f2_hi(S1), f2_lo(S2) + f2_hi(S2));
                ++li;
            }
            if ((li & (kBwdBatch - 1)) == 0 || li >= nl) {
                // end of a batch of kBwdBatch lines: lanes 2r and 2r + 1 add the two halves of
                // line r's partial sums over the warp's lanes (row r holds lane j's at column
                // j ^ r), combine them and leave the warp's total for the CTA reduction
                __syncwarp();
                const int base = (li - 1) & ~(kBwdBatch - 1);
                const int r = lane >> 1, h = lane & 1;
                float a1 = 0.0f, a2 = 0.0f;
                if (base + r < nl) {
                    const float2 *row = s_part + r * 32;
#pragma unroll 8
                    for (int t = 0; t < 16; ++t) {
                        const float2 v = row[(16 * h + t) ^ r];
                        a1 += v.x;
                        a2 += v.y;
                    }
                }
                a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
                a2 += __shfl_xor_sync(0xffffffffu, a2, 1);
                if (h == 0 && base + r < nl) s_red[(base + r) * GW + warp] = make_float2(a1, a2);
                __syncwarp();
            }
        }
        __syncthreads();
        // thread k adds sum k & 1 of line k >> 1 over the warps in FP32, in warp order, and
        // converts once for the FP64 accumulator: FP64 arithmetic runs at a small fraction
        // of the FP32 rate, and a chain of FP64 adds here would hold the CTA at the next barrier
        for (int k = tid; k < 2 * nl; k += nthr) {
            const int li = k >> 1;
            const float *r = reinterpret_cast<const float *>(s_red + li * GW) + (k & 1);
            float a = r[0];
            for (int w = 1; w < GW; ++w) a += r[2 * w];
            atomicAdd(g.gacc + (int64_t)(k & 1) * g.nl + c0 + li, (double)a);
        }
    }
    cc += nch;
    return true;
}

template <int J, int DS, int MINB>
__global__ void __launch_bounds__(128, MINB) k_line_bwd(LineArgs g, int GW, int LC) {
    extern __shared__ float4 smem4[];
    const int warp = threadIdx.x >> 5;
    const size_t wq = warp_stage_quads(LC, DS, kNQB);
    float4 *mine = smem4 + (size_t)warp * wq;
    const WarpStage ws = make_stage(mine, LC, DS, kNQB);
    float2 *s_red2 = reinterpret_cast<float2 *>(smem4 + (size_t)GW * wq);
    float2 *s_part = s_red2 + (size_t)2 * LC * GW + (size_t)warp * kBwdBatch * 32;
    unsigned cc = 0;
    for_each_item(g, [&](const LineArgs &v, int tile, int group, int lo, int hi, int) {
        return far_bwd_item<J, DS>(v, tile, group, lo, hi, GW, LC, ws, s_part, s_red2, cc);
    });
}

// ---------------------------------------------------------------------------
// Near-core kernels: the cells with |v|^2 + a^2 < 400 (mid wing and core).  A CTA owns
// the same wavelength tile as the far kernels and every depth; its warps take
// (line, depth) items of the lines whose near zone can reach the tile, clip the
// item's near span analytically, and let the lanes sweep the span 32 points at a
// time.  Each cell is classified with the far kernels' own arithmetic (same
// prefactors, same offset and the same |v|^2 + a^2 test), so every cell is counted
// exactly once across the two kernels.
// ---------------------------------------------------------------------------

// Near span of an item clipped to the tile and the window; returns false if empty.
__device__ __forceinline__ bool near_span(const LineArgs &g, float ilf, float frac, float k, float a2, int t0, int T,
                                          int &lo, int &hi) {
    const float r2 = kFar2 - a2;
    if (!(k > 0.0f) || !(r2 > 0.0f)) return false;
    const float xl = ilf + frac;
    const int il = (int)ilf;
    const float span = sqrtf(r2) / (k * g.lnr) * 1.01f + 1.0f;
    lo = max(max(t0, (int)floorf(xl - span)), il - g.W);
    hi = min(min(t0 + T - 1, (int)ceilf(xl + span)), il + g.W);
    return lo <= hi;
}

// One near-core item (a line at one depth) after its lane-parallel set-up.  Its near
// span [lo, hi] (clipped to the tile and the window) is split analytically into the
// core segment (|z|^2 < 36, cells [c0, r0)) and the mid-wing cells on either side
// (nl cells from lo, then the cells from r0 to hi).
struct alignas(16) NearItem {
    float ilf, frac, k, a2;      // centre, Doppler factor c/dv_D, a^2
    float a, A, Aa6;             // damping, strength, strength x vdW damping
    int lo, nl, c0, r0;          // span start, mid cells left of the core, core segment [c0, r0)
    int dlb;                     // local depth | (local line index << 8)
};

constexpr int kNearBatch = 512;      // lines per shared-memory batch of the backward sums
constexpr int kNearWarps = 8;        // warps per near-core CTA

// Dense pass over the concatenated cells of one segment kind of the warp's 32 items:
// cell n of the concatenation belongs to item src with pref[src] <= n < pref[src + 1]
// (each lane advances its own cursor; consecutive lanes hold consecutive cells, so
// the items of one iteration form ordered runs).
//   forward:  cell(item, i, H, dH) adds the cell's term where it belongs;
//   backward: val(item, i, H, dH) returns the cell's (G A H, G A a6 dH) pair and
//             done(item, sum) receives the per-run sums of each item.
template <int T, bool D, bool CORE, class Cell, class Val, class Done>
__device__ __forceinline__ void near_pass(const LineArgs &g, const NearItem *mine, const int *pref, const float *s_daw,
                                          Cell &cell, Val &val, Done &done) {
    const int lane = threadIdx.x & 31;
    const int total = pref[32];
    int src = 0;
    for (int n0 = 0; n0 < total; n0 += 32) {
        const int n = n0 + lane;
        int run = -1;
        float2 v = make_float2(0.0f, 0.0f);
        if (n < total) {
            while (pref[src + 1] <= n) ++src;
            const NearItem &it = mine[src];
            const int off = n - pref[src];
            const int i = CORE ? it.c0 + off : (off < it.nl ? it.lo + off : it.r0 + (off - it.nl));
            const float x = fabsf(offset_u((it.ilf - (float)i) + it.frac, g.lnr) * it.k);
            run = src;
            // a mid-wing cell at |z| >= 20 belongs to the far-wing kernels (same test)
            if (CORE || fmaf(x, x, it.a2) < kFar2) {
                float H, dH;
                if (CORE)
                    voigt_core<D>(x, it.a, H, dH, s_daw);
                else
                    voigt_mid<D>(x, it.a, H, dH);
                if (D)
                    v = val(it, i, H, dH);
                else
                    cell(it, i, H, dH);
            }
        }
        if (D) {
            // segmented sum over the runs of equal items
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float nx = __shfl_up_sync(0xffffffffu, v.x, o);
                const float ny = __shfl_up_sync(0xffffffffu, v.y, o);
                const int ns = __shfl_up_sync(0xffffffffu, run, o);
                if (lane >= o && ns == run) {
                    v.x += nx;
                    v.y += ny;
                }
            }
            const int next = __shfl_down_sync(0xffffffffu, run, 1);
            if (run >= 0 && (lane == 31 || next != run)) done(mine[run], v);
        }
    }
}

// Backward pass with a blocked assignment (mid wing or core): lane l takes the
// concatenated cells [l P, (l + 1) P), P = ceil(total / 32), so that each lane's cells
// belong to a few consecutive items; the lane sums an item's cells in registers and
// hands the sum to done when it moves to the next item (no cross-lane reduction).
// voigt_mid has no branch on the item's parameters; the core form branches on the
// damping (Taylor order, table or rational), where lanes of different items diverge.
template <bool CORE, class Val, class Done>
__device__ __forceinline__ void near_pass_blocked(const LineArgs &g, const NearItem *mine, const int *pref,
                                                  const float *s_daw, Val &val, Done &done) {
    const int lane = threadIdx.x & 31;
    const int total = pref[32];
    const int per = (total + 31) >> 5;
    const int nb = min(lane * per, total), ne = min(nb + per, total);
    if (nb >= ne) return;
    int src = 0;
    while (pref[src + 1] <= nb) ++src;
    NearItem it = mine[src];
    int start = pref[src], end = pref[src + 1];
    float2 acc = make_float2(0.0f, 0.0f);
    for (int n = nb; n < ne; ++n) {
        if (n >= end) {
            done(it, acc);
            acc = make_float2(0.0f, 0.0f);
            do {
                ++src;
            } while (pref[src + 1] <= n);
            it = mine[src];
            start = pref[src];
            end = pref[src + 1];
        }
        const int off = n - start;
        const int i = CORE ? it.c0 + off : (off < it.nl ? it.lo + off : it.r0 + (off - it.nl));
        const float x = fabsf(offset_u((it.ilf - (float)i) + it.frac, g.lnr) * it.k);
        // a mid-wing cell at |z| >= 20 belongs to the far-wing kernels (same test)
        if (CORE || fmaf(x, x, it.a2) < kFar2) {
            float H, dH;
            if (CORE)
                voigt_core<true>(x, it.a, H, dH, s_daw);
            else
                voigt_mid<true>(x, it.a, H, dH);
            const float2 v = val(it, i, H, dH);
            acc.x += v.x;
            acc.y += v.y;
        }
    }
    done(it, acc);
}

// Near-core sweep shared by the forward (D = false) and the backward (D = true).
// Each warp takes rounds of 32 (line, depth) items: every lane sets up one item
// (coarse span from c/dv_D alone, then the exact prefactors, the clipped span and
// its core / mid split), a warp scan turns the per-item cell counts into offsets,
// and the warp then sweeps all mid-wing cells of the round and all core cells of
// the round, 32 consecutive cells at a time, so the two Voigt forms never diverge
// within a warp and no lane idles while cells remain.
template <int T, bool D, class Cell, class Val, class Done>
__device__ __forceinline__ void near_sweep(const LineArgs &g, int t0, int64_t nlo, int64_t nitems, int ndg, int dbase,
                                           NearItem *s_items, int *s_pref, const float *s_daw, Cell &&cell,
                                           Val &&val, Done &&done) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    NearItem *mine = s_items + warp * 32;
    int *pm = s_pref + warp * 66, *pc = pm + 33;      // prefix counts of mid and core cells
    for (int64_t r0 = (int64_t)warp * 32; r0 < nitems; r0 += (int64_t)nwarp * 32) {
        const int64_t it = r0 + lane;
        int nmid = 0, ncore = 0;
        NearItem item;
        if (it < nitems) {
            const int64_t l = nlo + it / ndg;
            const int dl = (int)(it % ndg), d = dbase + dl;
            item.ilf = g.ilf[l];
            item.frac = g.frac[l];
            item.dlb = dl | ((int)(it / ndg) << 8);
            const float k = (float)kC * __ldg(g.invdv + g.sp[l] * g.nd + d);
            int lo, hi;
            if (pair_kept(g.keep, l, d) && near_span(g, item.ilf, item.frac, k, 0.0f, t0, T, lo, hi)) {
                float p[16];
                line_params<D ? 16 : 8>(g, l, d, p);
                if (near_span(g, item.ilf, item.frac, p[0], p[1], t0, T, lo, hi)) {
                    item.k = p[0];
                    item.a2 = p[1];
                    item.A = p[7];
                    item.a = D ? p[15] : sqrtf(p[1]);
                    item.Aa6 = D ? p[14] : 0.0f;
                    // core segment: |x| < sqrt(36 - a^2), x = u k, |u| ~ |x_l - i| ln r
                    int c0 = hi + 1, c1 = hi;
                    if (p[1] < kMid2) {
                        const float w = sqrtf(kMid2 - p[1]) / (p[0] * g.lnr);
                        const float xl = item.ilf + item.frac;
                        c0 = max(lo, (int)ceilf(xl - w));
                        c1 = min(hi, (int)floorf(xl + w));
                        if (c0 > c1) {
                            c0 = hi + 1;
                            c1 = hi;
                        }
                    }
                    ncore = c1 - c0 + 1;
                    nmid = (hi - lo + 1) - ncore;
                    item.lo = lo;
                    item.nl = ncore > 0 ? c0 - lo : nmid;
                    item.c0 = c0;
                    item.r0 = ncore > 0 ? c1 + 1 : hi + 1;
                }
            }
        }
        // exclusive prefix of the packed counts (mid << 16 | core; a round holds < 2^16 cells)
        const int own = (nmid << 16) | ncore;
        int inc = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        __syncwarp();
        const int exc = inc - own;
        pm[lane] = exc >> 16;
        pc[lane] = exc & 0xffff;
        if (lane == 31) {
            pm[32] = inc >> 16;
            pc[32] = inc & 0xffff;
        }
        if (own != 0) mine[lane] = item;
        __syncwarp();
        if (D) {
            // mid wing blocked; the core keeps interleaved cells (its damping branches would
            // diverge across the items of a blocked warp: measured 238 -> 339 ms per batch step)
            near_pass_blocked<false>(g, mine, pm, s_daw, val, done);
            __syncwarp();
            near_pass<T, D, true>(g, mine, pc, s_daw, cell, val, done);
        } else {
            near_pass<T, D, false>(g, mine, pm, s_daw, cell, val, done);
            __syncwarp();
            near_pass<T, D, true>(g, mine, pc, s_daw, cell, val, done);
        }
    }
}

// Forward near-core sums into knear.  Work items: (star, tile, depth group of NDG layers).
template <int T, int NDG>
__global__ void __launch_bounds__(32 * kNearWarps) k_line_near_fwd(LineArgs gq) {
    extern __shared__ float4 smem4[];
    float *s_acc = reinterpret_cast<float *>(smem4);                               // [NDG][T]
    NearItem *s_items = reinterpret_cast<NearItem *>(s_acc + NDG * T);             // [warps][32]
    int *s_pref = reinterpret_cast<int *>(s_items + kNearWarps * 32);              // [warps][2][33]
    float *s_daw = reinterpret_cast<float *>(s_pref + kNearWarps * 66);            // Dawson table
    for (int k = threadIdx.x; k < kDawsonNodes * (kDawsonK + 1); k += blockDim.x) s_daw[k] = g_dawson[k];
    for_each_item(gq, [&](const LineArgs &g, int tile, int group, int nlo, int nhi, int) {
    const int tid = threadIdx.x;
    const int t0 = tile * T;
    const int dbase = group * NDG, ndg = min(NDG, g.nd - dbase);
    for (int k = tid; k < NDG * T; k += blockDim.x) s_acc[k] = 0.0f;
    __syncthreads();
    near_sweep<T, false>(
        g, t0, nlo, (int64_t)(nhi - nlo) * ndg, ndg, dbase, s_items, s_pref, s_daw,
        [&](const NearItem &it, int i, float H, float) {
            atomicAdd(s_acc + (it.dlb & 0xff) * T + (i - t0), it.A * H);
        },
        [&](const NearItem &, int, float, float) { return make_float2(0.0f, 0.0f); },
        [&](const NearItem &, float2) {});
    __syncthreads();
    for (int k = tid; k < ndg * T; k += blockDim.x) {
        const int dl = k / T, q = k - dl * T;
        g.knear[(int64_t)(dbase + dl) * g.ld + t0 + q] = s_acc[k];
    }
    });
}

// Backward: per-line sums over the near cells of G stim A H and G stim A a6 dH/da.
// Lines are processed in batches whose per-line sums live in shared memory; one
// global atomic per (line, tile, depth group) at the end of each batch.
template <int T, int NDG>
__global__ void __launch_bounds__(32 * kNearWarps, 5) k_line_near_bwd(LineArgs gq) {
    extern __shared__ float4 smem4[];
    float *s_g = reinterpret_cast<float *>(smem4);                                 // [NDG][T] G * stim
    float2 *s_sum = reinterpret_cast<float2 *>(s_g + NDG * T);                     // [kNearBatch]
    NearItem *s_items = reinterpret_cast<NearItem *>(s_sum + kNearBatch);          // [warps][32]
    int *s_pref = reinterpret_cast<int *>(s_items + kNearWarps * 32);              // [warps][2][33]
    float *s_daw = reinterpret_cast<float *>(s_pref + kNearWarps * 66);            // Dawson table
    for (int k = threadIdx.x; k < kDawsonNodes * (kDawsonK + 1); k += blockDim.x) s_daw[k] = g_dawson[k];
    for_each_item(gq, [&](const LineArgs &g, int tile, int group, int nlo, int nhi, int) {
    const int tid = threadIdx.x;
    const int t0 = tile * T;
    const int dbase = group * NDG, ndg = min(NDG, g.nd - dbase);
    for (int k = tid; k < ndg * T; k += blockDim.x) {
        const int dl = k / T, q = k - dl * T;
        s_g[k] = (t0 + q < g.nlam) ? g.Gt[(int64_t)(dbase + dl) * g.ld + t0 + q] : 0.0f;
    }
    for (int b0 = nlo; b0 < nhi; b0 += kNearBatch) {
        const int nb = min(kNearBatch, nhi - b0);
        __syncthreads();
        for (int k = tid; k < nb; k += blockDim.x) s_sum[k] = make_float2(0.0f, 0.0f);
        __syncthreads();
        near_sweep<T, true>(
            g, t0, b0, (int64_t)nb * ndg, ndg, dbase, s_items, s_pref, s_daw,
            [&](const NearItem &, int, float, float) {},
            [&](const NearItem &it, int i, float H, float dH) {
                const float gs = s_g[(it.dlb & 0xff) * T + (i - t0)];
                return make_float2(gs * it.A * H, gs * it.Aa6 * dH);
            },
            [&](const NearItem &it, float2 v) {
                const int lb = it.dlb >> 8;
                atomicAdd(&s_sum[lb].x, v.x);
                atomicAdd(&s_sum[lb].y, v.y);
            });
        __syncthreads();
        for (int k = tid; k < nb; k += blockDim.x) {
            const float2 v = s_sum[k];
            if (v.x != 0.0f) atomicAdd(g.gacc + b0 + k, (double)v.x);
            if (v.y != 0.0f) atomicAdd(g.gacc + g.nl + b0 + k, (double)v.y);
        }
    }
    __syncthreads();
    });
}

template <int T, int NDG, bool BWD>
constexpr size_t near_smem() {
    return (size_t)NDG * T * sizeof(float) + (BWD ? kNearBatch * sizeof(float2) : 0) +
           (size_t)kNearWarps * 32 * sizeof(NearItem) + (size_t)kNearWarps * 66 * sizeof(int) +
           (size_t)kDawsonNodes * (kDawsonK + 1) * sizeof(float);
}

static LineArgs make_args(pz_ctx *c) {
    LineArgs g;
    g.nlam = c->nlam;
    g.ld = c->ld;
    g.nd = c->nd;
    g.W = c->W;
    g.lnr = (float)c->lnr;
    for (int j = 0; j < 4; ++j) {
        g.rj[j] = (float)std::exp(-j * c->lnr);
        g.rm1j[j] = (float)std::expm1(-j * c->lnr);
    }
    g.star = c->L.star;
    g.fext = nullptr;
    g.fpart = c->d_fpart;
    g.fcnt = c->d_fcnt;
    g.finfo = reinterpret_cast<const LineInfo *>(c->d_finfo);
    g.status = c->d_status;
    g.keep = c->d_keep;
    g.dsel = c->bwd_dsel;
    g.lam0cm = (float)(c->lambda0_nm * 1e-7);
    g.ilf = c->L.ilf;
    g.frac = c->L.frac;
    g.E = c->L.E;
    g.lamcm = c->L.lamcm;
    g.grad = c->L.grad;
    g.g4 = c->L.g4;
    g.g6 = c->L.g6;
    g.Q = c->L.Q;
    g.sp = c->L.sp;
    g.R = c->d_R;
    g.invdv = c->d_invdv;
    g.Ksd = c->d_Ksd;
    g.thr = c->d_thr;
    g.nslab = c->nslab;
    g.beta_hi = c->d_beta_hi;
    g.beta_lo = c->d_beta_lo;
    g.ne = c->d_ne;
    g.npert = c->d_npert;
    g.c2T = c->d_c2T;
    g.kline = (float *)c->d_kline;
    g.knear = c->d_knear;
    g.Gt = c->d_Gt;
    g.gacc = c->d_gacc + c->gacc_off;
    g.nl = c->L.n;
    g.items = nullptr;
    g.n_items = 0;
    g.ngroups = 1;
    g.ctr = nullptr;
    g.sstride = (int64_t)c->ns * c->nd;
    g.dstride = c->nd;
    g.bstride = (int64_t)c->nd * c->ld;
    g.tstride = (int64_t)c->ns * c->nslab;
    return g;
}

// Persistent grid: as many CTAs as fit on the GPU at once, at most one per item.
template <class K>
static int persistent_grid(pz_ctx *c, K kernel, int threads, size_t smem, int n_items) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    int64_t n = (int64_t)per_sm * std::max(c->n_sm, 1);
    return (int)std::max<int64_t>(1, std::min<int64_t>(n, n_items));
}

template <int T, bool BWD>
static cudaError_t launch_near(pz_ctx *c, LineArgs g, cudaStream_t s) {
    if (BWD) {
        if (c->n_nitems_b == 0) return cudaSuccess;
        g.items = c->d_nitems_b;
        g.n_items = c->n_nitems_b;
        g.ngroups = (c->nd + kNearDepthsBwd - 1) / kNearDepthsBwd;
        g.ctr = c->d_ctr + 3;
        constexpr size_t smem = near_smem<T, kNearDepthsBwd, true>();
        static std::atomic<bool> attr_set[kMaxDevices];
        if (!attr_set[c->device].load(std::memory_order_acquire)) {
            cudaFuncSetAttribute(k_line_near_bwd<T, kNearDepthsBwd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            attr_set[c->device].store(true, std::memory_order_release);
        }
        int grid = persistent_grid(c, k_line_near_bwd<T, kNearDepthsBwd>, 32 * kNearWarps, smem, g.n_items);
        cudaEvent_t ev = prof_begin(c, s);
        k_line_near_bwd<T, kNearDepthsBwd><<<grid, 32 * kNearWarps, smem, s>>>(g);
        prof_end(c, s, PZ_K_NEAR_BWD, ev);
    } else {
        if (c->n_nitems_f == 0) return cudaSuccess;
        g.items = c->d_nitems_f;
        g.n_items = c->n_nitems_f;
        g.ngroups = (c->nd + kNearDepthsFwd - 1) / kNearDepthsFwd;
        g.ctr = c->d_ctr + 0;
        constexpr size_t smem = near_smem<T, kNearDepthsFwd, false>();
        static std::atomic<bool> attr_set[kMaxDevices];
        if (!attr_set[c->device].load(std::memory_order_acquire)) {
            cudaFuncSetAttribute(k_line_near_fwd<T, kNearDepthsFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            attr_set[c->device].store(true, std::memory_order_release);
        }
        int grid = persistent_grid(c, k_line_near_fwd<T, kNearDepthsFwd>, 32 * kNearWarps, smem, g.n_items);
        cudaEvent_t ev = prof_begin(c, s);
        k_line_near_fwd<T, kNearDepthsFwd><<<grid, 32 * kNearWarps, smem, s>>>(g);
        prof_end(c, s, PZ_K_NEAR_FWD, ev);
    }
    c->launches++;
    return cudaGetLastError();
}

// Dynamic shared memory of the far-wing kernels: the warps' stages (layer constants,
// line records, prefactors) and (forward) the compensated sums of every thread, or
// (backward) the per-line sums.
static size_t far_fwd_smem(const Tiling &t) {
    return (size_t)t.GW * warp_stage_quads(t.LC, t.DS, kNQF) * sizeof(float4) +
           (size_t)t.DS * 32 * t.GW * 2 * sizeof(float4);
}
static size_t far_bwd_smem(const Tiling &t) {
    return (size_t)t.GW * warp_stage_quads(t.LCB, t.DS, kNQB) * sizeof(float4) +
           (size_t)2 * t.LCB * t.GW * sizeof(float2) + (size_t)t.GW * kBwdBatch * 32 * sizeof(float2);
}
constexpr size_t kFarSmemMax = 200 * 1024;   // the opt-in size the far-wing kernels are given

bool tiling_fits(const Tiling &t) { return far_fwd_smem(t) <= kFarSmemMax && far_bwd_smem(t) <= kFarSmemMax; }

// Line records of the far-wing kernels for the current tiling, into the context's
// buffer (sized by ensure_far_tables).
static cudaError_t launch_far_info(pz_ctx *c, LineArgs &g, int DS, cudaStream_t s) {
    const int DC = c->tiling.depth_per_cta();
    const int64_t n = (int64_t)g.ngroups * c->L.n;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->n_sm * 16);
    g.finfo = reinterpret_cast<const LineInfo *>(c->d_finfo);
    k_far_info<<<grid, 256, 0, s>>>(g, DC, DS, g.ngroups, reinterpret_cast<LineInfo *>(c->d_finfo));
    c->launches++;
    return cudaGetLastError();
}

size_t far_info_bytes(const pz_ctx *c) {
    const int DC = c->tiling.depth_per_cta();
    const int ng = (c->nd + DC - 1) / DC;
    return (size_t)ng * std::max<int64_t>(c->L.n, 1) * sizeof(LineInfo);
}

template <int J, int DS, int MINB>
static cudaError_t launch_fwd_t(pz_ctx *c, cudaStream_t s) {
    const Tiling &t = c->tiling;
    LineArgs g = make_args(c);
    const size_t smem = far_fwd_smem(t);
    // with a centre test the kernel stages only the lines each warp's slab sweeps (GATHER)
    const bool gather = c->d_keep != nullptr;
    auto kern = gather ? k_line_fwd<J, DS, MINB, true> : k_line_fwd<J, DS, MINB, false>;
    static std::atomic<bool> attr_set[kMaxDevices][2];
    if (!attr_set[c->device][gather].load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFarSmemMax);
        attr_set[c->device][gather].store(true, std::memory_order_release);
    }
    cudaError_t e = cudaMemsetAsync(c->d_ctr, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = launch_near<32 * J, false>(c, g, s);
    if (e != cudaSuccess || c->n_fitems == 0) return e;
    g.items = c->d_fitems;
    g.fext = c->d_fext;
    g.n_items = c->n_fitems;
    g.ngroups = (c->nd + t.depth_per_cta() - 1) / t.depth_per_cta();
    g.ctr = c->d_ctr + 1;
    if (c->L.n > 0) {
        e = launch_far_info(c, g, DS, s);
        if (e != cudaSuccess) return e;
    }
    if (c->n_fsplit > 0) {
        e = cudaMemsetAsync(c->d_fcnt, 0, sizeof(int) * c->n_fsplit, s);
        if (e != cudaSuccess) return e;
    }
    int grid = persistent_grid(c, kern, 32 * t.GW, smem, g.n_items);
    kern<<<grid, 32 * t.GW, smem, s>>>(g, t.GW, t.LC);
    c->launches++;
    return cudaGetLastError();
}

template <int J, int DS, int MINB>
static cudaError_t launch_bwd_t(pz_ctx *c, cudaStream_t s) {
    const Tiling &t = c->tiling;
    LineArgs g = make_args(c);
    const size_t smem = far_bwd_smem(t);
    static std::atomic<bool> attr_set[kMaxDevices];
    if (!attr_set[c->device].load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(k_line_bwd<J, DS, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFarSmemMax);
        attr_set[c->device].store(true, std::memory_order_release);
    }
    cudaError_t e = cudaMemsetAsync(c->d_ctr + 2, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (c->n_bitems > 0) {
        LineArgs gb = g;
        gb.items = c->d_bitems;
        gb.n_items = c->n_bitems;
        gb.ngroups = (c->nd + t.depth_per_cta() - 1) / t.depth_per_cta();
        gb.ctr = c->d_ctr + 2;
        e = launch_far_info(c, gb, DS, s);
        if (e != cudaSuccess) return e;
        int grid = persistent_grid(c, k_line_bwd<J, DS, MINB>, 32 * t.GW, smem, gb.n_items);
        k_line_bwd<J, DS, MINB><<<grid, 32 * t.GW, smem, s>>>(gb, t.GW, t.LCB);
        c->launches++;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_near<32 * J, true>(c, g, s);
}

// Supported (lambda points per thread, depths per warp, minimum resident CTAs per SM).
#define PZ_TILE_LIST(X) \
    X(4, 6, 1) X(4, 6, 2) X(4, 6, 3) X(4, 6, 4) X(4, 8, 1) X(4, 8, 2) X(4, 8, 3) X(4, 12, 1) X(4, 12, 2) \
    X(2, 6, 4) X(2, 8, 2) X(2, 8, 3) X(2, 8, 4) X(2, 12, 1) X(2, 12, 2) X(2, 12, 3) X(4, 6, 5) X(4, 6, 6) X(2, 6, 6) X(2, 8, 5)

#define PZ_TILE_DISPATCH(FN)                                                        \
    const Tiling &t = c->tiling;                                                    \
    PZ_TILE_LIST(PZ_TILE_CASE_##FN)                                                 \
    return cudaErrorInvalidConfiguration;
#define PZ_TILE_CASE_launch_fwd_t(A, B, M) \
    if (t.J == A && t.DS == B && t.minb == M) return launch_fwd_t<A, B, M>(c, s);
#define PZ_TILE_CASE_launch_bwd_t(A, B, M) \
    if (t.J == A && t.DS == B && t.minb == M) return launch_bwd_t<A, B, M>(c, s);

cudaError_t launch_line_fwd_mixed(pz_ctx *c, cudaStream_t s) { PZ_TILE_DISPATCH(launch_fwd_t) }
cudaError_t launch_line_bwd_mixed(pz_ctx *c, cudaStream_t s) { PZ_TILE_DISPATCH(launch_bwd_t) }

bool tiling_supported(int J, int DS, int minb) {
#define PZ_TILE_OK(A, B, M) \
    if (J == A && DS == B && minb == M) return true;
    PZ_TILE_LIST(PZ_TILE_OK)
#undef PZ_TILE_OK
    return false;
}

// ---------------------------------------------------------------------------
// Plain FP64 GPU form: one thread per (lambda, depth), FP64 Voigt, no shared
// memory, no compensation; every line term is evaluated from the line table.
// ---------------------------------------------------------------------------

struct Fp64Args {
    int64_t nlam, ld, nl;
    int nd, ns, W;
    double lnr, lam0cm;
    const int32_t *il;       // integer centres, sorted within each star's segment
    const int64_t *line_off; // [S+1] star segments
    const int32_t *star;
    const double *x64;       // fractional centre
    const int32_t *sp;
    const float *lg_gf, *dgf, *E, *lg_rad, *lg_4, *lg_6, *dg6, *dgrad, *dg4;
    const double *T, *rho, *ne, *npert, *pop, *mass, *xi, *dab;   // [S][nd], [S][ns][nd], [S][ns], [S]
    int dsel;                // backward: damping family of the second sum (0 vdW, 1 rad, 2 Stark)
    const int32_t *eos;
    double *kline;           // [S][nd][ld]
    const double *Gt;        // [S][nd][ld]
    double *gacc;
    const uint32_t *keep;    // centre-test mask [nl][kKeepWords] or NULL (all kept)
    const double *kc;        // [S][nd][ld] continuum opacity (centre test)
};

struct LineTerm64 {
    double A, a, a6, kv;   // strength, damping, the selected family's part of it, c/dv_D
};

__device__ __forceinline__ LineTerm64 term64(const Fp64Args &g, int64_t l, int st, int d) {
    LineTerm64 q;
    const int s = g.sp[l];
    const int64_t sd = (int64_t)st * g.nd + d;
    const double T = g.T[sd];
    const double xi = g.xi[st];
    const double dv = sqrt(2.0 * kKB * T / (g.mass[(int64_t)st * g.ns + s] * kAMU) + xi * xi);
    const double lamcm = g.lam0cm * exp(g.x64[l] * g.lnr);
    const double inv_dnu = lamcm / dv;
    const double gf = exp10((double)g.lg_gf[l] + (double)g.dgf[l]);
    const double dab = (g.eos && g.eos[s] >= 0) ? g.dab[g.eos[s]] : 0.0;
    const double pop = g.pop[((int64_t)st * g.ns + s) * g.nd + d] * exp10(dab);
    const double boltz = exp(-(double)g.E[l] * kEV / (kKB * T));
    q.A = (kPI * kE * kE / (kME * kC)) / kSQRTPI * gf * (pop / g.rho[sd]) * boltz * inv_dnu;
    const double g6n = exp10((double)g.lg_6[l] + (double)g.dg6[l]) * g.npert[sd];
    const double grad = exp10((double)g.lg_rad[l] + (double)g.dgrad[l]);
    const double g4n = exp10((double)g.lg_4[l] + (double)g.dg4[l]) * g.ne[sd];
    q.a = (grad + g4n + g6n) * inv_dnu / (4.0 * kPI);
    q.a6 = (g.dsel == 0 ? g6n : (g.dsel == 1 ? grad : g4n)) * inv_dnu / (4.0 * kPI);
    q.kv = kC / dv;
    return q;
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t lo, int64_t hi, int32_t key) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// one thread per (lambda, depth, star); loops over the star's lines whose window covers lambda
__global__ void k_line_fwd_fp64(Fp64Args g) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y, st = blockIdx.z;
    if (i >= g.nlam) return;
    const int64_t b0 = g.line_off[st], b1 = g.line_off[st + 1];
    const int64_t l0 = lower_bound_i32(g.il, b0, b1, (int32_t)(i - g.W));
    const int64_t l1 = lower_bound_i32(g.il, b0, b1, (int32_t)(i + g.W + 1));
    double sum = 0.0;
    for (int64_t l = l0; l < l1; ++l) {
        if (!pair_kept(g.keep, l, d)) continue;
        LineTerm64 q = term64(g, l, st, d);
        double u = expm1((g.x64[l] - (double)i) * g.lnr);   // lambda_l/lambda_i - 1
        double H, dH;
        voigt64(u * q.kv, q.a, H, dH, false);
        sum += q.A * H;
    }
    const double lam = g.lam0cm * exp((double)i * g.lnr);
    const double stim = -expm1(-kC2 / (lam * g.T[(int64_t)st * g.nd + d]));
    g.kline[((int64_t)st * g.nd + d) * g.ld + i] = stim * sum;
}

// one thread per (line, depth); loops over the line's window
__global__ void k_line_bwd_fp64(Fp64Args g) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (l >= g.nl || !pair_kept(g.keep, l, d)) return;
    const int st = g.star[l];
    LineTerm64 q = term64(g, l, st, d);
    const int64_t il = g.il[l];
    const int64_t i0 = max((int64_t)0, il - g.W), i1 = min(g.nlam - 1, il + g.W);
    const double *Grow = g.Gt + ((int64_t)st * g.nd + d) * g.ld;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = i0; i <= i1; ++i) {
        double u = expm1((g.x64[l] - (double)i) * g.lnr);
        double H, dH;
        voigt64(u * q.kv, q.a, H, dH, true);
        double gs = Grow[i];
        s1 += gs * q.A * H;
        s2 += gs * q.A * dH * q.a6;
    }
    atomicAdd(g.gacc + l, s1);
    atomicAdd(g.gacc + g.nl + l, s2);
}

static Fp64Args make_args64(pz_ctx *c) {
    Fp64Args g;
    g.nlam = c->nlam;
    g.ld = c->ld;
    g.nl = c->L.n;
    g.nd = c->nd;
    g.ns = c->ns;
    g.W = c->W;
    g.lnr = c->lnr;
    g.lam0cm = c->lambda0_nm * 1e-7;
    g.il = c->L.il32;
    g.line_off = c->d_line_off;
    g.star = c->L.star;
    g.x64 = c->L.x64;
    g.sp = c->L.sp;
    g.lg_gf = c->L.lg_gf;
    g.dgf = c->L.dgf;
    g.E = c->L.E;
    g.lg_rad = c->L.lg_rad;
    g.lg_4 = c->L.lg_4;
    g.lg_6 = c->L.lg_6;
    g.dg6 = c->L.dg6;
    g.dgrad = c->L.dgrad;
    g.dg4 = c->L.dg4;
    g.dsel = c->bwd_dsel;
    g.T = c->d_T;
    g.rho = c->d_rho64;
    g.ne = c->d_ne64;
    g.npert = c->d_npert64;
    g.pop = c->d_pop64;
    g.mass = c->d_mass64;
    g.xi = c->d_xi64;
    g.dab = c->d_dab;
    g.eos = c->n_elem > 0 ? c->d_eos : nullptr;
    g.kline = (double *)c->d_kline;
    g.Gt = c->d_Gt64;
    g.gacc = c->d_gacc + c->gacc_off;
    g.keep = c->d_keep;
    g.kc = c->d_kc;
    return g;
}

// Centre-test mask, once per call of pz_set_centre_test, in FP64 (the decision is the
// same rule as the FP64 oracle's): the pair (l, d) is kept when the peak of its term at
// its centre grid point ic (i_l clipped to the grid), bounded with H(a, 0) <= 1,
// reaches eta times the continuum there:
//   (1 - exp(-h c / (lambda_ic k T_d))) A_ld >= eta kappa_c(ic, d).
// One thread per (line, depth); kept pairs set their bit and are counted.
__global__ void k_centre_mask(Fp64Args g, double eta, uint32_t *keep, unsigned long long *count) {
    const int64_t n = g.nl * g.nd;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = k / g.nd;
        const int d = (int)(k - l * g.nd);
        const int st = g.star[l];
        const LineTerm64 q = term64(g, l, st, d);
        const int64_t ic = min(max((int64_t)g.il[l], (int64_t)0), g.nlam - 1);
        const double lam = g.lam0cm * exp((double)ic * g.lnr);
        const double stim = -expm1(-kC2 / (lam * g.T[(int64_t)st * g.nd + d]));
        const double kc = g.kc[((int64_t)st * g.nd + d) * g.ld + ic];
        if (stim * q.A >= eta * kc) {
            atomicOr(keep + l * kKeepWords + (d >> 5), 1u << (d & 31));
            if (count) atomicAdd(count, 1ull);
        }
    }
}

cudaError_t launch_centre_mask(pz_ctx *c, double eta, unsigned long long *d_count, cudaStream_t s) {
    Fp64Args g = make_args64(c);
    const int64_t n = c->L.n * (int64_t)c->nd;
    if (n == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)std::max(c->n_sm, 1) * 32);
    k_centre_mask<<<grid, 256, 0, s>>>(g, eta, c->d_keep, d_count);
    return cudaGetLastError();
}

cudaError_t launch_line_fwd_fp64(pz_ctx *c, cudaStream_t s) {
    Fp64Args g = make_args64(c);
    dim3 grid((unsigned)((c->nlam + 127) / 128), c->nd, c->S);
    k_line_fwd_fp64<<<grid, 128, 0, s>>>(g);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_line_bwd_fp64(pz_ctx *c, cudaStream_t s) {
    if (c->L.n == 0) return cudaSuccess;
    Fp64Args g = make_args64(c);
    dim3 grid((unsigned)((c->L.n + 127) / 128), c->nd);
    k_line_bwd_fp64<<<grid, 128, 0, s>>>(g);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// corrections (Eq. 10): the per-line values are gathered from the caller-order (master)
// corrections, Q_l = Qbase_l 10^dgf, gamma_beta,l = gamma_beta,l(base) 10^dbeta for the
// three damping families, R_sd = Rbase_sd 10^dab
// ---------------------------------------------------------------------------
struct CorrArgs {
    int64_t n;
    const int32_t *orig;
    const double *Qbase;
    const float *g6base, *gradbase, *g4base;
    const float *mdgf, *mdg6, *mdgrad, *mdg4;   // caller order
    float *dgf, *dg6, *dgrad, *dg4;             // per line
    float *Q, *g6, *grad, *g4;
};

__global__ void k_apply_line_corr(CorrArgs a) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.n) return;
    const int32_t o = a.orig[l];
    const float cgf = a.mdgf[o], c6 = a.mdg6[o], cr = a.mdgrad[o], c4 = a.mdg4[o];
    a.dgf[l] = cgf;
    a.dg6[l] = c6;
    a.dgrad[l] = cr;
    a.dg4[l] = c4;
    a.Q[l] = (float)(a.Qbase[l] * exp10((double)cgf));
    a.g6[l] = (float)((double)a.g6base[l] * exp10((double)c6));
    a.grad[l] = (float)((double)a.gradbase[l] * exp10((double)cr));
    a.g4[l] = (float)((double)a.g4base[l] * exp10((double)c4));
}

// R over [S][ns][nd]
__global__ void k_apply_abund(int64_t n, int ns, int nd, const double *Rbase, const double *dab, const int32_t *eos,
                              int use, float *R) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    int s = (int)((idx / nd) % ns);
    double f = (use && eos[s] >= 0) ? exp10(dab[eos[s]]) : 1.0;
    R[idx] = (float)(Rbase[idx] * f);
}

cudaError_t launch_apply_corrections(pz_ctx *c, cudaStream_t s) {
    if (c->L.n > 0) {
        CorrArgs a{c->L.n,     c->L.orig,  c->L.Qbase, c->L.g6base, c->L.gradbase, c->L.g4base,
                   c->d_mdgf,  c->d_mdg6,  c->d_mdgrad, c->d_mdg4, c->L.dgf,      c->L.dg6,
                   c->L.dgrad, c->L.dg4,   c->L.Q,     c->L.g6,     c->L.grad,     c->L.g4};
        k_apply_line_corr<<<(unsigned)((c->L.n + 255) / 256), 256, 0, s>>>(a);
        c->launches++;
    }
    int64_t n = (int64_t)c->S * c->ns * c->nd;
    k_apply_abund<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c->ns, c->nd, c->d_Rbase, c->d_dab, c->d_eos,
                                                             c->n_elem > 0, c->d_R);
    c->launches++;
    return cudaGetLastError();
}

// plain gradient step on the caller-order corrections: delta -= lr * dL/ddelta
__global__ void k_update_corr(int64_t n, const double *gline, float lr_gf, float lr_g6, float *mdgf, float *mdg6) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    mdgf[k] = (float)((double)mdgf[k] - (double)lr_gf * gline[k]);
    mdg6[k] = (float)((double)mdg6[k] - (double)lr_g6 * gline[n + k]);
}

__global__ void k_update_abund(int n, const double *gab, double lr, double *dab) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dab[k] -= lr * gab[k];
}

cudaError_t launch_update(pz_ctx *c, float lr_gf, float lr_g6, float lr_ab, cudaStream_t s) {
    if (c->nl_caller > 0) {
        k_update_corr<<<(unsigned)((c->nl_caller + 255) / 256), 256, 0, s>>>(c->nl_caller, c->d_gline, lr_gf, lr_g6,
                                                                            c->d_mdgf, c->d_mdg6);
        c->launches++;
    }
    if (c->n_elem > 0) {
        k_update_abund<<<(c->n_elem + 255) / 256, 256, 0, s>>>(c->n_elem, c->d_gab, (double)lr_ab, c->d_dab);
        c->launches++;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// linked correction groups (Sec. 6): every member l of group q takes the group's four
// corrections, delta_{q(l)}, and the group's gradient is the sum of its members'
// ---------------------------------------------------------------------------
// x: [4][G] (gf, rad, Stark, vdW) -> caller-order masters; lines without a group take 0
__global__ void k_group_gather(int64_t n, int64_t G, const int32_t *grp, const float *x, float *mdgf, float *mdgrad,
                               float *mdg4, float *mdg6) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t q = grp[k];
    const bool in = q >= 0;
    mdgf[k] = in ? x[q] : 0.0f;
    mdgrad[k] = in ? x[G + q] : 0.0f;
    mdg4[k] = in ? x[2 * G + q] : 0.0f;
    mdg6[k] = in ? x[3 * G + q] : 0.0f;
}

// one thread per group: FP64 sums over the members in CSR order (deterministic) of the
// caller-order gradients gline [4][n] = (gf, vdW, rad, Stark) -> g [4][G] (gf, rad, Stark, vdW)
__global__ void k_group_reduce(int64_t G, int64_t n, const int64_t *off, const int32_t *mem, const double *gline,
                               float *g) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= G) return;
    double sgf = 0.0, s6 = 0.0, sr = 0.0, s4 = 0.0;
    for (int64_t k = off[q]; k < off[q + 1]; ++k) {
        const int64_t l = mem[k];
        sgf += gline[l];
        s6 += gline[n + l];
        sr += gline[2 * n + l];
        s4 += gline[3 * n + l];
    }
    g[q] = (float)sgf;
    g[G + q] = (float)sr;
    g[2 * G + q] = (float)s4;
    g[3 * G + q] = (float)s6;
}

cudaError_t launch_group_gather(pz_ctx *c, const float *x, cudaStream_t s) {
    const int64_t n = c->nl_caller;
    if (n == 0) return cudaSuccess;
    k_group_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c->n_groups, c->d_grp_of, x, c->d_mdgf,
                                                              c->d_mdgrad, c->d_mdg4, c->d_mdg6);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_group_reduce(pz_ctx *c, float *g, cudaStream_t s) {
    const int64_t G = c->n_groups;
    if (G == 0) return cudaSuccess;
    k_group_reduce<<<(unsigned)((G + 255) / 256), 256, 0, s>>>(G, c->nl_caller, c->d_grp_off, c->d_grp_mem,
                                                              c->d_gline, g);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// probe: the FP32 Voigt exactly as the mixed kernels evaluate it
// (far region through the same pre-scaled polynomial with A = 1, a6 = 1)
// ---------------------------------------------------------------------------
__global__ void k_probe_voigt(const float *a, const float *v, int64_t n, float *H, float *dH) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float aa = a[k], x = fabsf(v[k]);
    float a2 = aa * aa;
    float r2 = fmaf(x, x, a2);
    float h, dh;
    if (r2 >= kFar2) {
        float B1 = aa * kInvSqrtPiF;
        float t = rcp_approx(r2);
        float p = fmaf(t, 12.0f * a2 * a2 * B1, -15.0f * a2 * B1);
        p = fmaf(t, p, fmaf(-2.0f, a2, 3.75f) * B1);
        p = fmaf(t, p, 1.5f * B1);
        p = fmaf(t, p, B1);
        h = t * p;
        float C1 = kInvSqrtPiF;
        float q = fmaf(t, -120.0f * a2 * a2 * a2 * C1, 180.0f * a2 * a2 * C1);
        q = fmaf(t, q, a2 * fmaf(12.0f, a2, -67.5f) * C1);
        q = fmaf(t, q, fmaf(-12.0f, a2, 3.75f) * C1);
        q = fmaf(t, q, fmaf(-2.0f, a2, 1.5f) * C1);
        q = fmaf(t, q, C1);
        dh = t * q;
    } else {
        voigt_general<true>(x, aa, h, dh);
    }
    H[k] = h;
    if (dH) dH[k] = dh;
}

cudaError_t launch_probe_voigt(const float *a, const float *v, int64_t n, float *H, float *dH, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_probe_voigt<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, v, n, H, dH);
    return cudaGetLastError();
}

// Pipe-throughput probes (roofline denominators).  Every thread runs 8 independent
// dependency chains for `iters` rounds; the chains stay bounded (x -> 1/(x + 1), which
// no algebraic rewrite removes, for the reciprocal; a contraction toward a fixed point
// for the FMA) and one result per thread is stored so that the work is live.
//   kind 0: packed f32x2 FMA, 16 FP32 operations per thread per round;
//   kind 1: rcp.approx.ftz.f32 (plus one FP32 add), 8 MUFU operations per thread per round;
//   kind 2: FP64 FMA, 8 FP64 FMA operations per thread per round.
__global__ void k_probe_pipe(int kind, int iters, float *out) {
    const float seed = 1.0f + 1e-3f * (float)(threadIdx.x & 63);
    float r = 0.0f;
    if (kind == 0) {
        f2_t x[8];
        const f2_t m = f2_pack(0.999f, 0.998f), c = f2_pack(1e-3f, 2e-3f);
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = f2_pack(seed + k, seed - k);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = f2_fma(x[k], m, c);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float lo, hi;
            f2_unpack(x[k], lo, hi);
            r += lo + hi;
        }
    } else if (kind == 1) {
        float x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = seed + (float)k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = rcp_approx(x[k] + 1.0f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) r += x[k];
    } else {
        double x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = (double)seed + k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fma(x[k], 0.999, 1e-3);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) r += (float)x[k];
    }
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

cudaError_t launch_probe_pipe(int kind, int iters, int blocks, float *out, cudaStream_t s) {
    k_probe_pipe<<<blocks, kProbeThreads, 0, s>>>(kind, iters, out);
    return cudaGetLastError();
}

// Bounded-wait probe: one CTA waits on an mbarrier phase that nothing completes, gives
// up after limit_ns and records the failure exactly as the far-wing kernels do.
__global__ void k_probe_wait(uint64_t limit_ns, int32_t *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, kStatusWaitGaveUp);
}

cudaError_t launch_probe_wait(uint64_t limit_ns, int32_t *status, cudaStream_t s) {
    k_probe_wait<<<1, 32, 0, s>>>(limit_ns, status);
    return cudaGetLastError();
}

}  // namespace pz

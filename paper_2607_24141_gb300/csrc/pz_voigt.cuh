// pz_voigt.cuh -- device Voigt function H(a,v) = Re w(v + i a) and dH/da.
//
// The line profile of Eq. 4 is phi = H(a,v) / (sqrt(pi) dnu_D) with
// a = gamma / (4 pi dnu_D) and v = (nu - nu_l)/dnu_D (Eq. 5).  The paper does
// not name its profile algorithm; this file evaluates H in four regions of
// z = |v| + i a chosen for FP32 on sm_103a (every region keeps Re w to a few
// FP32 ulps even where Re w << |w|):
//
//   |z| >= 20        Laplace asymptotic series of w, two corrections, written
//                    as a polynomial in t = 1/|z|^2 whose coefficients the
//                    kernels pre-scale per (line, depth):
//                      H sqrt(pi) = a t (1 + 1.5 t + (3.75 - 2a^2) t^2 - 15 a^2 t^3 + 12 a^4 t^4)
//                      dH/da sqrt(pi) = t (1 + (1.5 - 2a^2) t + (3.75 - 12 a^2) t^2
//                                       + (12 a^4 - 67.5 a^2) t^3 + 180 a^4 t^4 - 120 a^6 t^5)
//                    (relative truncation error < 3e-7).
//   6 <= |z| < 20    the same series to six corrections in real arithmetic
//                    through the Chebyshev recurrences of sin/cos((2n+1) arg z).
//   |z| < 6, a < 0.5 w = exp(-z^2) + (2i/sqrt(pi)) D(z), D Dawson's integral.
//                    Re/Im D(x + i a) from a Taylor expansion of D about the
//                    nearest table node x_j = j/16 in the complex offset
//                    (x - x_j) + i a; the node coefficients D^(k)(x_j)/k!
//                    (k <= 16) are computed once per device in FP64.
//   |z| < 6, a >= 0.5 Weideman's (1994) rational approximation of order 16,
//                    whose coefficients are the Fourier cosine coefficients of
//                    (L^2 + t^2) e^(-t^2) on t = L tan(theta/2), computed once
//                    per device in FP64.
// In the two core regions dH/da = 2 (v L + a H) - 2/sqrt(pi), L = Im w.
//
// The plain FP64 form uses the asymptotic series to full FP64 accuracy for
// |z| >= 8 and Weideman's approximation of order 32 otherwise.
#pragma once

#include <cuda_runtime.h>

#include "pz_internal.h"

namespace pz {

// Device tables (defined here; this header is included by one translation unit).
__constant__ float c_weid[kWeidN + 1];
__constant__ float c_weidL;
__constant__ double c_weid64[kWeidN64 + 1];
__constant__ double c_weidL64;
// Dawson-derivative table, coefficient-major: g_dawson[k * kDawsonNodes + j] = D^(k)(x_j)/k!.
// Lanes evaluating nearby x read adjacent words of each coefficient row.
__device__ float g_dawson[kDawsonNodes * (kDawsonK + 1)];

constexpr float kInvSqrtPiF = 0.564189583547756287f;
constexpr float kTwoInvSqrtPiF = 1.12837916709551257f;

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Asymptotic series with NC corrections in real arithmetic.  H and (if D) dH/da.
template <int NC, bool D>
__device__ __forceinline__ void voigt_asym(float x, float a, float &H, float &dH) {
    float t = rcp_approx(fmaf(x, x, a * a));
    float qr = x * t, qi = -a * t;                 // q = 1/z
    float q2r = fmaf(qr, qr, -qi * qi), q2i = 2.0f * qr * qi;
    float kr = qr, ki = qi;                        // q^(2n+1)
    float sH = 0.0f, sD = 0.0f, c = 1.0f;
#pragma unroll
    for (int n = 0; n <= NC; ++n) {
        sH = fmaf(c, -ki, sH);
        if (D) sD = fmaf(c * (2.0f * n + 1.0f), fmaf(kr, qr, -ki * qi), sD);
        c *= (2.0f * n + 1.0f) * 0.5f;
        float nr = fmaf(kr, q2r, -ki * q2i);
        ki = fmaf(kr, q2i, ki * q2r);
        kr = nr;
    }
    H = sH * kInvSqrtPiF;
    if (D) dH = sD * kInvSqrtPiF;
}

// Mid wing, 6 <= |z| < 20: the Laplace series to NC corrections in real arithmetic.
// With t = 1/|z|^2, s = a^2 t, cos(theta) = v/|z|, w = 2 - 4s:
//   H sqrt(pi)     = a sum_n c_n t^(n+1) U_2n(cos theta),   U_2n+2 = w U_2n - U_2n-2, U_0 = 1, U_-2 = -1
//   dH/da sqrt(pi) =   sum_n c_n (2n+1) t^(n+1) T_2n+2(cos theta), T_2m+2 = w T_2m - T_2m-2, T_0 = 1, T_2 = w/2
// (c_0 = 1, c_n+1 = c_n (2n+1)/2; U and T Chebyshev polynomials: sin((2n+1)theta) = sin(theta) U_2n,
// cos(2m theta) = T_2m).  NC = 6 keeps the truncation below 2e-7 relative at |z| = 6.
template <bool D>
__device__ __forceinline__ void voigt_mid(float x, float a, float &H, float &dH) {
    constexpr int NC = 6;
    const float t = rcp_approx(fmaf(x, x, a * a));
    const float s = a * a * t;
    const float w = fmaf(-4.0f, s, 2.0f);
    float u0 = 1.0f, um = -1.0f;              // U_2n, U_2n-2
    float g0 = fmaf(0.5f, w, 0.0f), gm = 1.0f; // T_2n+2, T_2n
    float tp = t, c = 1.0f, sh = 0.0f, sd = 0.0f;
#pragma unroll
    for (int n = 0; n <= NC; ++n) {
        sh = fmaf(c * tp, u0, sh);
        if (D) sd = fmaf(c * (2.0f * n + 1.0f) * tp, g0, sd);
        const float un = fmaf(w, u0, -um);
        um = u0;
        u0 = un;
        if (D) {
            const float gn = fmaf(w, g0, -gm);
            gm = g0;
            g0 = gn;
        }
        c *= (2.0f * n + 1.0f) * 0.5f;
        tp *= t;
    }
    H = a * sh * kInvSqrtPiF;
    if (D) dH = sd * kInvSqrtPiF;
}

// Taylor sum of D about the node x_j in the complex offset d + i a to order KK:
// pr + i pi = sum_k T_k(x_j) (d + i a)^k, T_k = D^(k)(x_j)/k! (Horner in complex arithmetic).
template <int KK>
__device__ __forceinline__ void dawson_taylor(float d, float a, const float *T, float &pr, float &pi) {
    pr = T[KK * kDawsonNodes];
    pi = 0.0f;
#pragma unroll
    for (int k = KK - 1; k >= 0; --k) {
        const float nr = fmaf(pr, d, fmaf(-pi, a, T[k * kDawsonNodes]));
        pi = fmaf(pr, a, pi * d);
        pr = nr;
    }
}

// Core, small a: Dawson-derivative table (coefficient-major, in global or shared
// memory).  x >= 0, x*x + a*a < 36, a < 0.5.  The Taylor order follows a (|d| <= 1/32):
// measured in FP64 against the Faddeeva function over 0 <= x <= 6, the truncation stays
// below 3e-8 with order 6 for a < 0.1, 1.1e-8 with order 10 for a < 0.3 and 4e-9 with
// order 14 for a < 0.5.  sin/cos of 2xa (< 6) use the MUFU forms (absolute error below
// 5e-7, scaled by exp(a^2 - x^2) <= H in H and L).
__device__ __forceinline__ void voigt_core_table(float x, float a, float &H, float &L, const float *tab) {
    int j = __float2int_rn(x * (float)kDawsonPerUnit);
    j = min(max(j, 0), kDawsonNodes - 1);
    float d = x - (float)j * (1.0f / kDawsonPerUnit);
    const float *T = tab + j;
    float pr, pi;
    if (a < 0.1f)
        dawson_taylor<6>(d, a, T, pr, pi);
    else if (a < 0.3f)
        dawson_taylor<10>(d, a, T, pr, pi);
    else
        dawson_taylor<14>(d, a, T, pr, pi);
    // exp(a^2 - x^2) with the rounding residual of x^2 folded in
    float x2 = x * x;
    float x2e = fmaf(x, x, -x2);
    float g = expf(fmaf(a, a, -x2) - x2e);
    float s, c;
    __sincosf(2.0f * x * a, &s, &c);
    H = fmaf(g, c, -kTwoInvSqrtPiF * pi);
    L = fmaf(-g, s, kTwoInvSqrtPiF * pr);
}

// Core, a >= 0.5: Weideman rational approximation, order kWeidN.
__device__ __forceinline__ void voigt_core_weideman(float x, float a, float &H, float &L) {
    const float Lw = c_weidL;
    float dr = Lw + a, di = -x;          // L - i z
    float nr = Lw - a, ni = x;           // L + i z
    float inv = 1.0f / fmaf(dr, dr, di * di);
    float Zr = fmaf(nr, dr, ni * di) * inv;
    float Zi = fmaf(ni, dr, -nr * di) * inv;
    float pr = c_weid[kWeidN], pi = 0.0f;
#pragma unroll
    for (int n = kWeidN - 1; n >= 1; --n) {
        float t = fmaf(pr, Zr, fmaf(-pi, Zi, c_weid[n]));
        pi = fmaf(pr, Zi, pi * Zr);
        pr = t;
    }
    float idr = dr * inv, idi = -di * inv;          // 1/(L - i z)
    float i2r = fmaf(idr, idr, -idi * idi), i2i = 2.0f * idr * idi;
    H = fmaf(2.0f, fmaf(pr, i2r, -pi * i2i), idr * kInvSqrtPiF);
    L = fmaf(2.0f, fmaf(pr, i2i, pi * i2r), idi * kInvSqrtPiF);
}

// Core region |z| < 6 (both sub-regions), H and, if D, dH/da.  tab: the Dawson table.
template <bool D>
__device__ __forceinline__ void voigt_core(float x, float a, float &H, float &dH, const float *tab) {
    float L;
    if (a < kCoreA)
        voigt_core_table(x, a, H, L, tab);
    else
        voigt_core_weideman(x, a, H, L);
    if (D) dH = 2.0f * fmaf(x, L, a * H) - kTwoInvSqrtPiF;
}

// General evaluation (any region).  x >= 0.  Returns H and, if D, dH/da.
template <bool D>
__device__ __forceinline__ void voigt_general(float x, float a, float &H, float &dH) {
    float r2 = fmaf(x, x, a * a);
    if (r2 >= kMid2) {
        if (r2 >= kFar2)
            voigt_asym<2, D>(x, a, H, dH);
        else
            voigt_mid<D>(x, a, H, dH);
        return;
    }
    voigt_core<D>(x, a, H, dH, g_dawson);
}

// ---- FP64 plain form --------------------------------------------------------
__device__ __forceinline__ void voigt64(double x, double a, double &H, double &dH, bool want_d) {
    x = fabs(x);
    double r2 = x * x + a * a;
    if (r2 >= 64.0) {
        double t = 1.0 / r2;
        double qr = x * t, qi = -a * t;
        double q2r = qr * qr - qi * qi, q2i = 2.0 * qr * qi;
        double kr = qr, ki = qi;
        double sH = 0.0, sD = 0.0, c = 1.0, mag = sqrt(t), m2 = t;
        for (int n = 0; n < 40; ++n) {
            sH += c * (-ki);
            if (want_d) sD += c * (2.0 * n + 1.0) * (kr * qr - ki * qi);
            if (c * mag < 1e-17 * fabs(sH) && n > 1) break;
            c *= (2.0 * n + 1.0) * 0.5;
            mag *= m2;
            double nr = kr * q2r - ki * q2i;
            ki = kr * q2i + ki * q2r;
            kr = nr;
        }
        H = sH * (1.0 / kSQRTPI);
        dH = sD * (1.0 / kSQRTPI);
        return;
    }
    const double Lw = c_weidL64;
    double dr = Lw + a, di = -x, nr = Lw - a, ni = x;
    double inv = 1.0 / (dr * dr + di * di);
    double Zr = (nr * dr + ni * di) * inv, Zi = (ni * dr - nr * di) * inv;
    double pr = c_weid64[kWeidN64], pi = 0.0;
    for (int n = kWeidN64 - 1; n >= 1; --n) {
        double t = pr * Zr - pi * Zi + c_weid64[n];
        pi = pr * Zi + pi * Zr;
        pr = t;
    }
    double idr = dr * inv, idi = -di * inv;
    double i2r = idr * idr - idi * idi, i2i = 2.0 * idr * idi;
    H = 2.0 * (pr * i2r - pi * i2i) + idr / kSQRTPI;
    double L = 2.0 * (pr * i2i + pi * i2r) + idi / kSQRTPI;
    dH = 2.0 * (x * L + a * H) - 2.0 / kSQRTPI;
}

}  // namespace pz

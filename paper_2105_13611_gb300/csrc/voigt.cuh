// FP32 Voigt function H(v, a) = Re w(v + i a) for the profile of Eq. (l_nu_line).
//
// Three tiers, chosen per point by |z|^2 = v^2 + a^2:
//
//  far   |z|^2 >= 1600: the one-level Laplace continued fraction
//        w ~ (i/sqrt(pi)) / (z - 1/(2z)) with its real part written out:
//        H = (a/sqrt(pi)) y (2 + 4y) / (1 + 8 a^2 y^2),  y = 1/(2|z|^2 - 1).
//        Relative error <= 1.2e-6; one reciprocal, no cancellation.
//  mid   36 <= |z|^2 < 1600: the Laplace continued fraction with five levels
//        (partial numerators 5/2, 2, 3/2, 1, 1/2) evaluated bottom-up on
//        separate real and imaginary parts.  The imaginary part of every level
//        is a sum of positive terms, so H = Im t / (sqrt(pi) |t|^2) keeps full
//        relative accuracy even for tiny a.  exp(-v^2) is added for a < 1e-2,
//        where the fraction omits the Gaussian core.
//  core  |z|^2 < 36: Humlicek's (1979) shifted-contour Gauss-Hermite sum.
//        Shifting the integration path of w(z) = (i/pi) int e^{-t^2}/(z-t) dt
//        by delta = 1.5 below the real axis and applying 12-point Gauss-Hermite
//        quadrature gives w(z) ~ sum_k c_k /(z + i delta - s_k) with
//        c_k = (i/pi) e^{delta^2} omega_k e^{2 i delta s_k}.  For a >= 2 the real
//        part of the sum is used directly ("region I"); for a < 2 the exact
//        exp(-v^2) is taken for the real axis and only the a-dependent part
//        Re[R(z) - R(v)] comes from the sum, written with an explicit factor a
//        ("region II").  The constants are computed on the host from the
//        Hermite nodes and weights (mpsa::voigt_init).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace mpsa {

constexpr int kGHPairs = 6;          // 12-point Gauss-Hermite, symmetric pairs
constexpr float kGHDelta = 1.5f;     // contour shift
constexpr float kInvSqrtPi = 0.56418958354775628f;

struct VoigtConsts {
    float s[kGHPairs];   // positive Hermite nodes
    float U[kGHPairs];   // e^{delta^2}/pi * omega_k * cos(2 delta s_k)
    float S[kGHPairs];   // e^{delta^2}/pi * omega_k * sin(2 delta s_k)
};

// Host: the constants from the Hermite nodes and weights (voigt.cu).
int voigt_host_consts(VoigtConsts* out);

// FP64 Voigt for the all-FP64 precision variant: the Laplace continued fraction with 4
// levels for |z|^2 >= 1600 and 16 levels for 36 <= |z|^2 < 1600 (relative error 1.1e-12),
// and the 32-point shifted Gauss-Hermite sum with delta = 2 below (region II for a < 1,
// region I above; 5e-14).
constexpr int kGHPairs64 = 16;
constexpr double kGHDelta64 = 2.0;
struct VoigtConsts64 {
    double s[kGHPairs64], U[kGHPairs64], S[kGHPairs64];
};
int voigt_host_consts64(VoigtConsts64* out);

// Every translation unit that evaluates H keeps its own copy of the constants;
// it uploads them with voigt_upload() once per device before its first launch.
static __constant__ VoigtConsts c_voigt;
static __constant__ VoigtConsts64 c_voigt64;

static inline int voigt_upload() {
    VoigtConsts h;
    VoigtConsts64 h64;
    int rc = voigt_host_consts(&h);
    if (rc == MPSA_OK) rc = voigt_host_consts64(&h64);
    if (rc != MPSA_OK) return rc;
    cudaError_t e = cudaMemcpyToSymbol(c_voigt, &h, sizeof(h));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_voigt64, &h64, sizeof(h64));
    return e == cudaSuccess ? MPSA_OK : fail(MPSA_ECUDA, "cudaMemcpyToSymbol(c_voigt): %s", cudaGetErrorString(e));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// far tier (|z|^2 >= 1600).  V = v^2, A = a^2, ka = a/sqrt(pi).  Where (2 + 2A)/|z|^4 <= 1e-6
// the rational form ka / (|z|^2 - 3/2) (relative error below that bound, from the asymptotic
// series of H to order |z|^-4); otherwise the one-level continued fraction in y = 1/(2|z|^2 - 1)
// with its 8A y^2 correction.
__device__ __forceinline__ float voigt_far(float V, float A, float ka) {
    const float Z = V + A;
    if (Z * Z >= 1.0e6f * fmaf(2.f, A, 2.f)) return ka * rcp_approx(Z - 1.5f);
    float y = rcp_approx(fmaf(2.f, V, fmaf(2.f, A, -1.f)));
    float e = 8.f * A * y * y;
    return ka * y * fmaf(4.f, y, 2.f) * fmaf(e, e - 1.f, 1.f);
}

// mid tier (five continued-fraction levels).  The fraction t <- z - (k/2)/t is carried
// bottom-up as t = P/Q, (P, Q) <- (z P - (k/2) Q, P), so that one reciprocal serves all five
// levels: H = Re(i Q/P)/sqrt(pi) = (Q_r P_i - Q_i P_r) / (sqrt(pi) |P|^2).  For 36 <= |z|^2 <
// 1600, |P| <= |z|^6 < 5e9 and |P|^2 stays inside FP32.
__device__ __forceinline__ float voigt_mid(float v, float a) {
    float pr = v, pi = a, qr = 1.f, qi = 0.f;
#pragma unroll
    for (int k = 5; k >= 1; --k) {
        const float c = 0.5f * (float)k;
        const float npr = fmaf(v, pr, fmaf(-a, pi, -c * qr));
        const float npi = fmaf(v, pi, fmaf(a, pr, -c * qi));
        qr = pr;
        qi = pi;
        pr = npr;
        pi = npi;
    }
    float h = kInvSqrtPi * fmaf(qr, pi, -qi * pr) * rcp_approx(fmaf(pr, pr, pi * pi));
    if (a < 1e-2f) h += expf(-v * v);
    return h;
}

// core tier (shifted Gauss-Hermite, regions I and II).
__device__ __forceinline__ float voigt_core(float v, float a) {
    const float d = kGHDelta;
    const float Y1 = a + d, Y12 = Y1 * Y1;
    float sum = 0.f;
    if (a < 2.f) {
        const float dY = Y1 * d, Yd = Y1 + d, d2 = d * d;
#pragma unroll
        for (int k = 0; k < kGHPairs; ++k) {
            const float sk = c_voigt.s[k], Uk = c_voigt.U[k], Sk = c_voigt.S[k];
            float r = v - sk, rp = v + sk;
            float r2 = r * r, rp2 = rp * rp;
            float p1 = (r2 + d2) * (r2 + Y12);
            float p2 = (rp2 + d2) * (rp2 + Y12);
            float t1 = fmaf(Uk, r2 - dY, Sk * r * Yd);
            float t2 = fmaf(Uk, rp2 - dY, -Sk * rp * Yd);
            sum = fmaf(fmaf(t1, p2, t2 * p1), rcp_approx(p1 * p2), sum);
        }
        return fmaf(a, sum, expf(-v * v));
    }
#pragma unroll
    for (int k = 0; k < kGHPairs; ++k) {
        const float sk = c_voigt.s[k], Uk = c_voigt.U[k], Sk = c_voigt.S[k];
        float r = v - sk, rp = v + sk;
        float q1 = fmaf(r, r, Y12), q2 = fmaf(rp, rp, Y12);
        float UY = Uk * Y1;
        sum = fmaf(fmaf(q2, fmaf(-Sk, r, UY), q1 * fmaf(Sk, rp, UY)), rcp_approx(q1 * q2), sum);
    }
    return sum;
}

// H(v, a) for any v (sign ignored) and a > 0.
__device__ __forceinline__ float voigt_H(float v, float a) {
    v = fabsf(v);
    const float V = v * v, A = a * a, Z = V + A;
    if (Z >= 1600.f) return voigt_far(V, A, a * kInvSqrtPi);
    if (Z >= 36.f) return voigt_mid(v, a);
    return voigt_core(v, a);
}

// The same function with the two inner tiers as out-of-line calls: used where it is
// replicated many times in one kernel (the far tier, taken by most points, stays inline).
static __device__ __noinline__ float voigt_inner_tiers(float v, float a) {
    return (v * v + a * a >= 36.f) ? voigt_mid(v, a) : voigt_core(v, a);
}
__device__ __forceinline__ float voigt_H_lean(float v, float a) {
    v = fabsf(v);
    const float V = v * v, A = a * a;
    if (V + A >= 1600.f) return voigt_far(V, A, a * kInvSqrtPi);
    return voigt_inner_tiers(v, a);
}

// FP64 H(v, a) (see VoigtConsts64).
__device__ inline double voigt_H64(double v, double a) {
    v = fabs(v);
    const double Z = v * v + a * a;
    if (Z >= 36.0) {
        // continued fraction t <- z - (k/2)/t, bottom-up, with t = P/Q kept as a fraction
        // (P, Q) <- (z P - (k/2) Q, P) so that only the final step divides; H = Re(i Q/P)/sqrt(pi).
        // |P| grows like |z|^(levels+1), far inside the FP64 range for any grid.
        const int levels = Z >= 1600.0 ? 4 : 16;   // 4 levels reach 1e-14 for |z| >= 40
        double pr = v, pi = a, qr = 1.0, qi = 0.0;
        for (int k = levels; k >= 1; --k) {
            const double c = 0.5 * k;
            const double npr = fma(-c, qr, fma(v, pr, -a * pi));
            const double npi = fma(-c, qi, fma(v, pi, a * pr));
            qr = pr;
            qi = pi;
            pr = npr;
            pi = npi;
        }
        double h = (qr * pi - qi * pr) / (1.7724538509055160273 * fma(pr, pr, pi * pi));
        if (a < 1e-2) h += exp(a * a - v * v) * cos(2.0 * v * a);
        return h;
    }
    const double d = kGHDelta64;
    const double Y1 = a + d, Y12 = Y1 * Y1;
    double sum = 0.0;
    if (a < 1.0) {
        const double dY = Y1 * d, Yd = Y1 + d, d2 = d * d;
        for (int k = 0; k < kGHPairs64; ++k) {
            const double sk = c_voigt64.s[k], Uk = c_voigt64.U[k], Sk = c_voigt64.S[k];
            const double r = v - sk, rp = v + sk, r2 = r * r, rp2 = rp * rp;
            sum += (Uk * (r2 - dY) + Sk * r * Yd) / ((r2 + d2) * (r2 + Y12)) +
                   (Uk * (rp2 - dY) - Sk * rp * Yd) / ((rp2 + d2) * (rp2 + Y12));
        }
        return exp(-v * v) + a * sum;
    }
    for (int k = 0; k < kGHPairs64; ++k) {
        const double sk = c_voigt64.s[k], Uk = c_voigt64.U[k], Sk = c_voigt64.S[k];
        const double r = v - sk, rp = v + sk;
        sum += (Uk * Y1 - Sk * r) / (r * r + Y12) + (Uk * Y1 + Sk * rp) / (rp * rp + Y12);
    }
    return sum;
}

}  // namespace mpsa

// Host-side set-up of the Voigt constants: 12-point Gauss-Hermite nodes and
// weights computed from the Hermite polynomials, then the shifted-contour
// coefficients of Humlicek (1979).  FP64 on the host, copied once per device.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "voigt.cuh"

namespace mpsa {

namespace {

// Physicists' Hermite polynomial H_n(x) and H_{n-1}(x) by the three-term recurrence
// H_{k+1} = 2x H_k - 2k H_{k-1}.
void hermite(int n, double x, double* hn, double* hn1) {
    double h0 = 1.0, h1 = 2.0 * x;
    if (n == 0) { *hn = h0; *hn1 = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double h2 = 2.0 * x * h1 - 2.0 * k * h0;
        h0 = h1;
        h1 = h2;
    }
    *hn = h1;
    *hn1 = h0;
}

}  // namespace

namespace {
// positive roots and weights of the n-point Gauss-Hermite rule (n even)
int gauss_hermite(int n, double* nodes, double* weights) {
    const int half = n / 2;
    int found = 0;
    const double xmax = sqrt(2.0 * n + 1.0) + 1.0;
    const int steps = 40000;
    double xprev = 1e-9, hprev, dummy;
    hermite(n, xprev, &hprev, &dummy);
    for (int i = 1; i <= steps && found < half; ++i) {
        double x = xmax * i / steps, h;
        hermite(n, x, &h, &dummy);
        if ((h > 0) != (hprev > 0)) {
            double lo = xprev, hi = x, hlo = hprev;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi), hm;
                hermite(n, mid, &hm, &dummy);
                if ((hm > 0) == (hlo > 0)) { lo = mid; hlo = hm; } else { hi = mid; }
            }
            nodes[found++] = 0.5 * (lo + hi);
        }
        xprev = x;
        hprev = h;
    }
    if (found != half) return fail(MPSA_EINVAL, "gauss_hermite(%d): found %d roots", n, found);
    // omega_k = 2^{n-1} n! sqrt(pi) / (n^2 H_{n-1}(x_k)^2), in logs to avoid overflow
    double lfact = 0.0;
    for (int k = 2; k <= n; ++k) lfact += log((double)k);
    for (int k = 0; k < half; ++k) {
        double hn, hn1;
        hermite(n, nodes[k], &hn, &hn1);
        weights[k] = exp((n - 1) * log(2.0) + lfact + 0.5 * log(kPI) - 2.0 * log((double)n) - 2.0 * log(fabs(hn1)));
    }
    return MPSA_OK;
}
}  // namespace

int voigt_host_consts64(VoigtConsts64* out) {
    double nodes[kGHPairs64], weights[kGHPairs64];
    int r = gauss_hermite(2 * kGHPairs64, nodes, weights);
    if (r != MPSA_OK) return r;
    const double dl = kGHDelta64;
    const double pre = exp(dl * dl) / kPI;
    for (int k = 0; k < kGHPairs64; ++k) {
        out->s[k] = nodes[k];
        out->U[k] = pre * weights[k] * cos(2.0 * dl * nodes[k]);
        out->S[k] = pre * weights[k] * sin(2.0 * dl * nodes[k]);
    }
    return MPSA_OK;
}

int voigt_host_consts(VoigtConsts* out) {
    double nodes[kGHPairs], weights[kGHPairs];
    int r = gauss_hermite(2 * kGHPairs, nodes, weights);
    if (r != MPSA_OK) return r;
    VoigtConsts& h = *out;
    const double dl = (double)kGHDelta;
    const double pre = exp(dl * dl) / kPI;
    for (int k = 0; k < kGHPairs; ++k) {
        h.s[k] = (float)nodes[k];
        h.U[k] = (float)(pre * weights[k] * cos(2.0 * dl * nodes[k]));
        h.S[k] = (float)(pre * weights[k] * sin(2.0 * dl * nodes[k]));
    }
    return MPSA_OK;
}

}  // namespace mpsa

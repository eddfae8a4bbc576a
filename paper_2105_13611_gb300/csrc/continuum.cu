// synth_continuum: continuous opacity from the closed-form sources of the paper's continuum
// (Sect. 2.1: electron scattering, bound-free and free-free absorption of H I, Rayleigh
// scattering on H I) on a log-lambda grid, per row of the population table.
//
// Per unit volume at frequency nu = c / lambda:
//   electron scattering     n_e sigma_T
//   H I bound-free          sum over levels n = 1..8 with nu >= chi_H / (h n^2) of
//                           N_n K_bf / (n^5 nu^3) (1 - e^{-h nu/kT}),
//                           N_n = n_HI (2 n^2 / U_HI) e^{-chi_H (1 - 1/n^2)/kT} (Kramers, Gaunt factor 1)
//   H I free-free           K_ff n_e n_HII / (sqrt(T) nu^3) (1 - e^{-h nu/kT})   (Kramers, Gaunt factor 1)
//   H I Rayleigh            n_HI (5.799e-13 / L^4 + 1.422e-6 / L^6 + 2.784 / L^8) cm^2, L in Angstrom,
//                           held at L = 1300 Angstrom below (the series diverges towards Lyman alpha)
// divided by rho.  K_bf = 64 pi^4 m_e e^10 / (3 sqrt(3) c h^6), K_ff = (4 e^6 / (3 m_e h c))
// sqrt(2 pi / (3 k m_e)).  The per-row constants are formed in FP64 (k_cont_rows), the
// per-point sums in FP32; whether a level's edge is passed is decided by grid index, the
// edges found on the host in FP64 (the last grid point at or shortward of each edge).
#include <math.h>

#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace mpsa {
namespace {

constexpr int kLevels = 8;
constexpr double kChiH = 13.598;                 // eV
constexpr double kSigmaT = 6.6524587321e-25;     // cm^2
constexpr float kRayMinA = 1300.f;               // Angstrom

// The frequency enters in units of 1e15 Hz (so 1/nu^3 and the coefficients stay inside the FP32
// range: 1/nu^3 in s^3 would underflow at short wavelengths and K_bf N_n / rho overflow).
constexpr double kNuUnit = 1e15;

struct ContRow {
    float elec;             // n_e sigma_T / rho
    float bf[kLevels + 1];  // suffix sums over levels n..8 of N_n K_bf / (n^5 rho) / nu_unit^3; bf[8] = 0
    float ff;               // K_ff n_e n_HII / (sqrt(T) rho) / nu_unit^3
    float ray;              // n_HI / rho
    float h_kT;             // h nu_unit / kT
};

__global__ void k_cont_rows(int n_sel, const int* __restrict__ sel, int n_el, const double* __restrict__ el,
                            const double* __restrict__ pop, int sources, ContRow* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sel) return;
    const double* row = pop + (size_t)sel[s] * pop_stride(n_el);
    const double T = row[kPopT], ne = row[kPopNe], nHI = row[kPopNHI], rho = row[kPopRho];
    const double kT = kKB * T, x = log(T / 5040.0);
    // partition functions of H I and H II at T (element 0 is hydrogen)
    const double* c0 = el + kElLnU;
    const double U1 = exp(c0[0] + x * (c0[1] + x * c0[2]));
    const double U2 = el[kElStages] > 1.0 ? exp(c0[3] + x * (c0[4] + x * c0[5])) : 1.0;
    const double nHII = el[kElStages] > 1.0 ? row[pop_nu(0, 1)] * U2 : 0.0;
    const double Kbf = 64.0 * pow(kPI, 4) * kME * pow(kE, 10) / (3.0 * sqrt(3.0) * kC * pow(kH, 6));
    const double Kff = 4.0 * pow(kE, 6) / (3.0 * kME * kH * kC) * sqrt(2.0 * kPI / (3.0 * kKB * kME));
    const double chi = kChiH * kEV;
    ContRow r;
    r.elec = (sources & MPSA_CONT_ELEC) ? (float)(ne * kSigmaT / rho) : 0.f;
    double acc = 0.0;
    r.bf[kLevels] = 0.f;
    for (int n = kLevels; n >= 1; --n) {
        const double Nn = nHI * 2.0 * n * n / U1 * exp(-chi * (1.0 - 1.0 / ((double)n * n)) / kT);
        acc += (sources & MPSA_CONT_HBF) ? Nn * Kbf / (pow((double)n, 5) * rho) / (kNuUnit * kNuUnit * kNuUnit) : 0.0;
        r.bf[n - 1] = (float)acc;
    }
    r.ff = (sources & MPSA_CONT_HFF) ? (float)(Kff * ne * nHII / (sqrt(T) * rho) / (kNuUnit * kNuUnit * kNuUnit)) : 0.f;
    r.ray = (sources & MPSA_CONT_HRAY) ? (float)(nHI / rho) : 0.f;
    r.h_kT = (float)(kH * kNuUnit / kT);
    out[s] = r;
}

// one thread per grid point, rows on the grid's y dimension
__global__ void __launch_bounds__(256) k_continuum(int N, float lam0_cm, float lnq, const int* __restrict__ edge,
                                                   const ContRow* __restrict__ rows, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (j >= N) return;
    const ContRow& r = rows[s];
    const float lam = lam0_cm * expf((float)j * lnq);      // cm
    const float t = lam * (float)(kNuUnit / 2.99792458e10);   // nu_unit / nu
    const float inv_nu3 = t * t * t;
    const float stim = -expm1f(-r.h_kT / t);
    // levels with their edge at or longward of this point: n >= n_min
    int n_min = 0;
#pragma unroll
    for (int n = 0; n < kLevels; ++n) n_min += j > edge[n];
    const float L = fmaxf(lam * 1e8f, kRayMinA);
    const float iL2 = 1.f / (L * L);
    const float ray = ((2.784f * iL2 + 1.422e-6f) * iL2 + 5.799e-13f) * iL2 * iL2;
    out[(size_t)s * N + j] = r.elec + (r.bf[n_min] + r.ff) * inv_nu3 * stim + r.ray * ray;
}

// grid index of the last point at or shortward of each level's edge (lambda_j <= lambda_n, i.e.
// nu_j >= nu_n), by bisection on the FP64 grid wavelengths; -1 if none
void level_edges(double lam0_nm, double R, int N, int* edge) {
    const double lnq = log1p(1.0 / R);
    for (int n = 1; n <= kLevels; ++n) {
        const double nu_n = kChiH * kEV / (kH * n * n);
        auto ok = [&](long long j) { return kC / (lam0_nm * exp((double)j * lnq) * 1e-7) >= nu_n; };
        long long lo = -1, hi = N;   // ok(lo) (or lo = -1), !ok(hi) (or hi = N)
        while (hi - lo > 1) {
            const long long mid = (lo + hi) / 2;
            if (ok(mid)) lo = mid; else hi = mid;
        }
        edge[n - 1] = (int)lo;
    }
}

}  // namespace

int continuum_launch(mpsa_ctx* ctx, const double* pop, int n_sel, const int* d_sel, double lam0_nm, double R, int N,
                     int sources, float* out, cudaStream_t st) {
    Scratch sc(st, ctx->pool);
    ContRow* rows;
    int* d_edge;
    int r;
    if ((r = sc.alloc(&rows, n_sel)) || (r = sc.alloc(&d_edge, kLevels))) return r;
    int edge[kLevels];
    level_edges(lam0_nm, R, N, edge);
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_edge, edge, sizeof edge, cudaMemcpyHostToDevice, st));
    k_cont_rows<<<(n_sel + 63) / 64, 64, 0, st>>>(n_sel, d_sel, ctx->n_el, ctx->d_el, pop, sources, rows);
    k_continuum<<<dim3((N + 255) / 256, n_sel), 256, 0, st>>>(N, (float)(lam0_nm * 1e-7), (float)log1p(1.0 / R),
                                                              d_edge, rows, out);
    MPSA_CUDA_TRY(cudaGetLastError());
    return MPSA_OK;
}

}  // namespace mpsa

using namespace mpsa;

extern "C" int synth_continuum(mpsa_ctx* ctx, const mpsa_lgrid* grid, int32_t n_sel, const int32_t* sel,
                               int32_t sources, float* kappa_out, void* stream) {
    if (!ctx || !grid || !sel || !kappa_out) return fail(MPSA_EINVAL, "synth_continuum: NULL argument");
    if (!ctx->d_pop) return fail(MPSA_ESTATE, "synth_continuum: no atmosphere grid set");
    if (n_sel < 1 || n_sel > 65535) return fail(MPSA_EINVAL, "synth_continuum: n_sel = %d (1..65535)", n_sel);
    if (sources & ~MPSA_CONT_ALL) return fail(MPSA_EINVAL, "synth_continuum: sources = %d", sources);
    const int rows = ctx->n_comp * ctx->n_points;
    for (int i = 0; i < n_sel; ++i)
        if (sel[i] < 0 || sel[i] >= rows)
            return fail(MPSA_EINVAL, "synth_continuum: sel[%d] = %d of %d rows", i, sel[i], rows);
    int N, r;
    if ((r = check_grid(grid, &N))) return r;
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st, ctx->pool);
    int* d_sel;
    if ((r = sc.alloc(&d_sel, n_sel))) return r;
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_sel, sel, n_sel * sizeof(int), cudaMemcpyHostToDevice, st));
    prof_mark(ctx, MPSA_KERNEL_CONTINUUM, st);
    r = continuum_launch(ctx, ctx->d_pop, n_sel, d_sel, grid->lambda0_nm, grid->R, N, sources, kappa_out, st);
    prof_mark(ctx, MPSA_KERNEL_CONTINUUM, st);
    return r;
}

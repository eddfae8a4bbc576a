// synth_spectrum: emergent intensity of one model atmosphere (paper Eq. Ilambda,
// LTE source S = B_lambda(T), no scattering).
//
// Per depth the populations (FP64, same kernel as set_atmosphere_grid), the line
// opacity on the window grid (synth_rows, the synth_opacity pipeline) and the
// flat continuum are computed; k_formal then integrates, per wavelength point,
//   tau_0 = kappa_0 m_0, tau_{d+1} = tau_d + (kappa_d + kappa_{d+1})(m_{d+1} - m_d)/2,
//   I_{D-1} = S_{D-1} + mu dS/dtau (diffusion),
//   I_d = I_{d+1} e^{-x} + S_d (1 - e^{-x}) + (S_{d+1} - S_d)(1 - e^{-x}(1 + x))/x,  x = dtau/mu,
//   I = I_0 e^{-tau_0/mu} + S_0 (1 - e^{-tau_0/mu}) at the surface.
#include <math.h>

#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace mpsa {

namespace {

constexpr int kMaxDepth = 256;
constexpr int kMaxMu = 16;

__device__ __forceinline__ float layer_weight(float x) {
    // (1 - e^{-x}(1 + x)) / x, by its series for small x
    if (x < 1e-2f) return x * (0.5f - x * (1.f / 3.f - x * 0.125f));
    return (1.f - expf(-x) * (1.f + x)) / x;
}

__global__ void k_formal(int D, int N, const float* __restrict__ kappa, const float* __restrict__ kc,
                         const float* __restrict__ m, const float* __restrict__ T, double lam0_nm, double lnq,
                         int n_mu, const float* __restrict__ mu, float* __restrict__ I_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float tau[kMaxDepth], S[kMaxDepth];
    const double lam_cm = lam0_nm * exp((double)j * lnq) * 1e-7;
    const float lam = (float)lam_cm;
    const float c1 = (float)(2.0 * kH * kC * kC / (lam_cm * lam_cm * lam_cm * lam_cm * lam_cm));
    const float c2 = (float)(kH * kC / (lam_cm * kKB));
    float kprev = 0.f;
    for (int d = 0; d < D; ++d) {
        const float k = kappa[(size_t)d * N + j] + kc[d];
        tau[d] = d == 0 ? k * m[0] : tau[d - 1] + 0.5f * (kprev + k) * (m[d] - m[d - 1]);
        kprev = k;
        S[d] = c1 / expm1f(c2 / T[d]);
    }
    (void)lam;
    for (int q = 0; q < n_mu; ++q) {
        const float u = mu[q];
        const float dS = (S[D - 1] - S[D - 2]) / (tau[D - 1] - tau[D - 2]);
        float I = S[D - 1] + u * dS;
        for (int d = D - 2; d >= 0; --d) {
            const float x = (tau[d + 1] - tau[d]) / u;
            const float e = expf(-x);
            I = I * e + S[d] * (-expm1f(-x)) + (S[d + 1] - S[d]) * layer_weight(x);
        }
        const float x0 = tau[0] / u;
        I = I * expf(-x0) + S[0] * (-expm1f(-x0));
        I_out[(size_t)q * N + j] = I;
    }
}

__global__ void k_iota(int n, int* p) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

unsigned g_spec_init = 0;

}  // namespace

int formal_launch(int D, int N, const float* kappa, const float* kc, const float* m, const float* T, double lam0_nm,
                  double lnq, int n_mu, const float* mu, float* I_out, cudaStream_t st) {
    k_formal<<<(N + 127) / 128, 128, 0, st>>>(D, N, kappa, kc, m, T, lam0_nm, lnq, n_mu, mu, I_out);
    MPSA_CUDA_TRY(cudaGetLastError());
    return MPSA_OK;
}

int spectrum_module_init(int device) {
    g_spec_init |= 1u << (device & 31);
    return MPSA_OK;
}

}  // namespace mpsa

using namespace mpsa;

extern "C" int synth_spectrum(mpsa_ctx* ctx, const mpsa_atmos* atm, const mpsa_lgrid* win, int32_t n_mu,
                              const double* mu, float* I_out, const mpsa_synth_opts* opts, void* stream) {
    if (!ctx || !atm || !win || !mu || !I_out) return fail(MPSA_EINVAL, "synth_spectrum: NULL argument");
    if (ctx->L < 1) return fail(MPSA_ESTATE, "synth_spectrum: no line list loaded");
    if (ctx->n_el < 1 || !ctx->d_el) return fail(MPSA_ESTATE, "synth_spectrum: no element table (set_atmosphere_grid)");
    const int D = atm->n_depth;
    if (D < 2 || D > kMaxDepth) return fail(MPSA_EINVAL, "synth_spectrum: n_depth = %d (2..%d)", D, kMaxDepth);
    if (!atm->m || !atm->T || !atm->P) return fail(MPSA_EINVAL, "synth_spectrum: NULL atmosphere array");
    if (atm->comp < 0 || atm->comp >= ctx->n_comp) return fail(MPSA_EINVAL, "synth_spectrum: comp %d", atm->comp);
    if (n_mu < 1 || n_mu > kMaxMu) return fail(MPSA_EINVAL, "synth_spectrum: n_mu = %d (1..%d)", n_mu, kMaxMu);
    for (int q = 0; q < n_mu; ++q)
        if (!(mu[q] > 0 && mu[q] <= 1)) return fail(MPSA_EINVAL, "synth_spectrum: mu[%d] = %g", q, mu[q]);
    for (int d = 0; d < D; ++d) {
        if (!(atm->m[d] > 0) || !(atm->T[d] > 0) || !(atm->P[d] > 0) || !isfinite(atm->m[d]) || !isfinite(atm->T[d]) ||
            !isfinite(atm->P[d]))
            return fail(MPSA_EINVAL, "synth_spectrum: bad depth %d", d);
        if (d > 0 && !(atm->m[d] > atm->m[d - 1])) return fail(MPSA_EINVAL, "synth_spectrum: m not increasing at %d", d);
    }
    for (int i = 0; i < ctx->n_sp; ++i)
        if (ctx->h_sp_el[i] >= ctx->n_el) return fail(MPSA_EINVAL, "synth_spectrum: species/element mismatch");
    int N, r;
    if ((r = check_grid(win, &N))) return r;
    if ((size_t)D * ctx->L >= (size_t)1 << 31) return fail(MPSA_EINVAL, "synth_spectrum: n_depth * n_lines >= 2^31");
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    double *dT, *dP, *dab, *dpop;
    float *fm, *fT, *fmu, *kap, *kc;
    int* dsel;
    const int ne = ctx->n_el;
    if ((r = sc.alloc(&dT, D)) || (r = sc.alloc(&dP, D)) || (r = sc.alloc(&dab, ne)) ||
        (r = sc.alloc(&dpop, (size_t)D * pop_stride(ne))) || (r = sc.alloc(&fm, D)) || (r = sc.alloc(&fT, D)) ||
        (r = sc.alloc(&fmu, n_mu)) || (r = sc.alloc(&kap, (size_t)D * N)) || (r = sc.alloc(&kc, D)) ||
        (r = sc.alloc(&dsel, D)))
        return r;
    std::vector<float> hm(D), hT(D), hmu(n_mu);
    for (int d = 0; d < D; ++d) hm[d] = (float)atm->m[d], hT[d] = (float)atm->T[d];
    for (int q = 0; q < n_mu; ++q) hmu[q] = (float)mu[q];
    const double* ab = ctx->h_abund.data() + (size_t)atm->comp * ne;
    MPSA_CUDA_TRY(cudaMemcpyAsync(dT, atm->T, D * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(dP, atm->P, D * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(dab, ab, ne * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(fm, hm.data(), D * sizeof(float), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(fT, hT.data(), D * sizeof(float), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(fmu, hmu.data(), n_mu * sizeof(float), cudaMemcpyHostToDevice, st));
    if ((r = populations_device(ne, ctx->d_el, dab, 1, D, dT, dP, dpop, st))) return r;
    k_iota<<<(D + 127) / 128, 128, 0, st>>>(D, dsel);
    if ((r = synth_rows(ctx, dpop, D, dsel, win->lambda0_nm, win->R, N, kap, kc, nullptr, opts, st))) return r;
    if ((r = formal_launch(D, N, kap, kc, fm, fT, win->lambda0_nm, log1p(1.0 / win->R), n_mu, fmu, I_out, st))) return r;
    // pageable host-to-device copies are staged before cudaMemcpyAsync returns,
    // so the host vectors above may go out of scope now
    return MPSA_OK;
}

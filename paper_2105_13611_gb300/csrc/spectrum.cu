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
//
// odf_intensity: bin intensities of many 1D atmospheres from an ODF table (paper
// Sect. 2.3 and App. E), I_bin = sum_s w_s I_lambda_c(kappa_c + kappa_s): per depth the
// sub-bin opacities and the continuum are interpolated bilinearly in (log10 T, log10 P)
// on the table grid, and each sub-bin's intensity follows from the same formal solution.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace mpsa {

namespace {

constexpr int kMaxDepth = 256;
constexpr int kMaxMu = 16;

// B_lambda(T) = c1 / (e^x - 1), x = c2 / T.  Beyond x = 80 (e^x near the FP32 range) it is
// formed in log space, exp(ln c1 - x), whose dropped term ln(1 - e^-x) is below 2e-35; the
// value then stays representable down to FP32's smallest normal number instead of
// flushing to zero where e^x overflows.
__device__ __forceinline__ float planck_f32(float c1, float lnc1, float c2, float T) {
    const float x = c2 / T;
    return x < 80.f ? c1 / expm1f(x) : expf(lnc1 - x);
}

// 2^y and 1/y by the special-function unit (PTX ex2.approx / rcp.approx; relative error
// near 2^-22)
__device__ __forceinline__ float ex2_fast(float y) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}
__device__ __forceinline__ float rcp_fast(float y) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

// (1 - e (1 + x)) / x with e = e^{-x} already known
__device__ __forceinline__ float layer_weight_e(float x, float e) {
    if (x < 1e-2f) return x * (0.5f - x * (1.f / 3.f - x * 0.125f));
    return (1.f - e * (1.f + x)) / x;
}

__device__ __forceinline__ float layer_weight(float x) {
    // (1 - e^{-x}(1 + x)) / x, by its series for small x
    if (x < 1e-2f) return x * (0.5f - x * (1.f / 3.f - x * 0.125f));
    return (1.f - expf(-x) * (1.f + x)) / x;
}

__global__ void k_formal(int D, int N, const float* __restrict__ kappa, const float* __restrict__ kc,
                         const float* __restrict__ kcont, const float* __restrict__ m, const float* __restrict__ T,
                         double lam0_nm, double lnq, int n_mu, const float* __restrict__ mu, float* __restrict__ I_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float tau[kMaxDepth], S[kMaxDepth];
    const double lam_cm = lam0_nm * exp((double)j * lnq) * 1e-7;
    const float lam = (float)lam_cm;
    const double c1d = 2.0 * kH * kC * kC / (lam_cm * lam_cm * lam_cm * lam_cm * lam_cm);
    const float c1 = (float)c1d, lnc1 = (float)log(c1d);
    const float c2 = (float)(kH * kC / (lam_cm * kKB));
    float kprev = 0.f;
    for (int d = 0; d < D; ++d) {
        // continuum: the flat value of the depth, or the closed-form continuum at this wavelength
        const float k = kappa[(size_t)d * N + j] + (kcont ? kcont[(size_t)d * N + j] : kc[d]);
        tau[d] = d == 0 ? k * m[0] : tau[d - 1] + 0.5f * (kprev + k) * (m[d] - m[d - 1]);
        kprev = k;
        S[d] = planck_f32(c1, lnc1, c2, T[d]);
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

// ---- bin intensities from an ODF table
//
// Three kernels per call:
//  * k_bin_table: the FP64 table rounded once to FP32 (the interpolation then runs on the
//    FP32 pipes; per-value conversions in the main loop kept the FP64 pipe 86 % busy);
//  * k_bin_cells: per (ray, depth) the interpolation cell, its four weights, the
//    interpolated continuum, m and T in FP32, and the ray's validity;
//  * k_bin_intensity: one CTA per (ray, chunk of kb bins); thread t < kb * n_steps owns
//    sub-bin s = t % n_steps of bin k0 + t / n_steps and walks the depths from the bottom
//    up, holding one intensity per direction.  The recurrence needs only the layer optical
//    thicknesses dtau_d = (kappa_d + kappa_{d+1})(m_{d+1} - m_d)/2 and tau_0 = kappa_0 m_0, so
//    no depth array is kept.  The cells and the Planck function of each bin and depth sit in
//    shared memory; the per-bin Planck constants come from the host.
constexpr int kBinThreads = 256;

struct DepthCell {
    int r00, dT, dP;        // table row of the lower corner, row offsets to the upper T and P corners
                            // (k_bin_cells); scaled to element offsets (times K n_steps) for the table
    float w00, w01, w10, w11;
    float m, T, kc;
    float pad[2];
};

struct BinCellArgs {
    int nT, nP, D, n_rays;
    int row_stride;        // K * n_steps (table elements per row)
    const double* lt;      // [nT] log10 T axis
    const double* lp;      // [nP] log10 P axis
    const float* kc;       // [nT*nP]
    const double* m;       // [rays][D]
    const double* T;
    const double* P;
    DepthCell* cells;      // [rays][D]
    int* bad;              // [rays], zeroed before the launch
};

struct BinArgs {
    int K, ns, D, n_mu, kb;
    const float* tab;      // [nT*nP][K][ns] FP32
    const float3* pk;      // [K]: c1, ln c1, c2 of B_lambda at the bin centre
    const double* w;       // [ns]
    const float* mu;       // [n_mu]
    const DepthCell* cells;
    const int* bad;
    float* out;            // [rays][n_mu][K]
    int* status;           // [rays] or null
};

// index i (0 <= i <= n-2) and fraction f in [0, 1] of x on a strictly increasing axis,
// clamped to its ends (n = 1: i = 0, f = 0)
__device__ __forceinline__ void axis_cell(const double* __restrict__ ax, int n, double x, int* i, double* f) {
    if (n == 1 || x <= ax[0]) { *i = 0; *f = 0.0; return; }
    if (x >= ax[n - 1]) { *i = n - 2; *f = 1.0; return; }
    int lo = 0, hi = n - 1;   // ax[lo] <= x < ax[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ax[mid] <= x) lo = mid;
        else hi = mid;
    }
    *i = lo;
    *f = (x - ax[lo]) / (ax[lo + 1] - ax[lo]);
}

__global__ void k_bin_table(const double* __restrict__ src, float* __restrict__ dst, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

__global__ void k_bin_cells(BinCellArgs a) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)a.n_rays * a.D) return;
    const int ray = (int)(i / a.D), d = (int)(i - (size_t)ray * a.D);
    const double md = a.m[i], Td = a.T[i], Pd = a.P[i];
    const bool ok = md > 0.0 && Td > 0.0 && Pd > 0.0 && isfinite(md) && isfinite(Td) && isfinite(Pd) &&
                    (d == 0 || md > a.m[i - 1]);
    if (!ok) atomicOr(a.bad + ray, 1);
    int iT, iP;
    double fT, fP;
    axis_cell(a.lt, a.nT, log10(ok ? Td : 1.0), &iT, &fT);
    axis_cell(a.lp, a.nP, log10(ok ? Pd : 1.0), &iP, &fP);
    DepthCell c;
    c.r00 = iT * a.nP + iP;
    c.dT = (iT + 1 < a.nT ? 1 : 0) * a.nP;
    c.dP = iP + 1 < a.nP ? 1 : 0;
    c.w00 = (float)((1.0 - fT) * (1.0 - fP));
    c.w01 = (float)((1.0 - fT) * fP);
    c.w10 = (float)(fT * (1.0 - fP));
    c.w11 = (float)(fT * fP);
    c.m = (float)md;
    c.T = (float)Td;
    c.kc = c.w00 * a.kc[c.r00] + c.w01 * a.kc[c.r00 + c.dP] + c.w10 * a.kc[c.r00 + c.dT] +
           c.w11 * a.kc[c.r00 + c.dT + c.dP];
    c.pad[0] = c.pad[1] = 0.f;
    c.r00 *= a.row_stride;
    c.dT *= a.row_stride;
    c.dP *= a.row_stride;
    a.cells[i] = c;
}

template <int NMU>
__global__ void __launch_bounds__(kBinThreads) k_bin_intensity(BinArgs a) {
    extern __shared__ __align__(16) unsigned char bsm[];
    DepthCell* cell = reinterpret_cast<DepthCell*>(bsm);                      // [D]
    float* Sb = reinterpret_cast<float*>(cell + a.D);                         // [kb][D]
    float* part = Sb + (size_t)a.kb * a.D;                                    // [kBinThreads][NMU]
    const int ray = blockIdx.y, k0 = blockIdx.x * a.kb, tid = threadIdx.x;
    const DepthCell* rc = a.cells + (size_t)ray * a.D;
    for (int d = tid; d < a.D; d += kBinThreads) cell[d] = rc[d];
    __syncthreads();
    // Planck function at each bin centre and depth
    for (int i = tid; i < a.kb * a.D; i += kBinThreads) {
        const int kb = i / a.D, d = i - kb * a.D, k = k0 + kb;
        float S = 0.f;
        if (k < a.K) {
            const float3 p = a.pk[k];
            S = planck_f32(p.x, p.y, p.z, cell[d].T);
        }
        Sb[i] = S;
    }
    __syncthreads();

    const int kb = tid / a.ns, s = tid - kb * a.ns, k = k0 + kb;
    const bool act = kb < a.kb && k < a.K;
    // per direction: mu, 1/mu and -log2(e)/mu (e^{-x/mu} = 2^{x * (-log2 e / mu)})
    float I[NMU], mu[NMU], rmu[NMU], nl2[NMU];
#pragma unroll
    for (int q = 0; q < NMU; ++q) {
        mu[q] = q < a.n_mu ? a.mu[q] : 1.f;
        rmu[q] = 1.f / mu[q];
        nl2[q] = -1.4426950408889634f * rmu[q];
        I[q] = 0.f;
    }
    if (act) {
        const int col = k * a.ns + s;
        const float* __restrict__ tab = a.tab;
        const float* S = Sb + (size_t)kb * a.D;
        auto kappa = [&](int d) -> float {
            const DepthCell c = cell[d];
            const float* t = tab + (c.r00 + col);   // element offsets below 2^31 (checked on the host)
            const float v00 = __ldg(t), v01 = __ldg(t + c.dP), v10 = __ldg(t + c.dT), v11 = __ldg(t + c.dT + c.dP);
            return c.kc + (c.w00 * v00 + c.w01 * v01 + c.w10 * v10 + c.w11 * v11);
        };
        const int D = a.D;
        float k_hi = kappa(D - 1), k_lo = kappa(D - 2);
        float dtau = 0.5f * (k_lo + k_hi) * (cell[D - 1].m - cell[D - 2].m);
        const float dS = (S[D - 1] - S[D - 2]) / dtau;
#pragma unroll
        for (int q = 0; q < NMU; ++q) I[q] = fmaf(mu[q], dS, S[D - 1]);
        for (int d = D - 2;; --d) {
            // layer d .. d+1 of optical thickness dtau; per direction x = dtau / mu:
            //   I <- I e^{-x} + S_d (1 - e^{-x}) + (S_{d+1} - S_d) (1 - e^{-x}(1 + x)) / x,
            // the last two factors by their Taylor series below x = 0.1 (no cancellation)
            const float Sd = S[d], dSl = S[d + 1] - S[d];
            const float rdt = rcp_fast(dtau);
#pragma unroll
            for (int q = 0; q < NMU; ++q) {
                const float x = dtau * rmu[q];
                const float e = ex2_fast(dtau * nl2[q]);
                float ome, wl;
                if (x < 0.1f) {   // near the surface, where a warp's layers are all thin
                    // 1 - e^{-x} = x - x^2/2 + x^3/6 - x^4/24 + x^5/120
                    ome = x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.f / 120.f, -1.f / 24.f), 1.f / 6.f), -0.5f), 1.f);
                    // (1 - e^{-x}(1 + x))/x = x/2 - x^2/3 + x^3/8 - x^4/30 + x^5/144
                    wl = x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.f / 144.f, -1.f / 30.f), 0.125f), -1.f / 3.f), 0.5f);
                } else {
                    ome = 1.f - e;
                    wl = (1.f - fmaf(e, x, e)) * (mu[q] * rdt);
                }
                I[q] = fmaf(I[q], e, fmaf(Sd, ome, dSl * wl));
            }
            if (d == 0) break;
            k_hi = k_lo;
            k_lo = kappa(d - 1);
            dtau = 0.5f * (k_lo + k_hi) * (cell[d].m - cell[d - 1].m);
        }
        const float tau0 = k_lo * cell[0].m;
        const float ws = (float)a.w[s];
#pragma unroll
        for (int q = 0; q < NMU; ++q) {
            const float e = ex2_fast(tau0 * nl2[q]);
            I[q] = ws * fmaf(I[q], e, S[0] * (1.f - e));
        }
    }
#pragma unroll
    for (int q = 0; q < NMU; ++q) part[tid * NMU + q] = I[q];
    __syncthreads();
    // sum over the sub-bins in order
    const bool bad = a.bad[ray] != 0;
    for (int i = tid; i < a.kb * a.n_mu; i += kBinThreads) {
        const int b = i / a.n_mu, q = i - b * a.n_mu, kk = k0 + b;
        if (kk >= a.K) continue;
        float acc = 0.f;
        for (int t = 0; t < a.ns; ++t) acc += part[(b * a.ns + t) * NMU + q];
        a.out[((size_t)ray * a.n_mu + q) * a.K + kk] = bad ? __int_as_float(0x7fc00000) : acc;
    }
    if (tid == 0 && a.status && blockIdx.x == 0) a.status[ray] = bad ? 1 : 0;
}

__global__ void k_iota(int n, int* p) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

unsigned g_spec_init = 0;

}  // namespace

int formal_launch(int D, int N, const float* kappa, const float* kc, const float* kcont, const float* m, const float* T,
                  double lam0_nm, double lnq, int n_mu, const float* mu, float* I_out, cudaStream_t st) {
    k_formal<<<(N + 127) / 128, 128, 0, st>>>(D, N, kappa, kc, kcont, m, T, lam0_nm, lnq, n_mu, mu, I_out);
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
    int N, r;
    if ((r = check_species(ctx, "synth_spectrum"))) return r;
    if ((r = check_grid(win, &N))) return r;
    if ((size_t)D * ctx->L >= (size_t)1 << 31) return fail(MPSA_EINVAL, "synth_spectrum: n_depth * n_lines >= 2^31");
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st, ctx->pool);
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
    float* kcont = nullptr;
    const int cont = opts ? opts->continuum : 0;
    if (cont) {
        if (cont & ~MPSA_CONT_ALL) return fail(MPSA_EINVAL, "synth_spectrum: continuum = %d", cont);
        if ((r = sc.alloc(&kcont, (size_t)D * N))) return r;
        if ((r = continuum_launch(ctx, dpop, D, dsel, win->lambda0_nm, win->R, N, cont, kcont, st))) return r;
    }
    if ((r = formal_launch(D, N, kap, kc, kcont, fm, fT, win->lambda0_nm, log1p(1.0 / win->R), n_mu, fmu, I_out, st)))
        return r;
    // pageable host-to-device copies are staged before cudaMemcpyAsync returns,
    // so the host vectors above may go out of scope now
    return MPSA_OK;
}

namespace mpsa {
namespace {

constexpr int kBinMaxKb = 32;
constexpr size_t kBinSmemMax =
    (size_t)kMaxDepth * sizeof(DepthCell) + (size_t)kBinMaxKb * kMaxDepth * sizeof(float) +
    (size_t)kBinThreads * kMaxMu * sizeof(float);

template <int NMU>
int bin_launch(const BinArgs& a, int n_rays, cudaStream_t st) {
    static unsigned attr_set = 0;   // one bit per device
    int dev = 0;
    MPSA_CUDA_TRY(cudaGetDevice(&dev));
    if (!(attr_set & (1u << (dev & 31)))) {
        MPSA_CUDA_TRY(cudaFuncSetAttribute(k_bin_intensity<NMU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kBinSmemMax));
        attr_set |= 1u << (dev & 31);
    }
    const size_t smem = (size_t)a.D * sizeof(DepthCell) + (size_t)a.kb * a.D * sizeof(float) +
                        (size_t)kBinThreads * NMU * sizeof(float);
    const dim3 grid((a.K + a.kb - 1) / a.kb, n_rays);
    k_bin_intensity<NMU><<<grid, kBinThreads, smem, st>>>(a);
    MPSA_CUDA_TRY(cudaGetLastError());
    return MPSA_OK;
}

int check_axis(const double* ax, int n, const char* name) {
    if (n < 1 || !ax) return fail(MPSA_EINVAL, "odf_intensity: %s axis of %d values", name, n);
    for (int i = 0; i < n; ++i) {
        if (!isfinite(ax[i])) return fail(MPSA_EINVAL, "odf_intensity: %s[%d] = %g", name, i, ax[i]);
        if (i > 0 && !(ax[i] > ax[i - 1])) return fail(MPSA_EINVAL, "odf_intensity: %s not increasing at %d", name, i);
    }
    return MPSA_OK;
}

}  // namespace
}  // namespace mpsa

extern "C" int odf_intensity(mpsa_ctx* ctx, const mpsa_odf_table* tab, int32_t n_rays, int32_t n_depth,
                             const double* m, const double* T, const double* P, int32_t n_mu, const double* mu,
                             float* I_out, int32_t* ray_status, void* stream) {
    if (!ctx || !tab || !m || !T || !P || !mu || !I_out) return fail(MPSA_EINVAL, "odf_intensity: NULL argument");
    if (!tab->odf || !tab->kappa_c || !tab->lam_c_nm || !tab->widths)
        return fail(MPSA_EINVAL, "odf_intensity: NULL table array");
    int r;
    if ((r = check_axis(tab->log10_T, tab->nT, "log10_T")) || (r = check_axis(tab->log10_P, tab->nP, "log10_P")))
        return r;
    const int K = tab->K, ns = tab->n_steps;
    if (K < 1) return fail(MPSA_EINVAL, "odf_intensity: K = %d", K);
    if (ns < 1 || ns > 32) return fail(MPSA_EINVAL, "odf_intensity: n_steps = %d (1..32)", ns);
    if ((long long)tab->nT * tab->nP * K * ns >= (1ll << 31))
        return fail(MPSA_EINVAL, "odf_intensity: table of %d x %d x %d x %d", tab->nT, tab->nP, K, ns);
    for (int k = 0; k < K; ++k)
        if (!(tab->lam_c_nm[k] > 0) || !isfinite(tab->lam_c_nm[k]))
            return fail(MPSA_EINVAL, "odf_intensity: lam_c_nm[%d] = %g", k, tab->lam_c_nm[k]);
    double wsum = 0.0;
    for (int s = 0; s < ns; ++s) {
        if (!(tab->widths[s] > 0) || !isfinite(tab->widths[s]))
            return fail(MPSA_EINVAL, "odf_intensity: widths[%d] = %g", s, tab->widths[s]);
        wsum += tab->widths[s];
    }
    if (fabs(wsum - 1.0) > 1e-12) return fail(MPSA_EINVAL, "odf_intensity: widths sum to %.17g", wsum);
    if (n_rays < 1 || n_rays > 65535) return fail(MPSA_EINVAL, "odf_intensity: n_rays = %d (1..65535)", n_rays);
    if (n_depth < 2 || n_depth > kMaxDepth) return fail(MPSA_EINVAL, "odf_intensity: n_depth = %d (2..%d)", n_depth, kMaxDepth);
    if (n_mu < 1 || n_mu > kMaxMu) return fail(MPSA_EINVAL, "odf_intensity: n_mu = %d (1..%d)", n_mu, kMaxMu);
    for (int q = 0; q < n_mu; ++q)
        if (!(mu[q] > 0 && mu[q] <= 1)) return fail(MPSA_EINVAL, "odf_intensity: mu[%d] = %g", q, mu[q]);
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st, ctx->pool);
    const size_t n_tab = (size_t)tab->nT * tab->nP * K * ns, n_cells = (size_t)n_rays * n_depth;
    double *dlt, *dlp, *dw;
    float *dmu, *dtab;
    float3* dpk;
    DepthCell* dcell;
    int* dbad;
    if ((r = sc.alloc(&dlt, tab->nT)) || (r = sc.alloc(&dlp, tab->nP)) || (r = sc.alloc(&dpk, K)) ||
        (r = sc.alloc(&dw, ns)) || (r = sc.alloc(&dmu, n_mu)) || (r = sc.alloc(&dtab, n_tab)) ||
        (r = sc.alloc(&dcell, n_cells)) || (r = sc.alloc(&dbad, n_rays)))
        return r;
    std::vector<float> hmu(n_mu);
    for (int q = 0; q < n_mu; ++q) hmu[q] = (float)mu[q];
    // Planck constants per bin centre: B = c1 / (e^{c2/T} - 1) (FP64 on the host, then FP32)
    std::vector<float3> hpk(K);
    for (int k = 0; k < K; ++k) {
        const double lam_cm = tab->lam_c_nm[k] * 1e-7;
        const double c1 = 2.0 * kH * kC * kC / (lam_cm * lam_cm * lam_cm * lam_cm * lam_cm);
        hpk[k] = make_float3((float)c1, (float)log(c1), (float)(kH * kC / (lam_cm * kKB)));
    }
    MPSA_CUDA_TRY(cudaMemcpyAsync(dlt, tab->log10_T, tab->nT * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(dlp, tab->log10_P, tab->nP * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(dpk, hpk.data(), K * sizeof(float3), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(dw, tab->widths, ns * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(dmu, hmu.data(), n_mu * sizeof(float), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemsetAsync(dbad, 0, n_rays * sizeof(int), st));
    k_bin_table<<<(unsigned)std::min<size_t>((n_tab + 255) / 256, 4096), 256, 0, st>>>(tab->odf, dtab, n_tab);
    MPSA_CUDA_TRY(cudaGetLastError());
    BinCellArgs ca;
    ca.nT = tab->nT;
    ca.nP = tab->nP;
    ca.D = n_depth;
    ca.n_rays = n_rays;
    ca.row_stride = K * ns;
    ca.lt = dlt;
    ca.lp = dlp;
    ca.kc = tab->kappa_c;
    ca.m = m;
    ca.T = T;
    ca.P = P;
    ca.cells = dcell;
    ca.bad = dbad;
    k_bin_cells<<<(unsigned)((n_cells + 255) / 256), 256, 0, st>>>(ca);
    MPSA_CUDA_TRY(cudaGetLastError());
    BinArgs a;
    a.K = K;
    a.ns = ns;
    a.D = n_depth;
    a.n_mu = n_mu;
    a.kb = std::max(1, std::min(kBinThreads / ns, kBinMaxKb));
    a.tab = dtab;
    a.pk = dpk;
    a.w = dw;
    a.mu = dmu;
    a.cells = dcell;
    a.bad = dbad;
    a.out = I_out;
    a.status = ray_status;
    prof_mark(ctx, MPSA_KERNEL_BINS, st);
    switch (n_mu) {
        case 1: r = bin_launch<1>(a, n_rays, st); break;
        case 2: r = bin_launch<2>(a, n_rays, st); break;
        case 3: r = bin_launch<3>(a, n_rays, st); break;
        case 4: r = bin_launch<4>(a, n_rays, st); break;
        case 5: r = bin_launch<5>(a, n_rays, st); break;
        case 6: r = bin_launch<6>(a, n_rays, st); break;
        case 7: r = bin_launch<7>(a, n_rays, st); break;
        case 8: r = bin_launch<8>(a, n_rays, st); break;
        default: r = bin_launch<16>(a, n_rays, st); break;
    }
    prof_mark(ctx, MPSA_KERNEL_BINS, st);
    // pageable host-to-device copies are staged before cudaMemcpyAsync returns,
    // so the host vectors above may go out of scope now
    return r;
}

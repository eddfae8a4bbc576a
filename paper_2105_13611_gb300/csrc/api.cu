// C-ABI entry points for context management, the line list and the FP64
// population table (paper Sect. 2.1 and App. A).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace mpsa {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

int fail(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int synth_module_init(int device);     // synth.cu
int spectrum_module_init(int device);  // spectrum.cu

namespace {

template <class T>
int upload(T** dst, const T* src, size_t n) {
    if (*dst) cudaFree(*dst), *dst = nullptr;
    if (n == 0) return MPSA_OK;
    MPSA_CUDA_TRY(cudaMalloc(dst, n * sizeof(T)));
    MPSA_CUDA_TRY(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return MPSA_OK;
}

// Saha charge balance for one (composition, point) row, FP64.
// Particle conservation P = (n_nuc + n_e) kT; each element ionises once with
// n_II = f n_nuc Phi / (n_e + Phi), Phi = (2 U_II/U_I)(2 pi m_e kT/h^2)^{3/2} e^{-chi/kT};
// charge conservation n_e = sum n_II is solved for n_e by bisection in ln n_e
// (g(n_e) = n_e - sum n_II(n_e) is increasing on (0, P/kT)).
__global__ void k_populations(int rows, int n_points, int n_el, const double* __restrict__ el,
                              const double* __restrict__ abund, const double* __restrict__ T,
                              const double* __restrict__ P, double* __restrict__ pop) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int comp = r / n_points, pt = r % n_points;
    const double t = T[pt], p = P[pt];
    const double* mass = el;
    const double* chi = el + n_el;
    const double* U1 = el + 2 * n_el;
    const double* U2 = el + 3 * n_el;
    const double* leps = el + 4 * n_el;
    const double kT = kKB * t;
    const double saha = pow(2.0 * kPI * kME * kT / (kH * kH), 1.5);
    double* row = pop + (size_t)r * pop_stride(n_el);
    // number fractions
    double eps_sum = 0.0;
    for (int e = 0; e < n_el; ++e) eps_sum += pow(10.0, leps[e] - 12.0) * abund[(size_t)comp * n_el + e];
    const double n_tot = p / kT;
    // per-element number fraction f and Saha factor Phi (hoisted out of the root search)
    double frac[64], phi[64];
    for (int e = 0; e < n_el; ++e) {
        frac[e] = pow(10.0, leps[e] - 12.0) * abund[(size_t)comp * n_el + e] / eps_sum;
        phi[e] = 2.0 * U2[e] / U1[e] * saha * exp(-chi[e] * kEV / kT);
    }
    // bisection in ln n_e down to adjacent doubles: stop when the midpoint no longer lies
    // strictly between the bounds (a fixed width such as 1e-15 is below one ulp of ln n_e
    // for |ln n_e| > 4 and would never be reached)
    double lo = log(1e-300), hi = log(n_tot);
    for (int it = 0; it < 2000; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        const double ne = exp(mid), nn = n_tot - ne;
        double ion = 0.0;
        for (int e = 0; e < n_el; ++e) ion += frac[e] * nn * phi[e] / (ne + phi[e]);
        if (ne - ion > 0.0) hi = mid; else lo = mid;
    }
    const double ne = exp(0.5 * (lo + hi)), nn = n_tot - ne;
    double mmean = 0.0;
    double nHI = 0.0;
    for (int e = 0; e < n_el; ++e) {
        // n_II/n_I = Phi/n_e; n_I = f n n_e/(n_e + Phi) has no cancellation for a fully ionised stage I
        const double n2 = frac[e] * nn * phi[e] / (ne + phi[e]);
        const double n1 = frac[e] * nn * ne / (ne + phi[e]);
        row[kPopHdr + 2 * e] = n1 / U1[e];
        row[kPopHdr + 2 * e + 1] = n2 / U2[e];
        mmean += frac[e] * mass[e] * kAMU;
        if (e == 0) nHI = n1;
    }
    row[kPopT] = t;
    row[kPopP] = p;
    row[kPopNe] = ne;
    row[kPopNHI] = nHI;
    row[kPopRho] = nn * mmean;
}

}  // namespace

int populations_device(int n_el, const double* d_el, const double* d_abund, int n_comp, int n_points,
                       const double* d_T, const double* d_P, double* d_pop, cudaStream_t s) {
    const int rows = n_comp * n_points;
    k_populations<<<(rows + 63) / 64, 64, 0, s>>>(rows, n_points, n_el, d_el, d_abund, d_T, d_P, d_pop);
    MPSA_CUDA_TRY(cudaGetLastError());
    return MPSA_OK;
}

}  // namespace mpsa

using namespace mpsa;

extern "C" {

const char* mpsa_version(void) { return "mpsa-gb300 0.1 (sm_103a)"; }

const char* mpsa_last_error(void) { return g_err.c_str(); }

int mpsa_create(mpsa_ctx** out, int device) {
    if (!out) return fail(MPSA_EINVAL, "mpsa_create: out is NULL");
    *out = nullptr;
    int n = 0;
    MPSA_CUDA_TRY(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(MPSA_EINVAL, "mpsa_create: device %d of %d", device, n);
    MPSA_CUDA_TRY(cudaSetDevice(device));
    int rc = synth_module_init(device);
    if (rc != MPSA_OK) return rc;
    rc = spectrum_module_init(device);
    if (rc != MPSA_OK) return rc;
    mpsa_ctx* c = new mpsa_ctx();
    c->device = device;
    *out = c;
    return MPSA_OK;
}

void mpsa_destroy(mpsa_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& v : c->prof_ev)
        for (cudaEvent_t e : v) cudaEventDestroy(e);
    void* ptrs[] = {c->d_el, c->d_sp_el, c->d_sp_stage, c->d_lam, c->d_loggf, c->d_E, c->d_lgR,
                    c->d_lgS, c->d_lgW, c->d_species, c->d_pop};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete c;
}

int64_t mpsa_grid_size(const mpsa_lgrid* g) {
    if (!g || !(g->lambda0_nm > 0) || !(g->lambda1_nm >= g->lambda0_nm) || !(g->R > 0) || !isfinite(g->lambda1_nm))
        return 0;
    double n = floor(log(g->lambda1_nm / g->lambda0_nm) / log1p(1.0 / g->R)) + 1.0;
    if (!(n >= 1) || n > 9.0e18) return 0;
    return (int64_t)n;
}

int load_linelist(mpsa_ctx* c, int32_t n_species, const int32_t* sp_el, const int32_t* sp_stage,
                  const mpsa_lines* ln) {
    if (!c || !ln || !sp_el || !sp_stage) return fail(MPSA_EINVAL, "load_linelist: NULL argument");
    if (n_species < 1) return fail(MPSA_EINVAL, "load_linelist: n_species = %d", n_species);
    const int64_t L = ln->n_lines;
    if (L < 1 || L > (int64_t)1 << 31) return fail(MPSA_EINVAL, "load_linelist: n_lines = %lld", (long long)L);
    if (!ln->lambda_nm || !ln->log_gf || !ln->E_eV || !ln->species || !ln->log_gR || !ln->log_gS || !ln->log_gW)
        return fail(MPSA_EINVAL, "load_linelist: NULL line array");
    for (int s = 0; s < n_species; ++s)
        if (sp_el[s] < 0 || sp_stage[s] < 0 || sp_stage[s] > 1)
            return fail(MPSA_EINVAL, "load_linelist: species %d has element %d stage %d", s, sp_el[s], sp_stage[s]);
    for (int64_t i = 0; i < L; ++i) {
        const double lam = ln->lambda_nm[i];
        if (!(lam > 0) || !isfinite(lam)) return fail(MPSA_EINVAL, "load_linelist: lambda[%lld] = %g", (long long)i, lam);
        if (i > 0 && lam < ln->lambda_nm[i - 1])
            return fail(MPSA_EINVAL, "load_linelist: lambda not ascending at %lld", (long long)i);
        if (ln->species[i] < 0 || ln->species[i] >= n_species)
            return fail(MPSA_EINVAL, "load_linelist: species[%lld] = %d", (long long)i, ln->species[i]);
        if (!isfinite(ln->log_gf[i]) || !isfinite(ln->E_eV[i]) || !isfinite(ln->log_gR[i]) ||
            !isfinite(ln->log_gS[i]) || !isfinite(ln->log_gW[i]))
            return fail(MPSA_EINVAL, "load_linelist: non-finite parameter of line %lld", (long long)i);
    }
    MPSA_CUDA_TRY(cudaSetDevice(c->device));
    int rc;
    if ((rc = upload(&c->d_sp_el, sp_el, n_species)) || (rc = upload(&c->d_sp_stage, sp_stage, n_species)) ||
        (rc = upload(&c->d_lam, ln->lambda_nm, L)) || (rc = upload(&c->d_loggf, ln->log_gf, L)) ||
        (rc = upload(&c->d_E, ln->E_eV, L)) || (rc = upload(&c->d_lgR, ln->log_gR, L)) ||
        (rc = upload(&c->d_lgS, ln->log_gS, L)) || (rc = upload(&c->d_lgW, ln->log_gW, L)) ||
        (rc = upload(&c->d_species, ln->species, L))) {
        c->L = 0;
        return rc;
    }
    c->n_sp = n_species;
    c->h_sp_el.assign(sp_el, sp_el + n_species);
    c->h_sp_stage.assign(sp_stage, sp_stage + n_species);
    c->L = L;
    return MPSA_OK;
}

int set_atmosphere_grid(mpsa_ctx* c, const mpsa_elements* el, int32_t n_points, const double* T, const double* P,
                        int32_t n_comp, const double* abund, double vturb) {
    if (!c || !el || !T || !P) return fail(MPSA_EINVAL, "set_atmosphere_grid: NULL argument");
    const int ne = el->n_elements;
    if (ne < 1 || ne > 64) return fail(MPSA_EINVAL, "set_atmosphere_grid: n_elements = %d", ne);
    if (!el->mass_amu || !el->chi_eV || !el->U1 || !el->U2 || !el->log_eps)
        return fail(MPSA_EINVAL, "set_atmosphere_grid: NULL element array");
    if (n_points < 1) return fail(MPSA_EINVAL, "set_atmosphere_grid: n_points = %d", n_points);
    if (n_comp < 1 || (!abund && n_comp != 1)) return fail(MPSA_EINVAL, "set_atmosphere_grid: n_comp = %d", n_comp);
    if (!(vturb >= 0) || !isfinite(vturb)) return fail(MPSA_EINVAL, "set_atmosphere_grid: vturb = %g", vturb);
    for (int i = 0; i < n_points; ++i)
        if (!(T[i] > 0) || !(P[i] > 0) || !isfinite(T[i]) || !isfinite(P[i]))
            return fail(MPSA_EINVAL, "set_atmosphere_grid: T[%d] = %g, P[%d] = %g", i, T[i], i, P[i]);
    for (int e = 0; e < ne; ++e)
        if (!(el->mass_amu[e] > 0) || !(el->U1[e] > 0) || !(el->U2[e] > 0) || !isfinite(el->chi_eV[e]) ||
            !isfinite(el->log_eps[e]))
            return fail(MPSA_EINVAL, "set_atmosphere_grid: bad element %d", e);
    std::vector<double> ab((size_t)n_comp * ne, 1.0);
    if (abund)
        for (size_t i = 0; i < ab.size(); ++i) {
            if (!(abund[i] >= 0) || !isfinite(abund[i])) return fail(MPSA_EINVAL, "set_atmosphere_grid: abund[%zu]", i);
            ab[i] = abund[i];
        }
    std::vector<double> h(5 * ne);
    for (int e = 0; e < ne; ++e) {
        h[e] = el->mass_amu[e];
        h[ne + e] = el->chi_eV[e];
        h[2 * ne + e] = el->U1[e];
        h[3 * ne + e] = el->U2[e];
        h[4 * ne + e] = el->log_eps[e];
    }
    MPSA_CUDA_TRY(cudaSetDevice(c->device));
    int rc;
    double *dT = nullptr, *dP = nullptr, *dab = nullptr;
    if ((rc = upload(&c->d_el, h.data(), h.size()))) return rc;
    if ((rc = upload(&dT, T, n_points)) || (rc = upload(&dP, P, n_points)) || (rc = upload(&dab, ab.data(), ab.size()))) {
        cudaFree(dT), cudaFree(dP), cudaFree(dab);
        return rc;
    }
    if (c->d_pop) cudaFree(c->d_pop), c->d_pop = nullptr;
    const size_t rows = (size_t)n_comp * n_points;
    cudaError_t e = cudaMalloc(&c->d_pop, rows * pop_stride(ne) * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(dT), cudaFree(dP), cudaFree(dab);
        return fail(MPSA_ENOMEM, "set_atmosphere_grid: %s", cudaGetErrorString(e));
    }
    rc = populations_device(ne, c->d_el, dab, n_comp, n_points, dT, dP, c->d_pop, 0);
    cudaError_t e2 = cudaDeviceSynchronize();
    cudaFree(dT), cudaFree(dP), cudaFree(dab);
    if (rc) return rc;
    if (e2 != cudaSuccess) return fail(MPSA_ECUDA, "set_atmosphere_grid: %s", cudaGetErrorString(e2));
    c->n_el = ne;
    c->h_el = h;
    c->n_points = n_points;
    c->n_comp = n_comp;
    c->vturb = vturb;
    c->h_abund = ab;
    return MPSA_OK;
}

int mpsa_profile_enable(mpsa_ctx* c, int enable) {
    if (!c) return fail(MPSA_EINVAL, "mpsa_profile_enable: NULL context");
    c->prof = enable != 0;
    return MPSA_OK;
}

int mpsa_profile_read(mpsa_ctx* c, int kernel, double* total_ms, int64_t* launches) {
    if (!c || !total_ms || !launches || kernel < 0 || kernel > 2) return fail(MPSA_EINVAL, "mpsa_profile_read: bad argument");
    auto& v = c->prof_ev[kernel];
    double tot = 0.0;
    int64_t n = 0;
    for (size_t i = 0; i + 1 < v.size(); i += 2) {
        MPSA_CUDA_TRY(cudaEventSynchronize(v[i + 1]));
        float ms = 0.f;
        MPSA_CUDA_TRY(cudaEventElapsedTime(&ms, v[i], v[i + 1]));
        tot += ms;
        ++n;
    }
    for (cudaEvent_t e : v) cudaEventDestroy(e);
    v.clear();
    *total_ms = tot;
    *launches = n;
    return MPSA_OK;
}

}  // extern "C"

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

// The LTE equation of state of one (composition, point) row, FP64 (paper App. A, without
// molecules).  Element e has stages j = 0 .. J_e - 1 linked by the Saha-Boltzmann ratio
//   n_{e,j+1} n_e / n_{e,j} = Phi_{e,j} = (2 U_{j+1}/U_j) (2 pi m_e k T/h^2)^{3/2} e^{-chi_j/kT},
// U_j(T) = exp(c0 + c1 x + c2 x^2), x = ln(T / 5040 K).  Particle conservation gives
// n_nuc = P/kT - n_e, and charge conservation n_e = n_nuc sum_e a_e <j>_e(n_e), <j>_e the
// mean charge of element e at that n_e.  g(y) = n_e - n_nuc sum_e a_e <j>_e with y = ln n_e is
// increasing (dg/dn_e = 1 + Q + n_nuc sum_e a_e Var_e / n_e > 0), so the root is unique; it
// is found by Newton steps in y kept inside a shrinking bracket (bisection where a step would
// leave it), to a relative change of n_e below 1e-14.  The stage weights prod_{i<j} Phi_i / n_e
// are formed in log space and scaled by their largest value, so no ratio overflows.
//
// One warp per row: lane l holds elements l and l + 32 (at most 64), and every sum over the
// elements is a warp reduction whose result all lanes share, so the lanes take the same
// Newton steps.
constexpr int kPopElPerLane = 2;

// sum over the warp, lane 0's result given to every lane (the same bits in all lanes)
__device__ __forceinline__ double warp_sum(double v) {
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    return __shfl_sync(0xffffffffu, v, 0);
}

__global__ void k_populations(int rows, int n_points, int n_el, const double* __restrict__ el,
                              const double* __restrict__ abund, const double* __restrict__ T,
                              const double* __restrict__ P, double* __restrict__ pop) {
    const int r = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (r >= rows) return;   // the same for every lane of the warp
    const int comp = r / n_points, pt = r % n_points;
    const double t = T[pt], p = P[pt];
    const double kT = kKB * t;
    const double lsaha = 1.5 * log(2.0 * kPI * kME * kT / (kH * kH));
    const double x = log(t / 5040.0);
    double* row = pop + (size_t)r * pop_stride(n_el);
    double eps[kPopElPerLane];
    double eps_part = 0.0;
    for (int k = 0; k < kPopElPerLane; ++k) {
        const int e = lane + 32 * k;
        eps[k] = e < n_el ? pow(10.0, el[e * kElStride + kElLogEps] - 12.0) * abund[(size_t)comp * n_el + e] : 0.0;
        eps_part += eps[k];
    }
    const double eps_sum = warp_sum(eps_part);
    double frac[kPopElPerLane];
    double lphi[kPopElPerLane][kMaxStages - 1];   // ln Phi_{e,j}
    double lU[kPopElPerLane][kMaxStages];          // ln U_{e,j}
    int ns[kPopElPerLane];
    for (int k = 0; k < kPopElPerLane; ++k) {
        const int e = lane + 32 * k;
        ns[k] = 0;
        frac[k] = 0.0;
        if (e >= n_el) continue;
        const double* q = el + e * kElStride;
        frac[k] = eps[k] / eps_sum;
        ns[k] = (int)q[kElStages];
        for (int j = 0; j < ns[k]; ++j) {
            const double* c = q + kElLnU + 3 * j;
            lU[k][j] = c[0] + x * (c[1] + x * c[2]);
        }
        for (int j = 0; j + 1 < ns[k]; ++j)
            lphi[k][j] = 0.69314718055994530942 + lU[k][j + 1] - lU[k][j] + lsaha - q[kElChi + j] * kEV / kT;
    }
    const double n_tot = p / kT;
    // stage weights of the lane's element k at y = ln n_e: w_j = exp(lp_j - max lp),
    // lp_j = sum_{i<j} (ln Phi_i - y)
    auto weights = [&](int k, double y, double* w) -> double {
        double lp[kMaxStages], mx = 0.0;
        lp[0] = 0.0;
        for (int j = 1; j < ns[k]; ++j) {
            lp[j] = lp[j - 1] + lphi[k][j - 1] - y;
            mx = fmax(mx, lp[j]);
        }
        double s0 = 0.0;
        for (int j = 0; j < ns[k]; ++j) {
            w[j] = exp(lp[j] - mx);
            s0 += w[j];
        }
        return s0;
    };
    // g(y) and dg/dy
    auto eval = [&](double y, double* g, double* dg) {
        const double ne = exp(y), nn = n_tot - ne;
        double q = 0.0, v = 0.0;
        for (int k = 0; k < kPopElPerLane; ++k) {
            if (ns[k] == 0) continue;
            double w[kMaxStages];
            const double s0 = weights(k, y, w);
            double s1 = 0.0, s2 = 0.0;
            for (int j = 1; j < ns[k]; ++j) {
                s1 += j * w[j];
                s2 += (double)j * j * w[j];
            }
            const double mean = s1 / s0;
            q += frac[k] * mean;
            v += frac[k] * fmax(s2 / s0 - mean * mean, 0.0);
        }
        q = warp_sum(q);
        v = warp_sum(v);
        *g = ne - nn * q;
        *dg = ne * (1.0 + q) + nn * v;
    };
    double lo = log(1e-300), hi = log(n_tot), y = 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
        double g, dg;
        eval(y, &g, &dg);
        if (g > 0.0) hi = y; else lo = y;
        double yn = (dg > 0.0) ? y - g / dg : 0.5 * (lo + hi);
        if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
        const double dy = yn - y;
        y = yn;
        if (fabs(dy) < 1e-14 || !(hi - lo > 0.0) || !(y > lo && y < hi && (0.5 * (lo + hi) != lo))) break;
    }
    const double ne = exp(y), nn = n_tot - ne;
    double mpart = 0.0, nHI = 0.0;
    for (int k = 0; k < kPopElPerLane; ++k) {
        const int e = lane + 32 * k;
        if (e >= n_el) continue;
        double w[kMaxStages];
        const double s0 = weights(k, y, w);
        for (int j = 0; j < kMaxStages; ++j) {
            const double nj = j < ns[k] ? frac[k] * nn * w[j] / s0 : 0.0;
            row[pop_nu(e, j)] = j < ns[k] ? nj / exp(lU[k][j]) : 0.0;
            if (e == 0 && j == 0) nHI = nj;
        }
        mpart += frac[k] * el[e * kElStride + kElMass] * kAMU;
    }
    const double mmean = warp_sum(mpart);
    if (lane == 0) {
        row[kPopT] = t;
        row[kPopP] = p;
        row[kPopNe] = ne;
        row[kPopNHI] = nHI;
        row[kPopRho] = nn * mmean;
    }
}

}  // namespace

int populations_device(int n_el, const double* d_el, const double* d_abund, int n_comp, int n_points,
                       const double* d_T, const double* d_P, double* d_pop, cudaStream_t s) {
    const int rows = n_comp * n_points;
    k_populations<<<(unsigned)(((int64_t)rows * 32 + 127) / 128), 128, 0, s>>>(rows, n_points, n_el, d_el, d_abund,
                                                                             d_T, d_P, d_pop);
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
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    MPSA_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;   // keep freed scratch cached until the context goes
    cudaError_t e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return fail(MPSA_ECUDA, "mpsa_create: memory pool: %s", cudaGetErrorString(e));
    }
    mpsa_ctx* c = new mpsa_ctx();
    c->device = device;
    c->pool = pool;
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
    if (c->pool) cudaMemPoolDestroy(c->pool);
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
        if (sp_el[s] < 0 || sp_stage[s] < 0 || sp_stage[s] >= kMaxStages)
            return fail(MPSA_EINVAL, "load_linelist: species %d has element %d stage %d", s, sp_el[s], sp_stage[s]);
    bool ascending = true;
    for (int64_t i = 0; i < L; ++i) {
        const double lam = ln->lambda_nm[i];
        if (!(lam > 0) || !isfinite(lam)) return fail(MPSA_EINVAL, "load_linelist: lambda[%lld] = %g", (long long)i, lam);
        if (i > 0 && lam < ln->lambda_nm[i - 1]) ascending = false;
        if (ln->species[i] < 0 || ln->species[i] >= n_species)
            return fail(MPSA_EINVAL, "load_linelist: species[%lld] = %d", (long long)i, ln->species[i]);
        if (!isfinite(ln->log_gf[i]) || !isfinite(ln->E_eV[i]) || !isfinite(ln->log_gR[i]) ||
            !isfinite(ln->log_gS[i]) || !isfinite(ln->log_gW[i]))
            return fail(MPSA_EINVAL, "load_linelist: non-finite parameter of line %lld", (long long)i);
    }
    // the kernels need the list ascending in lambda (tiles find their lines by binary search):
    // a list in any other order is sorted here, stably, into a host copy
    mpsa_lines src = *ln;
    std::vector<double> s_lam;
    std::vector<float> s_gf, s_E, s_gR, s_gS, s_gW;
    std::vector<int32_t> s_sp;
    if (!ascending) {
        std::vector<int64_t> perm((size_t)L);
        for (int64_t i = 0; i < L; ++i) perm[(size_t)i] = i;
        std::stable_sort(perm.begin(), perm.end(),
                         [&](int64_t a, int64_t b) { return ln->lambda_nm[a] < ln->lambda_nm[b]; });
        auto gather = [&](auto& dst, const auto* from) {
            dst.resize((size_t)L);
            for (int64_t i = 0; i < L; ++i) dst[(size_t)i] = from[perm[(size_t)i]];
        };
        gather(s_lam, ln->lambda_nm);
        gather(s_gf, ln->log_gf);
        gather(s_E, ln->E_eV);
        gather(s_sp, ln->species);
        gather(s_gR, ln->log_gR);
        gather(s_gS, ln->log_gS);
        gather(s_gW, ln->log_gW);
        src.lambda_nm = s_lam.data();
        src.log_gf = s_gf.data();
        src.E_eV = s_E.data();
        src.species = s_sp.data();
        src.log_gR = s_gR.data();
        src.log_gS = s_gS.data();
        src.log_gW = s_gW.data();
    }
    MPSA_CUDA_TRY(cudaSetDevice(c->device));
    int rc;
    if ((rc = upload(&c->d_sp_el, sp_el, n_species)) || (rc = upload(&c->d_sp_stage, sp_stage, n_species)) ||
        (rc = upload(&c->d_lam, src.lambda_nm, L)) || (rc = upload(&c->d_loggf, src.log_gf, L)) ||
        (rc = upload(&c->d_E, src.E_eV, L)) || (rc = upload(&c->d_lgR, src.log_gR, L)) ||
        (rc = upload(&c->d_lgS, src.log_gS, L)) || (rc = upload(&c->d_lgW, src.log_gW, L)) ||
        (rc = upload(&c->d_species, src.species, L))) {
        c->L = 0;
        return rc;
    }
    c->n_sp = n_species;
    c->h_sp_el.assign(sp_el, sp_el + n_species);
    c->h_sp_stage.assign(sp_stage, sp_stage + n_species);
    c->L = L;
    return MPSA_OK;
}

}  // extern "C"

namespace mpsa {
namespace {

// Population table of every (composition, point) row from packed element records (shared by
// set_atmosphere_grid and set_atmosphere_grid_eos).
int atmosphere_grid(mpsa_ctx* c, const char* who, int ne, const std::vector<double>& rec, int32_t n_points,
                    const double* T, const double* P, int32_t n_comp, const double* abund, double vturb) {
    if (n_points < 1) return fail(MPSA_EINVAL, "%s: n_points = %d", who, n_points);
    if (n_comp < 1 || (!abund && n_comp != 1)) return fail(MPSA_EINVAL, "%s: n_comp = %d", who, n_comp);
    if (!(vturb >= 0) || !isfinite(vturb)) return fail(MPSA_EINVAL, "%s: vturb = %g", who, vturb);
    if ((int64_t)n_comp * n_points > (1ll << 30)) return fail(MPSA_EINVAL, "%s: %d x %d rows", who, n_comp, n_points);
    for (int i = 0; i < n_points; ++i)
        if (!(T[i] > 0) || !(P[i] > 0) || !isfinite(T[i]) || !isfinite(P[i]))
            return fail(MPSA_EINVAL, "%s: T[%d] = %g, P[%d] = %g", who, i, T[i], i, P[i]);
    std::vector<double> ab((size_t)n_comp * ne, 1.0);
    if (abund)
        for (size_t i = 0; i < ab.size(); ++i) {
            if (!(abund[i] >= 0) || !isfinite(abund[i])) return fail(MPSA_EINVAL, "%s: abund[%zu]", who, i);
            ab[i] = abund[i];
        }
    MPSA_CUDA_TRY(cudaSetDevice(c->device));
    int rc;
    double *dT = nullptr, *dP = nullptr, *dab = nullptr;
    if ((rc = upload(&c->d_el, rec.data(), rec.size()))) return rc;
    if ((rc = upload(&dT, T, n_points)) || (rc = upload(&dP, P, n_points)) || (rc = upload(&dab, ab.data(), ab.size()))) {
        cudaFree(dT), cudaFree(dP), cudaFree(dab);
        return rc;
    }
    if (c->d_pop) cudaFree(c->d_pop), c->d_pop = nullptr;
    const size_t rows = (size_t)n_comp * n_points;
    cudaError_t e = cudaMalloc(&c->d_pop, rows * pop_stride(ne) * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(dT), cudaFree(dP), cudaFree(dab);
        c->n_el = 0;
        return fail(MPSA_ENOMEM, "%s: %s", who, cudaGetErrorString(e));
    }
    rc = populations_device(ne, c->d_el, dab, n_comp, n_points, dT, dP, c->d_pop, 0);
    cudaError_t e2 = cudaDeviceSynchronize();
    cudaFree(dT), cudaFree(dP), cudaFree(dab);
    if (rc) return rc;
    if (e2 != cudaSuccess) return fail(MPSA_ECUDA, "%s: %s", who, cudaGetErrorString(e2));
    c->n_el = ne;
    c->h_el = rec;
    c->n_points = n_points;
    c->n_comp = n_comp;
    c->vturb = vturb;
    c->h_abund = ab;
    return MPSA_OK;
}

}  // namespace
}  // namespace mpsa

extern "C" {

int set_atmosphere_grid(mpsa_ctx* c, const mpsa_elements* el, int32_t n_points, const double* T, const double* P,
                        int32_t n_comp, const double* abund, double vturb) {
    if (!c || !el || !T || !P) return fail(MPSA_EINVAL, "set_atmosphere_grid: NULL argument");
    const int ne = el->n_elements;
    if (ne < 1 || ne > 64) return fail(MPSA_EINVAL, "set_atmosphere_grid: n_elements = %d", ne);
    if (!el->mass_amu || !el->chi_eV || !el->U1 || !el->U2 || !el->log_eps)
        return fail(MPSA_EINVAL, "set_atmosphere_grid: NULL element array");
    for (int e = 0; e < ne; ++e)
        if (!(el->mass_amu[e] > 0) || !(el->U1[e] > 0) || !(el->U2[e] > 0) || !isfinite(el->chi_eV[e]) ||
            !isfinite(el->log_eps[e]))
            return fail(MPSA_EINVAL, "set_atmosphere_grid: bad element %d", e);
    // the single-ionisation table is the two-stage case with constant partition functions
    std::vector<double> rec((size_t)ne * kElStride, 0.0);
    for (int e = 0; e < ne; ++e) {
        double* q = rec.data() + (size_t)e * kElStride;
        q[kElMass] = el->mass_amu[e];
        q[kElLogEps] = el->log_eps[e];
        q[kElStages] = 2.0;
        q[kElChi] = el->chi_eV[e];
        q[kElLnU] = log(el->U1[e]);
        q[kElLnU + 3] = log(el->U2[e]);
    }
    return atmosphere_grid(c, "set_atmosphere_grid", ne, rec, n_points, T, P, n_comp, abund, vturb);
}

int set_atmosphere_grid_eos(mpsa_ctx* c, const mpsa_eos* eos, int32_t n_points, const double* T, const double* P,
                            int32_t n_comp, const double* abund, double vturb) {
    if (!c || !eos || !T || !P) return fail(MPSA_EINVAL, "set_atmosphere_grid_eos: NULL argument");
    const int ne = eos->n_elements;
    if (ne < 1 || ne > 64) return fail(MPSA_EINVAL, "set_atmosphere_grid_eos: n_elements = %d", ne);
    if (!eos->mass_amu || !eos->log_eps || !eos->n_stages || !eos->chi_eV || !eos->lnU)
        return fail(MPSA_EINVAL, "set_atmosphere_grid_eos: NULL element array");
    std::vector<double> rec((size_t)ne * kElStride, 0.0);
    for (int e = 0; e < ne; ++e) {
        const int ns = eos->n_stages[e];
        if (!(eos->mass_amu[e] > 0) || !isfinite(eos->mass_amu[e]) || !isfinite(eos->log_eps[e]) || ns < 1 ||
            ns > kMaxStages)
            return fail(MPSA_EINVAL, "set_atmosphere_grid_eos: bad element %d", e);
        double* q = rec.data() + (size_t)e * kElStride;
        q[kElMass] = eos->mass_amu[e];
        q[kElLogEps] = eos->log_eps[e];
        q[kElStages] = ns;
        for (int j = 0; j + 1 < ns; ++j) {
            const double chi = eos->chi_eV[(size_t)e * (kMaxStages - 1) + j];
            if (!isfinite(chi)) return fail(MPSA_EINVAL, "set_atmosphere_grid_eos: chi of element %d stage %d", e, j);
            q[kElChi + j] = chi;
        }
        for (int j = 0; j < ns; ++j)
            for (int k = 0; k < 3; ++k) {
                const double v = eos->lnU[((size_t)e * kMaxStages + j) * 3 + k];
                if (!isfinite(v)) return fail(MPSA_EINVAL, "set_atmosphere_grid_eos: lnU of element %d stage %d", e, j);
                q[kElLnU + 3 * j + k] = v;
            }
    }
    return atmosphere_grid(c, "set_atmosphere_grid_eos", ne, rec, n_points, T, P, n_comp, abund, vturb);
}

int mpsa_get_populations(mpsa_ctx* c, int32_t row0, int32_t n_rows, double* out, int32_t* stride) {
    if (!c || (n_rows > 0 && !out)) return fail(MPSA_EINVAL, "mpsa_get_populations: NULL argument");
    if (!c->d_pop) return fail(MPSA_ESTATE, "mpsa_get_populations: no atmosphere grid set");
    const int rows = c->n_comp * c->n_points;
    if (row0 < 0 || n_rows < 0 || row0 + (int64_t)n_rows > rows)
        return fail(MPSA_EINVAL, "mpsa_get_populations: rows %d..%d of %d", row0, row0 + n_rows, rows);
    const int st = pop_stride(c->n_el);
    if (stride) *stride = st;
    if (n_rows == 0) return MPSA_OK;
    MPSA_CUDA_TRY(cudaSetDevice(c->device));
    MPSA_CUDA_TRY(cudaMemcpy(out, c->d_pop + (size_t)row0 * st, (size_t)n_rows * st * sizeof(double),
                             cudaMemcpyDeviceToHost));
    return MPSA_OK;
}

int mpsa_profile_enable(mpsa_ctx* c, int enable) {
    if (!c) return fail(MPSA_EINVAL, "mpsa_profile_enable: NULL context");
    c->prof = enable != 0;
    return MPSA_OK;
}

int mpsa_profile_read(mpsa_ctx* c, int kernel, double* total_ms, int64_t* launches) {
    if (!c || !total_ms || !launches || kernel < 0 || kernel > 3) return fail(MPSA_EINVAL, "mpsa_profile_read: bad argument");
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

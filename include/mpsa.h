/*
 * mpsa.h -- C ABI of the GB300 line-opacity / ODF / spectrum library.
 *
 * The library implements the data-parallel hot path of the MPS-ATLAS opacity
 * module (Witzke et al. 2021, arXiv 2105.13611): line-by-line opacity synthesis
 * (Sect. 2.1, Eq. l_nu_line; App. E), ODF binning (Sect. 2.3; App. E) and an LTE
 * emergent-intensity formal solution (Sect. 2.2, Eq. Ilambda).
 *
 * Conventions shared by every entry point
 *  - Return value: MPSA_OK (0) or a negative MPSA_E* code.  mpsa_last_error()
 *    returns a human-readable message for the calling thread's last failure.
 *  - Units are cgs; wavelengths at the API are in nm, energies in eV.
 *  - "host" pointers are read during the call only and may be freed on return.
 *    "device" pointers are CUDA device memory owned by the caller; the library
 *    never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it; calls do not synchronise the host unless they
 *    say so.  Outputs are valid once the stream reaches the enqueued work.
 *  - A context (mpsa_ctx) owns the resident device data (line list, element
 *    and species tables, FP64 population table).  A context is bound to one
 *    device and must not be used from two host threads at once.
 *  - Per-call scratch is stream-ordered device memory from a memory pool owned by
 *    the context (cudaMallocFromPoolAsync / cudaFreeAsync on the call's stream).
 *    The pool keeps freed memory cached for the next call until mpsa_destroy, so
 *    the device memory a context holds grows to the largest scratch of its calls.
 */
#ifndef MPSA_H
#define MPSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPSA_OK        0
#define MPSA_EINVAL   -1   /* bad argument: shape, NaN, unsorted, out of range   */
#define MPSA_ENOMEM   -2   /* device allocation failed                          */
#define MPSA_ECUDA    -3   /* a CUDA runtime call failed                        */
#define MPSA_ESTATE   -4   /* call out of order (e.g. no line list loaded)      */
#define MPSA_ETIMEOUT -5   /* a bounded wait gave up                            */

typedef struct mpsa_ctx mpsa_ctx;

/* Create a context on CUDA device `device`.  *out receives the handle. */
int mpsa_create(mpsa_ctx** out, int device);
/* Free every device buffer the context owns (synchronises the device). */
void mpsa_destroy(mpsa_ctx* ctx);
/* Message of the calling thread's last failed call ("" if none).  Valid until the next call. */
const char* mpsa_last_error(void);
/* Library version string. */
const char* mpsa_version(void);

/* Element table (host arrays of length n_elements).  Element 0 must be hydrogen
 * (its neutral stage supplies the van der Waals perturbers n_HI).  Each element
 * ionises once (stages I and II) with fixed partition functions U1, U2 and
 * first ionisation energy chi_eV; log_eps is the abundance (H = 12).  The
 * multi-stage table is mpsa_eos (set_atmosphere_grid_eos). */
typedef struct {
    int32_t n_elements;
    const double* mass_amu;
    const double* chi_eV;
    const double* U1;
    const double* U2;
    const double* log_eps;
} mpsa_elements;

/* Line list, structure of arrays (host arrays of length n_lines), sorted by
 * ascending lambda_nm.  species[i] indexes the species table given to
 * load_linelist.  Damping: total gamma = 10^log_gR + 10^log_gS * n_e +
 * 10^log_gW * n_HI [s^-1] (radiative, Stark per electron, van der Waals per H I). */
typedef struct {
    int64_t n_lines;
    const double* lambda_nm;
    const float* log_gf;
    const float* E_eV;        /* lower-level excitation energy */
    const int32_t* species;
    const float* log_gR;
    const float* log_gS;
    const float* log_gW;
} mpsa_lines;

/* Log-lambda grid lambda_j = lambda0 (1 + 1/R)^j, j = 0..N-1 with
 * N = floor(ln(lambda1/lambda0)/ln(1+1/R)) + 1 (App. E of the paper). */
typedef struct {
    double lambda0_nm;
    double lambda1_nm;
    double R;
} mpsa_lgrid;

/* Options of the synthesis.  Zero-initialised fields take the defaults. */
typedef struct {
    double cut;         /* profile cut relative to the flat continuum (default 1e-3)        */
    double kc_factor;   /* flat continuum kappa_c = kc_factor * median kappa0 (default 1e-2) */
    int32_t precision;  /* MPSA_PREC_* (default compensated FP32)                           */
    int32_t tile;       /* grid points per CTA tile; 0 = library default                   */
    int32_t continuum;  /* synth_spectrum: 0 = the flat continuum of the cut rule (default);
                           an OR of MPSA_CONT_* = that closed-form continuum (synth_continuum)
                           per depth and wavelength in the radiative transfer instead (the
                           cut rule keeps the flat continuum)                                */
    int32_t reserved;   /* 0 */
} mpsa_synth_opts;

#define MPSA_PREC_FP32_COMPENSATED 0   /* FP32 profiles, chunked FP32 partials + Kahan fold */
#define MPSA_PREC_FP32_NAIVE       1   /* FP32 profiles, plain FP32 running sums            */
#define MPSA_PREC_FP64             2   /* FP64 line terms, profiles and sums (precision study;
                                          FP64 runs far below the FP32 rate on this GPU)     */
#define MPSA_PREC_FP32_POP32       3   /* as 0, with the population table rounded to FP32
                                          before the line terms (precision study)            */

/*
 * load_linelist -- copy a line list and its species table into the context.
 * Paper: the line lists of Sect. 2.3 / Sect. 4.4 (Kurucz, VALD); lines carry
 * the quantities of Eq. (l_nu_line).
 *   n_species, species_element[n_species], species_stage[n_species] (host):
 *     species s belongs to element species_element[s] (index into the element
 *     table of set_atmosphere_grid) in stage species_stage[s] (0 = I, 1 = II, ...,
 *     4 = V; stages above II need set_atmosphere_grid_eos).
 *   lines (host): the list in any order.  The kernels need it ascending in
 *     lambda_nm: a list that is not is sorted (stably, lines of equal lambda
 *     keep their order) into a host copy before the upload.
 * Replaces any previously loaded list.  Synchronises the device on return.
 * Errors: MPSA_EINVAL (n_lines < 1, non-finite or non-positive lambda, species
 * out of range, non-finite line parameters), MPSA_ENOMEM, MPSA_ECUDA.
 */
int load_linelist(mpsa_ctx* ctx, int32_t n_species, const int32_t* species_element,
                  const int32_t* species_stage, const mpsa_lines* lines);

/*
 * set_atmosphere_grid -- build the FP64 population table (paper Sect. 2.1 and
 * App. A: Saha-Boltzmann populations with n_e from charge conservation), for
 * elements with stages I and II and constant partition functions (the two-stage
 * case of set_atmosphere_grid_eos, which solves it).
 *   el (host): element table.
 *   n_points, T[n_points], P[n_points] (host): temperatures [K] and gas
 *     pressures [dyn cm^-2] of the atmosphere points (any set, e.g. a T-P grid).
 *   n_comp, abund_scale (host, [n_comp][n_elements] row-major, or NULL with
 *     n_comp = 1): per-element abundance multipliers of each composition.
 *   vturb_cm_s: micro-turbulent velocity added to the thermal Doppler width.
 * The table holds, per (composition, point) in that order (row cp = comp *
 * n_points + point): n_e, n_HI, rho and N/U of the stages of every element
 * (layout: mpsa_get_populations).  Computed on the device in FP64.  Synchronises.
 * Errors: MPSA_EINVAL (non-positive T or P, n_elements < 1, bad scales).
 */
int set_atmosphere_grid(mpsa_ctx* ctx, const mpsa_elements* el, int32_t n_points,
                        const double* T, const double* P, int32_t n_comp,
                        const double* abund_scale, double vturb_cm_s);

/* Element table of the multi-stage equation of state (host arrays).  Element e has stages
 * 0 .. n_stages[e]-1 (I, II, ..., at most MPSA_MAX_STAGES); chi_eV[e][j] (row-major
 * [n_elements][MPSA_MAX_STAGES - 1]) is the ionisation energy from stage j to j + 1; the
 * partition function of stage j is ln U_j(T) = c0 + c1 x + c2 x^2 with x = ln(T / 5040 K) and
 * (c0, c1, c2) = lnU[e][j][0..2] (row-major [n_elements][MPSA_MAX_STAGES][3]); entries beyond
 * an element's stages are ignored.  Element 0 must be hydrogen. */
#define MPSA_MAX_STAGES 5
typedef struct {
    int32_t n_elements;
    const double* mass_amu;
    const double* log_eps;
    const int32_t* n_stages;
    const double* chi_eV;
    const double* lnU;
} mpsa_eos;

/*
 * set_atmosphere_grid_eos -- the population table from the multi-stage equation of state of
 * paper App. A (without molecules): Saha-Boltzmann ratios between all stages of every element
 * (up to stage V, App. E) with temperature-dependent partition functions, particle and charge
 * conservation solved for n_e by Newton-Raphson steps in ln n_e (kept inside a bracket) to a
 * relative change below 1e-14, in FP64 on the device.  The other arguments, the table and the
 * errors are those of set_atmosphere_grid (MPSA_EINVAL also for a stage count outside 1..5 or
 * a non-finite coefficient).  Species of load_linelist may then be in stages 0..4; a species
 * whose stage its element does not have gives MPSA_EINVAL at synthesis.  Synchronises.
 */
int set_atmosphere_grid_eos(mpsa_ctx* ctx, const mpsa_eos* eos, int32_t n_points, const double* T,
                            const double* P, int32_t n_comp, const double* abund_scale, double vturb_cm_s);

/*
 * mpsa_get_populations -- copy rows row0 .. row0+n_rows-1 of the population table to the host
 * (synchronous).  Row layout (*stride doubles per row, 5 + 5 n_elements): T, P, n_e, n_HI, rho,
 * then N/U of stages I..V of every element (0 for stages the element does not have); the
 * number densities are in cm^-3, rho in g cm^-3.  stride may be NULL; n_rows = 0 only returns
 * the stride.  Errors: MPSA_EINVAL, MPSA_ESTATE (no grid), MPSA_ECUDA.
 */
int mpsa_get_populations(mpsa_ctx* ctx, int32_t row0, int32_t n_rows, double* out, int32_t* stride);

/* Number of grid points N of a log-lambda grid (0 on invalid input). */
int64_t mpsa_grid_size(const mpsa_lgrid* grid);

/*
 * synth_opacity -- line-by-line opacity on a log-lambda grid (paper Eq.
 * l_nu_line summed over lines, Sect. 2.1; grid and cut of App. E / Sect. 4.3).
 *   grid (host): the lambda grid, N = mpsa_grid_size(grid) points.
 *   n_sel, sel[n_sel] (host): population-table rows cp = comp*n_points + point.
 *   kappa_out (device, float[n_sel][N], row-major): line opacity [cm^2 g^-1].
 *   kappa_c_out (device, float[n_sel], or NULL): the flat continuum of each row,
 *     kappa_c = kc_factor * median over all lines of the line-centre opacity.
 *   evals_out (device, int64[n_sel], or NULL): number of (line, grid point)
 *     profile evaluations inside the lines' cut windows.
 * A line contributes at grid point j iff its absorption coefficient there is
 * >= cut * kappa_c (FP32 decision).  Profiles are evaluated in FP32 (Voigt,
 * three-tier rational method), populations come from the FP64 table.
 * Stream-ordered, no host synchronisation; scratch comes from the context's
 * pool, released in stream order after the call's kernels.
 * Errors: MPSA_ESTATE (no line list / grid), MPSA_EINVAL, MPSA_ENOMEM, MPSA_ECUDA.
 */
int synth_opacity(mpsa_ctx* ctx, const mpsa_lgrid* grid, int32_t n_sel, const int32_t* sel,
                  float* kappa_out, float* kappa_c_out, int64_t* evals_out,
                  const mpsa_synth_opts* opts, void* stream);

/*
 * synth_continuum -- continuous opacity from the closed-form sources of the paper's continuum
 * (Sect. 2.1: electron scattering, bound-free and free-free absorption of H I, Rayleigh
 * scattering on H I; App. G groups 'Elec', 'H1', 'Hray'):
 *   MPSA_CONT_ELEC  n_e sigma_T;
 *   MPSA_CONT_HBF   H I levels n = 1..8, Kramers' cross-section K_bf / (n^5 nu^3) with Gaunt
 *                   factor 1 above each edge chi_H / (h n^2), Boltzmann level populations
 *                   n_HI (2 n^2 / U_HI) e^{-chi_H (1 - 1/n^2)/kT}, times 1 - e^{-h nu/kT};
 *   MPSA_CONT_HFF   hydrogen free-free, K_ff n_e n_HII / (sqrt(T) nu^3) (1 - e^{-h nu/kT}), Gaunt 1;
 *   MPSA_CONT_HRAY  n_HI (5.799e-13 / L^4 + 1.422e-6 / L^6 + 2.784 / L^8) cm^2 (L in Angstrom,
 *                   held at 1300 Angstrom below);
 * all divided by rho.  The other continuum sources of the paper (H-, He, metals, molecules)
 * need tabulated cross-sections and are not provided.
 *   grid (host), n_sel, sel[n_sel] (host): as for synth_opacity (n_sel 1..65535).
 *   sources: an OR of MPSA_CONT_* (MPSA_CONT_ALL for all four).
 *   kappa_out (device, float[n_sel][N]): kappa_c [cm^2 g^-1] per row and grid point.
 * Row constants in FP64, per-point sums in FP32.  Stream-ordered.
 * Errors: MPSA_ESTATE (no atmosphere grid), MPSA_EINVAL, MPSA_ENOMEM, MPSA_ECUDA.
 */
#define MPSA_CONT_ELEC 1
#define MPSA_CONT_HBF  2
#define MPSA_CONT_HFF  4
#define MPSA_CONT_HRAY 8
#define MPSA_CONT_ALL  15
int synth_continuum(mpsa_ctx* ctx, const mpsa_lgrid* grid, int32_t n_sel, const int32_t* sel, int32_t sources,
                    float* kappa_out, void* stream);

#define MPSA_MEAN_ARITH 0
#define MPSA_MEAN_GEOM  1

/*
 * build_odf -- opacity distribution functions (paper Sect. 2.3 and App. E):
 * per row and interval, the values are ordered ascending, the ordered profile
 * is split at cumulative width fractions c_s = w_1 + ... + w_s (FP64 partial
 * sums, c_n forced to 1; a point straddling a boundary is split fractionally)
 * and each sub-bin is replaced by its mean.
 *   kappa (device, float[n_rows][N]): non-negative, finite values.
 *   K, bounds[K+1] (host, int64): interval k = [bounds[k], bounds[k+1]);
 *     strictly increasing, bounds[0] >= 0, bounds[K] <= N, each interval
 *     shorter than 2^21 points.
 *   n_steps, widths[n_steps] (host): sub-bin width fractions, positive, summing
 *     to 1 within 1e-12.  n_steps <= 32.
 *   mean_kind: MPSA_MEAN_ARITH (arithmetic mean of the sub-bin) or
 *     MPSA_MEAN_GEOM (exp of the sub-bin integral of ln kappa divided by its
 *     width, the paper's default in Sect. 2.3; a sub-bin whose rank range
 *     reaches into zero values has geometric mean 0).
 *   odf_out (device, double[n_rows][K][n_steps]).
 *   n_rows: 1..65535 rows per call (one launch; split larger tables).
 * The order statistics at the boundaries are exact.  With n_steps <= 12 on
 * intervals of at most 65,536 points, a count pass over 14-bit prefixes of the
 * FP32 patterns and a gather pass compute both kinds of mean.  Arithmetic sums
 * of the values between the boundaries' bins are FP32 per lane: relative error
 * at most 3.8e-6, about 1e-7 in practice.  The boundaries' own bins are summed
 * exactly as integers, and so are all the geometric means' ln sums (units of
 * 2^-30).  A second kernel recomputes, by the multi-select below, any interval
 * whose boundary bins hold more than 8,192 values.  Every other case uses a
 * 4-level radix multi-select (12, 7, 6 and 6 bits) on the FP32 bit patterns
 * with exact integer partial sums; only the final cross-exponent reduction is
 * FP64, and geometric means take one more pass that sums ln kappa between
 * consecutive order statistics.  ln kappa is the exponent times ln 2 plus FP32
 * logf of the mantissa.  Stream-ordered, no host synchronisation.
 * Errors: MPSA_EINVAL, MPSA_ENOMEM, MPSA_ECUDA.
 */
int build_odf(mpsa_ctx* ctx, const float* kappa, int32_t n_rows, int64_t N,
              int32_t K, const int64_t* bounds, int32_t n_steps, const double* widths,
              int32_t mean_kind, double* odf_out, void* stream);

/*
 * build_odf_noalloc -- build_odf that allocates no device memory.  The paper has
 * no counterpart: this is an operational variant for callers that must not
 * allocate, e.g. a process whose device memory belongs to another framework's
 * caching allocator, or a latency-critical loop in which cudaMalloc (or a
 * cudaFree that may synchronise the device) is not allowed.
 *   device: CUDA device to run on (made current by the call).
 *   The other arguments, results and errors are those of build_odf (no context
 *   is needed); K must not exceed 65536 intervals (MPSA_EINVAL otherwise).
 * The interval bounds and widths are staged in one fixed file-scope device array
 * of about 0.5 MiB, which every device that loads the library keeps until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, once per device and safe from several host
 * threads); make this first call before any stream capture.  The address is not
 * looked up again, so do not call this entry point after a cudaDeviceReset.
 * Every call shares the array and overwrites it: calls that may overlap on the
 * GPU (for example on different streams) race and must be serialised by the
 * caller.  The host arrays are copied with cudaMemcpyAsync from pageable memory.
 * Stream-ordered otherwise.
 */
int build_odf_noalloc(int32_t device, const float* kappa, int32_t n_rows, int64_t N,
                      int32_t K, const int64_t* bounds, int32_t n_steps, const double* widths,
                      int32_t mean_kind, double* odf_out, void* stream);

/* One model atmosphere for synth_spectrum (host arrays of length n_depth,
 * ordered from the top down): column mass m [g cm^-2], T [K], P [dyn cm^-2]. */
typedef struct {
    int32_t n_depth;
    const double* m;
    const double* T;
    const double* P;
    int32_t comp;      /* composition row of the atmosphere grid's abundance scales */
} mpsa_atmos;

/*
 * synth_spectrum -- emergent intensity I(mu, lambda) of one atmosphere over a
 * wavelength window (paper Eq. Ilambda with LTE source S = B_lambda(T)).
 * For every depth the populations, the line opacity on the window grid (same
 * cut rule as synth_opacity, lines centred outside the window contribute their
 * wings) and the continuum (the flat one, or opts->continuum's sources of
 * synth_continuum at every wavelength) are built; tau follows by the trapezoid rule in
 * column mass and I by a linear-source integration from a diffusion lower
 * boundary (I = S + mu dS/dtau) to the surface.
 *   atm (host), win (host): the atmosphere and the window grid (N_win points).
 *   n_mu, mu[n_mu] (host): direction cosines in (0, 1].
 *   I_out (device, float[n_mu][N_win]).
 * Requires the element table of set_atmosphere_grid (the atmosphere's own
 * populations are computed in FP64 on the device).  Stream-ordered.
 * Errors: MPSA_ESTATE, MPSA_EINVAL, MPSA_ENOMEM, MPSA_ECUDA.
 */
int synth_spectrum(mpsa_ctx* ctx, const mpsa_atmos* atm, const mpsa_lgrid* win,
                   int32_t n_mu, const double* mu, float* I_out,
                   const mpsa_synth_opts* opts, void* stream);

/* An ODF table of one composition on a T-P grid: the sub-bin mean line opacities of
 * build_odf for the grid's points and the continuum opacity of each point. */
typedef struct {
    int32_t nT, nP;           /* grid: table row r = iT * nP + iP */
    const double* log10_T;    /* host [nT], strictly increasing */
    const double* log10_P;    /* host [nP], strictly increasing (P in dyn cm^-2) */
    int32_t K;                /* bins */
    int32_t n_steps;          /* sub-bins per bin, 1..32 */
    const double* odf;        /* device double[nT * nP][K][n_steps]: sub-bin mean line
                                 opacity [cm^2 g^-1] (build_odf's output for rows r) */
    const float* kappa_c;     /* device float[nT * nP]: continuum opacity [cm^2 g^-1]
                                 (synth_opacity's kappa_c_out for rows r), > 0 */
    const double* lam_c_nm;   /* host [K]: bin centre wavelengths [nm] */
    const double* widths;     /* host [n_steps]: sub-bin widths as fractions of the bin,
                                 positive, summing to 1 */
} mpsa_odf_table;

/*
 * odf_intensity -- emergent bin intensities of many 1D atmospheres from an ODF table
 * (module III through ODFs; paper Sect. 2.3 and App. E):
 *   I_bin,k(mu) = sum_s w_s I_lambda_c,k(kappa_c + kappa_s,k; mu).
 * At every depth of a ray the sub-bin opacities kappa_s,k and the continuum are
 * interpolated bilinearly in (log10 T, log10 P) on the table grid (coordinates clamped
 * to the grid's edges); per sub-bin, tau follows by the trapezoid rule in column mass
 * and I by the formal solution of synth_spectrum (S = B_lambda(T) at the bin centre,
 * diffusion lower boundary); the bin intensity is the width-weighted sum.  FP32
 * arithmetic; the table is read in FP64 and rounded per value.
 *   tab (host struct): the table (odf and kappa_c on the device, the rest on the host);
 *     nT * nP * K * n_steps below 2^31 values.
 *   n_rays (1..65535), n_depth (2..256): rays of n_depth points each, top down.
 *   m, T, P (device, double[n_rays][n_depth]): column mass [g cm^-2] (positive,
 *     strictly increasing), T [K] and P [dyn cm^-2] (positive, finite).
 *   n_mu (1..16), mu[n_mu] (host): direction cosines in (0, 1].
 *   I_out (device, float[n_rays][n_mu][K]).
 *   ray_status (device, int32[n_rays], may be NULL): 0 for a valid ray; 1 where its m, T
 *     or P break the rules above, in which case its I_out is NaN.
 * The ray arrays are checked on the device (no synchronisation).  Stream-ordered.
 * Errors: MPSA_EINVAL (host arguments), MPSA_ENOMEM, MPSA_ECUDA.
 */
int odf_intensity(mpsa_ctx* ctx, const mpsa_odf_table* tab, int32_t n_rays, int32_t n_depth,
                  const double* m, const double* T, const double* P, int32_t n_mu, const double* mu,
                  float* I_out, int32_t* ray_status, void* stream);

/*
 * Batched form: many rows on several grids in one persistent, graph-captured
 * launch (the paper's method, Eq. l_nu_line + App. E, over a heterogeneous set of
 * (composition, T, P) rows and wavelength windows).  At creation every group's line
 * preparation runs once, an autotuner (autotune != 0) times the persistent profile
 * kernel for each candidate configuration (points per thread, threads per CTA,
 * CTAs per SM) on a sample of tiles and keeps the fastest per grid point, the
 * (row, tile) units are ordered by decreasing estimated cost, and the whole
 * pipeline (preparation of every group, one persistent profile launch, the ODFs)
 * is captured into a CUDA graph.  mpsa_batch_run replays it on `stream`; the
 * results equal those of synth_opacity / build_odf within the stated tolerances.
 * The graph binds the context's resident buffers and the groups' output buffers:
 * re-create the batch after load_linelist or set_atmosphere_grid.
 */
typedef struct {
    mpsa_lgrid grid;
    int32_t n_sel;
    const int32_t* sel;        /* host: population-table rows */
    float* kappa_out;          /* device float[n_sel][N] */
    float* kappa_c_out;        /* device float[n_sel] or NULL */
    int64_t* evals_out;        /* device int64[n_sel] or NULL */
    int32_t K;                 /* intervals of the ODF of this group; 0 = no ODF */
    const int64_t* bounds;     /* host int64[K+1] */
    int32_t n_steps;
    const double* widths;      /* host */
    double* odf_out;           /* device double[n_sel][K][n_steps] */
    int32_t mean_kind;         /* MPSA_MEAN_ARITH or MPSA_MEAN_GEOM */
} mpsa_batch_group;

typedef struct {
    int32_t pts_per_thread, threads, min_blocks;   /* chosen profile-kernel configuration */
    int32_t n_rows;
    int64_t n_units;                                /* (row, tile) work units */
    int32_t n_tuned;                                /* configurations timed by the autotuner */
    double tune_ms_per_mpoint[8];                   /* their time per 1e6 grid points */
} mpsa_batch_info;

typedef struct mpsa_batch mpsa_batch;
int mpsa_batch_create(mpsa_ctx* ctx, int32_t n_groups, const mpsa_batch_group* groups,
                      const mpsa_synth_opts* opts, int32_t autotune, void* stream, mpsa_batch** out);
int mpsa_batch_run(mpsa_batch* b, void* stream);
int mpsa_batch_get_info(const mpsa_batch* b, mpsa_batch_info* out);
void mpsa_batch_destroy(mpsa_batch* b);

/*
 * Request server (continuous batching).  Not a step of the paper's method: the
 * serving form of the library.  A worker thread owns the context while the
 * server exists (do not call other entry points on that context meanwhile).
 * Requests wait in FIFO order; the oldest is started as soon as one of
 * max_inflight stream slots is free and its estimated device memory fits the
 * budget, so requests arriving while others run are admitted without waiting
 * for them and their kernels overlap on the device.  Spectrum requests run
 * whole on streams of the device's highest priority.  ODF requests run on its
 * lowest, one chunk of rows at a time (the next when the previous completes), so
 * a spectrum waits behind at most one chunk (running CTAs are not preempted).
 * Each request runs exactly
 * the kernels of the direct entry points (synthesis in chunks of
 * rows_per_chunk rows to bound scratch), so its result does not depend on what
 * else is in flight.
 */
typedef struct mpsa_server mpsa_server;

#define MPSA_REQ_SPECTRUM 1
#define MPSA_REQ_ODF      2

typedef struct {
    int32_t kind;              /* MPSA_REQ_SPECTRUM or MPSA_REQ_ODF */
    /* spectrum (synth_spectrum's arguments; host arrays copied at submit) */
    mpsa_atmos atm;
    mpsa_lgrid win;
    int32_t n_mu;
    const double* mu;
    float* I_out;              /* host float[n_mu][N_win], written on completion */
    /* ODF: rows of the atmosphere grid, synthesised on `grid` and reduced with
       build_odf's rules; host arrays copied at submit */
    int32_t n_sel;
    const int32_t* sel;
    mpsa_lgrid grid;
    int32_t K;
    const int64_t* bounds;
    int32_t n_steps;
    const double* widths;
    double* odf_out;           /* host double[n_sel][K][n_steps], written on completion */
    float* kappa_c_out;        /* host float[n_sel] or NULL */
    int32_t mean_kind;         /* ODF: MPSA_MEAN_ARITH or MPSA_MEAN_GEOM */
} mpsa_request;

typedef struct {
    int64_t submitted, completed, failed, running, queued;
    size_t bytes_in_use, bytes_peak;    /* admitted memory estimates */
} mpsa_server_stats;

/* Create a server on ctx (which needs a line list and an atmosphere grid).
 * hbm_budget_bytes bounds the summed memory estimates of running requests.
 * Errors: MPSA_EINVAL, MPSA_ESTATE, MPSA_ECUDA. */
int mpsa_server_create(mpsa_server** out, mpsa_ctx* ctx, size_t hbm_budget_bytes,
                       int32_t max_inflight, int32_t rows_per_chunk);
/* Queue a request; *ticket identifies it.  Output buffers must stay valid until
 * mpsa_server_wait returns for it.  MPSA_ENOMEM if it alone exceeds the budget. */
int mpsa_server_submit(mpsa_server* s, const mpsa_request* req, int64_t* ticket);
/* Wait up to timeout_ms for a request; MPSA_OK when its outputs are written
 * (latency_ms = completion - submission), MPSA_ETIMEOUT if it is not done yet
 * (wait again), or the request's error.  A finished ticket is released. */
int mpsa_server_wait(mpsa_server* s, int64_t ticket, int32_t timeout_ms, double* latency_ms);
int mpsa_server_get_stats(mpsa_server* s, mpsa_server_stats* out);
/* Drop every request still waiting for admission (their waits return
 * MPSA_ESTATE); running requests are not affected. */
int mpsa_server_cancel_queued(mpsa_server* s, int64_t* n_cancelled);
/* Finish queued and running requests, then free the server. */
void mpsa_server_destroy(mpsa_server* s);

/*
 * Kernel timing for measurement tools (not part of the method).  While enabled,
 * the library records a CUDA event pair on the launching stream around each
 * launch of its dominant kernels: MPSA_KERNEL_PROFILE (the profile kernel
 * of synth_opacity / synth_spectrum), MPSA_KERNEL_ODF (the kernel of
 * build_odf), MPSA_KERNEL_BINS (the kernel of odf_intensity) and
 * MPSA_KERNEL_CONTINUUM (the kernels of synth_continuum).  mpsa_profile_read waits for the recorded events, returns the
 * summed device time [ms] and launch count of one kernel, and clears its list.
 * Do not enable while capturing a CUDA graph.
 */
#define MPSA_KERNEL_PROFILE   0
#define MPSA_KERNEL_ODF       1
#define MPSA_KERNEL_BINS      2
#define MPSA_KERNEL_CONTINUUM 3
int mpsa_profile_enable(mpsa_ctx* ctx, int enable);
int mpsa_profile_read(mpsa_ctx* ctx, int kernel, double* total_ms, int64_t* launches);

/*
 * mpsa_voigt -- the Voigt function H(v, a) = Re w(v + i a) of the line profile
 * (paper Sect. 2.1: argument v = (nu - nu0)/dnu_D, damping a = gamma/(4 pi dnu_D)),
 * evaluated on the device exactly as the synthesis kernels evaluate it, for
 * accuracy tests of the profile tiers.
 *   v, a (device, double[n]): arguments (a > 0; the sign of v is ignored).
 *   precision: MPSA_PREC_FP64 evaluates the FP64 tiers in double; any other value
 *     rounds v and a to FP32 and evaluates the FP32 tiers (far: rational or
 *     one-level continued fraction; mid: five-level continued fraction; core:
 *     shifted 12-point Gauss-Hermite).
 *   out (device, double[n]): H, widened from FP32 for the FP32 tiers.
 * Stream-ordered.  Errors: MPSA_EINVAL, MPSA_ECUDA.
 */
int mpsa_voigt(mpsa_ctx* ctx, const double* v, const double* a, int64_t n, int32_t precision, double* out,
               void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MPSA_H */

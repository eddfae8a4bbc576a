// Library-internal entry points shared between translation units (not part of the C ABI).
#pragma once

#include "common.cuh"

namespace mpsa {

// Line preparation works on blocks of kPrepLines lines of one row, kPrepThreads threads each
// (per-block class counts, window-length sums and stable bucket placement) (synth.cu).
constexpr int kPrepThreads = 256;
constexpr int kPrepLines = 1024;

// FP64 Saha populations for n_comp x n_points rows (api.cu).
int populations_device(int n_el, const double* d_el, const double* d_abund, int n_comp, int n_points,
                       const double* d_T, const double* d_P, double* d_pop, cudaStream_t s);

// Line-by-line opacity for rows d_sel of a population table onto the grid
// (lam0_nm, R, N): kappa [n_sel][N], optional kappa_c [n_sel] and evaluation counts (synth.cu).
int synth_rows(mpsa_ctx* ctx, const double* pop, int n_sel, const int* d_sel, double lam0_nm, double R, int N,
               float* kappa, float* kc_out, int64_t* evals, const mpsa_synth_opts* opts, cudaStream_t st);

// Every species of the line list refers to an element of the table and to a stage that
// element has (synth.cu).
int check_species(const mpsa_ctx* ctx, const char* who);

// Validates a grid and returns its point count (synth.cu).
int check_grid(const mpsa_lgrid* g, int* N);

// ODF kernel launch on device-resident bounds [K+1], cumulative widths [n_steps+1]
// and widths [n_steps]; mean_kind MPSA_MEAN_ARITH or MPSA_MEAN_GEOM (odf.cu).
int odf_launch(const float* kappa, int n_rows, int64_t N, int K, const int64_t* d_bounds, int n_steps,
               const double* d_cw, const double* d_w, double* d_out, int mean_kind, cudaStream_t st);

// One-time kernel attribute set-up of the ODF kernel on the current device (call outside
// stream capture) (odf.cu).
int odf_setup();

// Host-side validation of ODF arguments for one launch of n_rows rows (at most 65,535);
// fills the cumulative widths cw[n_steps+1].  `who` names the entry point in the error
// message (odf.cu).
int odf_check(const char* who, int n_rows, int64_t N, int K, const int64_t* bounds, int n_steps,
              const double* widths, int mean_kind, double* cw);

// Continuous opacity of rows d_sel of `pop` on the grid (lam0, R, N) from the MPSA_CONT_* sources
// into out [n_sel][N] (continuum.cu).
int continuum_launch(mpsa_ctx* ctx, const double* pop, int n_sel, const int* d_sel, double lam0_nm, double R, int N,
                     int sources, float* out, cudaStream_t st);

// Formal solution for D depths on a window grid (spectrum.cu); inputs device-resident.  The
// continuum is kc[d] per depth, or kcont[d][j] per depth and wavelength when kcont is not null.
int formal_launch(int D, int N, const float* kappa, const float* kc, const float* kcont, const float* m,
                  const float* T, double lam0_nm, double lnq, int n_mu, const float* mu, float* I_out, cudaStream_t st);

}  // namespace mpsa

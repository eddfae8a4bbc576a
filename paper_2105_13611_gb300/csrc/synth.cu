// synth_opacity: line-by-line opacity on a log-lambda grid.
//
// Paper: Eq. (l_nu_line) of Sect. 2.1 summed over every line of the list on
// the grid lambda_j = lambda_0 (1 + 1/R)^j of App. E, with the cut of Sect. 4.3 /
// App. E (a line contributes where its absorption coefficient is at least
// cut * kappa_c; kappa_c is the flat continuum kc_factor * median line-centre
// opacity of the synthetic workload).
//
// Pipeline (all on the caller's stream):
//   k_place        per line: centre index c and fraction f on the grid (FP64 log)
//   k_consts       per (row, species): ln(sqrt(pi) e^2/(m_e c) N/U / rho), u, c/u from the FP64 table
//   k_kappa0       per (row, line): ln S, a, ln kappa0 in FP32 log space
//   k_med_*        per row: lower median of ln kappa0 by multi-CTA radix selection -> ln t_p, kappa_c
//   k_prep         per (row, line): strength relative to t_p, cut windows (outer: no point
//                  beyond can pass the cut; inner: every point inside passes), width class
//   k_scan_class, k_scan_fin, k_scatter   stable counting sort of the kept lines by width class
//   k_ranges       per (row, class, tile boundary): first line whose centre lies at or
//                  beyond the boundary (binary search in the centre-sorted class)
//   k_tiles        the profile kernel: one CTA per (row, 2048-point tile); each thread owns
//                  8 grid points in registers; every line whose window reaches the tile is
//                  evaluated at the thread's points; FP32 partial sums per chunk of lines are
//                  folded into Kahan-compensated totals; no atomics; coalesced stores.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "voigt.cuh"
#include "internal.cuh"

namespace mpsa {

namespace {

constexpr float kLn10 = 2.302585092994046f;
constexpr float kFourPi = 12.566370614359172f;
constexpr float kFarV = 41.f;            // far formula valid for |v| >= 40
// The far evaluation v = G_k (kv B) + kv E1 rounds two terms, each at most the larger of
// the tile's span and the centre's distance in x = d ln q; with the centre at least one
// tile (2048 points) from every point of the tile, |x| is at least that span, so v keeps
// about 2e-7 relative accuracy.
constexpr int kFarDist = kTile;

__device__ __forceinline__ int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

// ---------------------------------------------------------------------------
// k_place: c = floor(x0), f = x0 - c with x0 = ln(lambda0/lambda_start)/ln(1+1/R)
// (FP64: an FP32 logarithm would misplace lines by whole grid points).
__global__ void k_place(int64_t L, const double* __restrict__ lam_nm, double lam0_nm, double lnq,
                        int* __restrict__ c_out, float* __restrict__ f_out, float* __restrict__ lamcm_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    const double lam = lam_nm[i];
    double x0 = log(lam / lam0_nm) / lnq;
    x0 = fmin(fmax(x0, -268435456.0), 268435456.0);
    const double c = floor(x0);
    c_out[i] = (int)c;
    f_out[i] = (float)(x0 - c);
    lamcm_out[i] = (float)(lam * 1e-7);
}

// per-row scalars (FP32) and per-(row, species) scalars
struct RowConst {
    float ne, nHI, inv_kT_eV, hc_kT_cm;
};
struct SpConst {
    float lnC, u, kv;
};

__global__ void k_consts(int n_sel, const int* __restrict__ sel, int n_sp, const int* __restrict__ sp_el,
                         const int* __restrict__ sp_stage, int n_el, const double* __restrict__ el,
                         const double* __restrict__ pop, double vturb, int pop32, RowConst* __restrict__ rc,
                         SpConst* __restrict__ sc) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_sel * n_sp) return;
    const int s = t / n_sp, sp = t % n_sp;
    const double* row = pop + (size_t)sel[s] * pop_stride(n_el);
    const double T = row[kPopT];
    const int e = sp_el[sp], st = sp_stage[sp];
    const double m = el[e * kElStride + kElMass] * kAMU;
    const double u = sqrt(2.0 * kKB * T / m + vturb * vturb);
    const double NU = row[pop_nu(e, st)];
    const double pre = sqrt(kPI) * kE * kE / (kME * kC);
    SpConst o;
    if (pop32)   // precision-study variant: the population table rounded to FP32 first
        o.lnC = NU > 0 ? (float)log(pre) + logf((float)NU) - logf((float)row[kPopRho]) : -INFINITY;
    else
        o.lnC = NU > 0 ? (float)(log(pre) + log(NU) - log(row[kPopRho])) : -INFINITY;
    o.u = (float)u;
    o.kv = (float)(kC / u);
    sc[t] = o;
    if (sp == 0) {
        RowConst r;
        r.ne = (float)row[kPopNe];
        r.nHI = (float)row[kPopNHI];
        r.inv_kT_eV = (float)(kEV / (kKB * T));
        r.hc_kT_cm = (float)(kH * kC / (kKB * T));
        rc[s] = r;
    }
}

// ---------------------------------------------------------------------------
// k_kappa0: Eq. (l_nu_line) in log space, FP32.
//   Delta nu_D = u / lambda0, a = gamma / (4 pi Delta nu_D),
//   ln S = ln C_s + ln(gf) - E/kT + ln(1 - e^{-h nu0/kT}) - ln Delta nu_D,
//   ln kappa0 = ln S + ln H(0, a).
// One thread per line and up to kKappa0Rows rows: the line's data and its three damping
// constants are read and formed once, then each row's values follow.
constexpr int kKappa0Rows = 8;

__global__ void k_kappa0(int64_t L, int n_sel, const int* __restrict__ species, const float* __restrict__ loggf,
                         const float* __restrict__ E, const float* __restrict__ lgR, const float* __restrict__ lgS,
                         const float* __restrict__ lgW, const float* __restrict__ lamcm, int n_sp,
                         const RowConst* __restrict__ rc, const SpConst* __restrict__ sc,
                         float* __restrict__ lnS_out, float* __restrict__ a_out, float* __restrict__ lnk0_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    const int sp = species[i];
    const float lam = lamcm[i], lglam = logf(lam), lg = loggf[i], Ei = E[i];
    const float gR = exp10f(lgR[i]), gS = exp10f(lgS[i]), gW = exp10f(lgW[i]);
    const int s1 = min(n_sel, (int)(blockIdx.y + 1) * kKappa0Rows);
    for (int s = blockIdx.y * kKappa0Rows; s < s1; ++s) {
        const RowConst r = rc[s];
        const SpConst q = sc[(size_t)s * n_sp + sp];
        const float gamma = gR + gS * r.ne + gW * r.nHI;
        const float a = gamma * lam / (kFourPi * q.u);
        const float lnDnu = logf(q.u) - lglam;
        const float stim = -expm1f(-r.hc_kT_cm / lam);
        const float lnS = q.lnC + lg * kLn10 - Ei * r.inv_kT_eV + logf(stim) - lnDnu;
        const size_t o = (size_t)s * L + i;
        lnS_out[o] = lnS;
        a_out[o] = a;
        lnk0_out[o] = lnS + logf(voigt_H(0.f, a));
    }
}

// ---------------------------------------------------------------------------
// Lower median (rank (L-1)/2) of ln kappa0 per row: MSB radix selection on order-preserving
// keys of the FP32 bit patterns in three levels of 11, 11 and 10 bits.  At every level a grid
// of CTAs per row histograms its share of the row (the values whose key matches the prefix
// resolved so far) in shared memory and adds the non-empty bins to the row's global
// histogram; one CTA per row then finds the bin holding the rank (k_med_pick).
__device__ __forceinline__ unsigned fkey(float x) {
    unsigned b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unkey(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

struct MedState {
    unsigned prefix;   // key bits resolved so far
    unsigned rank;     // rank of the median among the keys with that prefix
};
constexpr int kMedBins = 2048;
__host__ __device__ constexpr int med_shift(int level) { return level == 0 ? 21 : (level == 1 ? 10 : 0); }
__host__ __device__ constexpr int med_bits(int level) { return level == 2 ? 10 : 11; }

__global__ void k_med_init(int n_sel, int64_t L, MedState* __restrict__ st, unsigned* __restrict__ ghist) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_sel * kMedBins) ghist[i] = 0u;
    if (i < n_sel) st[i] = MedState{0u, (unsigned)((L - 1) / 2)};
}

__global__ void __launch_bounds__(1024) k_med_hist(int64_t L, const float* __restrict__ lnk0, int level,
                                                   const MedState* __restrict__ st, unsigned* __restrict__ ghist) {
    __shared__ unsigned h[kMedBins];
    const int s = blockIdx.y;
    const int shift = med_shift(level), nbits = med_bits(level);
    const unsigned pmask = level == 0 ? 0u : (0xffffffffu << (shift + nbits));
    const unsigned prefix = st[s].prefix;
    for (int i = threadIdx.x; i < kMedBins; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    const float* x = lnk0 + (size_t)s * L;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += stride) {
        const unsigned k = fkey(__ldg(x + i));
        if ((k & pmask) == prefix) atomicAdd(&h[(k >> shift) & ((1u << nbits) - 1u)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (1 << nbits); i += blockDim.x)
        if (h[i]) atomicAdd(&ghist[(size_t)s * kMedBins + i], h[i]);
}

__global__ void __launch_bounds__(1024) k_med_pick(int level, MedState* __restrict__ st,
                                                   unsigned* __restrict__ ghist, float ln_kc_factor, float ln_cut,
                                                   float* __restrict__ ln_tp, float* __restrict__ kc_out) {
    __shared__ int wsum[32];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned* h = ghist + (size_t)s * kMedBins;
    const int nb = 1 << med_bits(level);
    // two bins per thread; block-wide inclusive scan of their counts
    const unsigned c0 = 2 * tid < nb ? h[2 * tid] : 0u, c1 = 2 * tid + 1 < nb ? h[2 * tid + 1] : 0u;
    const int v = (int)(c0 + c1);
    int incl = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        int ti = t;
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ti, d);
            if (lane >= d) ti += y;
        }
        wsum[lane] = ti - t;
    }
    __syncthreads();
    const unsigned before = (unsigned)(wsum[warp] + incl - v);
    const MedState cur = st[s];
    if (cur.rank >= before && cur.rank < before + (unsigned)v) {
        const bool lo = cur.rank < before + c0;
        const unsigned bin = 2u * tid + (lo ? 0u : 1u);
        MedState nx;
        nx.rank = cur.rank - (lo ? before : before + c0);
        nx.prefix = cur.prefix | (bin << med_shift(level));
        st[s] = nx;
        if (level == 2) {
            const float med = unkey(nx.prefix);
            ln_tp[s] = med + ln_kc_factor + ln_cut;
            if (kc_out) kc_out[s] = expf(med + ln_kc_factor);
        }
    }
    __syncthreads();
    // clear the histogram for the next level
    if (2 * tid < kMedBins) h[2 * tid] = 0u;
    if (2 * tid + 1 < kMedBins) h[2 * tid + 1] = 0u;
}

// ---------------------------------------------------------------------------
// Cut windows.  For H monotone in |v| the points where s_rel * H(v, a) >= 1 form
// |v| <= v*.  Bisection (geometric, 40 steps) on the FP32 H gives
//   v_out: H(v) < r (1 - 1e-4) for all v >= v_out  (no point beyond can pass the cut)
//   v_in : H(v) >= r (1 + 1e-4) for all v <= v_in  (every point inside passes)
// with r = 1/s_rel; the margins exceed the FP32 errors of H (3e-6) and of v (2e-6).
// H(v, a) <= 4a/(sqrt(pi) v^2) + exp(-v^2/4) bounds the search.
__device__ float v_bound(float a, float t) {
    return fmaxf(sqrtf(8.f * a * kInvSqrtPi / t), 2.f * sqrtf(logf(fmaxf(2.f / t, 1.f)))) * 1.01f + 1.f;
}

// Crossing of H(v, a) = t by the Illinois variant of regula falsi on ln H against ln v.
// Invariant: H(e^xlo) >= t > H(e^xhi); the bracket shrinks to a few FP32 ulps of ln v.
// The search first tries a bracket of +-5 % around ve = max(sqrt(a / (sqrt(pi) t)),
// sqrt(-ln t)), the crossing of the Lorentz wing a / (sqrt(pi) v^2) or of the Doppler core
// e^{-v^2}; where H confirms it the search starts there, else from the ends it has verified.
// Returns the verified ends.
__device__ void crossing(float a, float t, float vb, float* v_ge, float* v_lt) {
    const float lt = logf(t);
    auto f = [&](float x) {
        const float h = voigt_H(expf(x), a);
        return h > 0.f ? logf(h) - lt : -1.0e4f;
    };
    float xlo = logf(1e-4f), xhi = logf(vb), flo, fhi;
    const float ve = fmaxf(sqrtf(a * kInvSqrtPi / t), sqrtf(fmaxf(-lt, 0.f)));
    const float xg0 = logf(ve) - 0.05f, xg1 = xg0 + 0.1f;
    bool probe_lo = true;
    if (xg0 > xlo && xg1 < xhi) {
        const float f0 = f(xg0);
        if (f0 >= 0.f) {                   // H >= t at xg0, so also at |v| = 1e-4
            probe_lo = false;
            xlo = xg0;
            flo = f0;
            const float f1 = f(xg1);
            if (f1 < 0.f) {
                xhi = xg1;
                fhi = f1;
            } else {
                xlo = xg1;
                flo = f1;
                fhi = f(xhi);
            }
        } else {
            xhi = xg0;
            fhi = f0;
        }
    } else {
        fhi = f(xhi);
    }
    if (probe_lo) {
        flo = f(xlo);
        if (flo < 0.f) {                   // below t already at |v| = 1e-4
            *v_ge = -1.f;
            *v_lt = 1e-4f;
            return;
        }
    }
    int side = 0;
    // stop at ~2 FP32 ulps of ln v (the ends stay verified, so precision only sets tightness)
    for (int it = 0; it < 60 && xhi - xlo > 3e-7f * fmaxf(1.f, fabsf(xhi)); ++it) {
        float x = (xlo * fhi - xhi * flo) / (fhi - flo);
        if (!(x > xlo && x < xhi)) x = 0.5f * (xlo + xhi);
        if (!(x > xlo && x < xhi)) break;
        const float fx = f(x);
        if (fx >= 0.f) {
            xlo = x;
            flo = fx;
            if (side == 1) fhi *= 0.5f;
            side = 1;
        } else {
            xhi = x;
            fhi = fx;
            if (side == -1) flo *= 0.5f;
            side = -1;
        }
    }
    *v_ge = expf(xlo);
    *v_lt = expf(xhi);
}

__device__ void cut_speeds(float a, float r, float* v_out, float* v_in) {
    const float t_out = r * (1.f - 1e-4f), t_in = r * (1.f + 1e-4f);
    float ge, lt;
    crossing(a, t_out, v_bound(a, t_out), &ge, &lt);
    *v_out = lt;
    if (voigt_H(0.f, a) < t_in) {
        *v_in = -1.f;
        return;
    }
    crossing(a, t_in, v_bound(a, t_in), &ge, &lt);
    *v_in = ge < 0.f ? 0.f : ge;
}

// grid offsets d >= 0 at which |v| reaches vv, red side (d > 0: |v| = kv (1 - e^{-d lnq}))
// and blue side (|v| = kv (e^{d lnq} - 1)).
__device__ __forceinline__ float d_red(float vv, float kv, float lnq) {
    const float t = vv / kv;
    return t >= 1.f ? 1.0e9f : fminf(-log1pf(-t) / lnq, 1.0e9f);
}
__device__ __forceinline__ float d_blue(float vv, float kv, float lnq) { return fminf(log1pf(vv / kv) / lnq, 1.0e9f); }

constexpr unsigned char kDropped = 255;

// The tile kernel's constants of one kept (row, line), stored in bucket order so that a
// tile's candidates are one contiguous run of records (three 16-byte loads per line)
// instead of gathers from nine line-indexed arrays.
struct __align__(16) LineRec {
    int c;
    float f, kv, a;
    float srel;
    int jlo, jhi, ilo;
    int ihi, pad0, pad1, pad2;
};

struct PrepOut {
    int* c;
    float* f;
    float* srel;
    float* a;
    float* kv;
    int* jlo;
    int* jhi;
    int* ilo;
    int* ihi;
    unsigned char* cls;
    int* blkcnt;          // [n_sel][kNumClasses][nb]
    long long* wpart;     // [n_sel][nb]
    int* surv;            // [n_sel][L] lines left for the crossing search, each prep block's together
    int* nsurv;           // [n_sel] their number
};

// k_prep: one CTA of kPrepThreads threads per block of kPrepLines lines of one row.  Every line
// is tested: its peak against the cut threshold, then the cheap bound below on its window's
// reach.  The lines that remain are appended, as one run per block, to the row's list for
// k_windows; the others are marked dropped.  The block's class counts and window-length sum,
// which k_windows adds to, start at zero here.
__global__ void __launch_bounds__(kPrepThreads) k_prep(int64_t L, int N, float lnq, const int* __restrict__ species,
                                                       const int* __restrict__ cpos, const float* __restrict__ fpos,
                                                       int n_sp, const SpConst* __restrict__ sc,
                                                       const float* __restrict__ lnS, const float* __restrict__ av,
                                                       const float* __restrict__ lnk0, const float* __restrict__ ln_tp,
                                                       int nb, PrepOut o) {
    __shared__ short s_list[kPrepLines];
    __shared__ int s_n, s_base;
    const int s = blockIdx.y, lane = threadIdx.x & 31;
    const int64_t i0 = (int64_t)blockIdx.x * kPrepLines;
    if (threadIdx.x == 0) s_n = 0;
    if (threadIdx.x < kNumClasses) o.blkcnt[((size_t)s * kNumClasses + threadIdx.x) * nb + blockIdx.x] = 0;
    if (threadIdx.x == 0) o.wpart[(size_t)s * nb + blockIdx.x] = 0;
    __syncthreads();
    const float ltp = ln_tp[s];
    constexpr int kPer = kPrepLines / kPrepThreads;
    // every load of the thread's lines first, so they are in flight together
    float lk[kPer], ls[kPer], la[kPer], lf[kPer], lkv[kPer];
    int lc[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int64_t i = i0 + k * kPrepThreads + threadIdx.x;
        lk[k] = -INFINITY;
        if (i < L) {
            const size_t q = (size_t)s * L + i;
            lk[k] = lnk0[q];
            ls[k] = lnS[q];
            la[k] = av[q];
            lf[k] = fpos[i];
            lc[k] = cpos[i];
            lkv[k] = sc[(size_t)s * n_sp + species[i]].kv;
        }
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int off = k * kPrepThreads + threadIdx.x;
        const int64_t i = i0 + off;
        bool reach = false;
        if (i < L) {
            reach = lk[k] >= ltp;
            const int c = lc[k];
            if (reach && (c < -2 || c > N)) {
                // A centre off the grid: H(v, a) <= 4a/(sqrt(pi) v^2) + exp(-v^2/4) (the convolution
                // split at |t| = v/2), so the line stays below the cut beyond vb, with
                // 1/r = s_rel = e^rel, rel = ln S - ln t_p >= 0 (the peak passed).  The line is
                // kept if its bound window [c + f - d_blue(vb) - 2, c + f + d_red(vb) + 2] reaches
                // the grid; the grid side's offset is compared in FP32 (FP64 issues slowly on this
                // part) against an integer bound rounded towards keeping the line (k_windows drops
                // the few extra ones exactly).  Centres on the grid are kept without a test.
                const float rel = fminf(ls[k] - ltp, 88.f);
                const float a = la[k], kv = lkv[k], f = lf[k];
                const float vb =
                    fmaxf(sqrtf(8.f * kInvSqrtPi * a * expf(rel)), 2.f * sqrtf(fmaxf(0.69314718f + rel, 0.f))) + 1.f;
                if (c < -2) reach = fminf(f + d_red(vb, kv, lnq), 1.0e9f) >= __int2float_rd(-2 - c);
                else reach = fmaxf(f - d_blue(vb, kv, lnq), -1.0e9f) <= __int2float_ru(N + 1 - c);
            }
            // only kept lines are read later (through their bucket), so dropped ones write the class alone
            if (!reach) o.cls[(size_t)s * L + i] = kDropped;
        }
        const unsigned m = __ballot_sync(0xffffffffu, reach);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&s_n, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (reach) s_list[base + __popc(m & ((1u << lane) - 1u))] = (short)off;
    }
    __syncthreads();
    const int n = s_n;
    if (threadIdx.x == 0 && n > 0) s_base = atomicAdd(&o.nsurv[s], n);
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += kPrepThreads) o.surv[(size_t)s * L + s_base + t] = (int)(i0 + s_list[t]);
}

// k_windows: the outer and inner cut windows of every listed line (crossing searches on the
// FP32 H), its width class and window length.  Threads run over the row's list, so warps are
// dense whatever fraction of the lines the cheap bound kept.  The per-block class counts and
// window-length sums are integer atomics, combined first across the lanes of a warp that
// hold lines of the same prep block (a block's lines are one run of the list).
__global__ void __launch_bounds__(kPrepThreads) k_windows(int64_t L, int N, float lnq, const int* __restrict__ species,
                                                          const int* __restrict__ cpos, const float* __restrict__ fpos,
                                                          int n_sp, const SpConst* __restrict__ sc,
                                                          const float* __restrict__ lnS, const float* __restrict__ av,
                                                          const float* __restrict__ ln_tp, int nb, PrepOut o) {
    const int s = blockIdx.y, lane = threadIdx.x & 31;
    const int n = o.nsurv[s];
    const float ltp = ln_tp[s];
    const int stride = gridDim.x * kPrepThreads;
    // every lane of a warp runs the same number of passes (the warp-wide combining below)
    const int t0 = blockIdx.x * kPrepThreads + (threadIdx.x & ~31);
    for (int tw = t0; tw < n; tw += stride) {
        const int t = tw + lane;
        int blk = -1 - lane, key2 = -1;   // lanes past the list: a segment of their own
        long long w = 0;
        if (t < n) {
            const int64_t i = o.surv[(size_t)s * L + t];
            const size_t q = (size_t)s * L + i;
            blk = (int)(i / kPrepLines);
            const float rel = fminf(lnS[q] - ltp, 88.f);
            const float r = expf(-rel);
            const int c = cpos[i];
            const float f = fpos[i], a = av[q], kv = sc[(size_t)s * n_sp + species[i]].kv;
            unsigned char cl = kDropped;
            const float srel = expf(rel);
            float vo, vi;
            cut_speeds(a, r, &vo, &vi);
            const float vo2 = vo * (1.f + 1e-5f);
            long long hi = (long long)c + (long long)floorf(fminf(f + d_red(vo2, kv, lnq), 1.0e9f)) + 2;
            long long lo = (long long)c + (long long)ceilf(fmaxf(f - d_blue(vo2, kv, lnq), -1.0e9f)) - 2;
            hi = hi > N - 1 ? N - 1 : hi;
            lo = lo < 0 ? 0 : lo;
            if (lo <= hi) {
                const int jlo = (int)lo, jhi = (int)hi;
                int ilo = 1, ihi = 0;
                if (vi >= 0.f) {
                    const float vi2 = vi * (1.f - 1e-5f);
                    long long ih = (long long)c + (long long)floorf(fminf(f + d_red(vi2, kv, lnq), 1.0e9f)) - 2;
                    long long il = (long long)c + (long long)ceilf(fmaxf(f - d_blue(vi2, kv, lnq), -1.0e9f)) + 2;
                    ih = ih > jhi ? jhi : ih;
                    il = il < jlo ? jlo : il;
                    if (il <= ih) {
                        ilo = (int)il;
                        ihi = (int)ih;
                    }
                }
                const int key = c < -1 ? -1 : (c > N ? N : c);
                const int hw = max(jhi - key, key - jlo);
                cl = (unsigned char)(32 - __clz(hw));
                key2 = blk * kNumClasses + cl;
                w = (long long)(jhi - jlo + 1);
                o.c[q] = c;
                o.f[q] = f;
                o.srel[q] = srel;
                o.a[q] = a;
                o.kv[q] = kv;
                o.jlo[q] = jlo;
                o.jhi[q] = jhi;
                o.ilo[q] = ilo;
                o.ihi[q] = ihi;
            }
            o.cls[q] = cl;
        }
        // window-length sum of each prep block's run of lanes (runs are contiguous): segmented
        // inclusive scan, the run's last lane adds the total
        for (int d = 1; d < 32; d <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, d);
            const int yb = __shfl_up_sync(0xffffffffu, blk, d);
            if (lane >= d && yb == blk) w += y;
        }
        const int nextb = __shfl_down_sync(0xffffffffu, blk, 1);
        if (blk >= 0 && (lane == 31 || nextb != blk) && w > 0)
            atomicAdd((unsigned long long*)&o.wpart[(size_t)s * nb + blk], (unsigned long long)w);
        // kept lines per (prep block, class)
        const unsigned same = __match_any_sync(0xffffffffu, key2);
        if (key2 >= 0 && lane == __ffs(same) - 1)
            atomicAdd(&o.blkcnt[((size_t)s * kNumClasses + key2 % kNumClasses) * nb + blk], __popc(same));
    }
}

// k_scan_class: per (class, row), exclusive scan in place of the per-block counts of the
// class (one CTA each) and the class total.
__global__ void __launch_bounds__(1024) k_scan_class(int nb, int* __restrict__ blkcnt, int* __restrict__ classcnt) {
    __shared__ int wsum[32];
    __shared__ int carry;
    const int b = blockIdx.x, s = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int* row = blkcnt + ((size_t)s * kNumClasses + b) * nb;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        const int k = base + tid;
        const int v = k < nb ? row[k] : 0;
        int incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
            int ti = t;
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, ti, d);
                if (lane >= d) ti += y;
            }
            wsum[lane] = ti - t;
        }
        __syncthreads();
        const int c0 = carry;
        const int ex = c0 + wsum[warp] + incl - v;
        if (k < nb) row[k] = ex;
        __syncthreads();
        if (tid == (int)blockDim.x - 1) carry = ex + v;
        __syncthreads();
    }
    if (tid == 0) classcnt[s * kNumClasses + b] = carry;
}

// k_scan_fin: per row, the class base offsets and the total number of profile evaluations.
__global__ void __launch_bounds__(1024) k_scan_fin(int nb, const int* __restrict__ classcnt,
                                                   int* __restrict__ classbase, const long long* __restrict__ wpart,
                                                   long long* __restrict__ evals) {
    __shared__ long long wsum[32];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        int acc = 0;
        for (int b = 0; b < kNumClasses; ++b) {
            classbase[s * kNumClasses + b] = acc;
            acc += classcnt[s * kNumClasses + b];
        }
    }
    if (!evals) return;
    long long acc = 0;
    for (int k = tid; k < nb; k += blockDim.x) acc += wpart[(size_t)s * nb + k];
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (tid == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        evals[s] = t;
    }
}

// k_scatter: stable placement of kept lines into class buckets (centre order preserved), one
// CTA per prep block of kPrepLines lines; warp w takes the block's w-th run of consecutive
// lines.  A first pass counts each warp's lines per class, a scan over the warps gives the
// offsets, and a second pass places the lines.  A block that kept no line (window-length sum
// zero) returns at once.
__global__ void __launch_bounds__(kPrepThreads) k_scatter(int64_t L, int N, const unsigned char* __restrict__ cls,
                                                          const int* __restrict__ cpos, const int* __restrict__ blkoff,
                                                          const int* __restrict__ classbase, int nb,
                                                          int* __restrict__ bidx, int* __restrict__ bkey,
                                                          const PrepOut o, LineRec* __restrict__ rec) {
    constexpr int kWarps = kPrepThreads / 32, kGroups = kPrepLines / kPrepThreads;
    __shared__ int wcnt[kWarps][kNumClasses];
    const int s = blockIdx.y;
    if (o.wpart[(size_t)s * nb + blockIdx.x] == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < kWarps * kNumClasses; t += kPrepThreads) (&wcnt[0][0])[t] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * kPrepLines + (int64_t)warp * (32 * kGroups) + lane;
    const unsigned lt = (1u << lane) - 1u;
    int b[kGroups];
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
        const int64_t i = i0 + 32 * g;
        b[g] = (i < L) ? (int)cls[(size_t)s * L + i] : (int)kDropped;
        const unsigned same = __match_any_sync(0xffffffffu, b[g]);
        if (b[g] < kNumClasses && __popc(same & lt) == 0) wcnt[warp][b[g]] += __popc(same);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < kNumClasses) {
        int run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const int t = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
        const int64_t i = i0 + 32 * g;
        const int bg = b[g];
        const unsigned same = __match_any_sync(0xffffffffu, bg);
        const int lrank = __popc(same & lt);
        if (bg < kNumClasses) {
            const int pos = classbase[s * kNumClasses + bg] + blkoff[((size_t)s * kNumClasses + bg) * nb + blockIdx.x] +
                            wcnt[warp][bg] + lrank;
            const int c = cpos[i];
            bidx[(size_t)s * L + pos] = (int)i;
            bkey[(size_t)s * L + pos] = c < -1 ? -1 : (c > N ? N : c);
            const size_t q = (size_t)s * L + i;
            LineRec r;
            r.c = o.c[q];
            r.f = o.f[q];
            r.kv = o.kv[q];
            r.a = o.a[q];
            r.srel = o.srel[q];
            r.jlo = o.jlo[q];
            r.jhi = o.jhi[q];
            r.ilo = o.ilo[q];
            r.ihi = o.ihi[q];
            r.pad0 = r.pad1 = r.pad2 = 0;
            rec[(size_t)s * L + pos] = r;
        }
        __syncwarp();
        if (bg < kNumClasses && lrank == 0) wcnt[warp][bg] += __popc(same);
        __syncwarp();
    }
}

// k_ranges: cum[s][b][ts] = position of the first line of class b whose centre key is
// >= (ts - 1) * kTile, ts = 0 .. nT + 2 (tiles -1 .. nT, with off-grid centres clamped).
__global__ void k_ranges(int n_sel, int64_t L, int nT, int tile, const int* __restrict__ bkey,
                         const int* __restrict__ classbase, const int* __restrict__ classcnt, int* __restrict__ cum) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int W = nT + 3;
    if (t >= (int64_t)n_sel * kNumClasses * W) return;
    const int ts = (int)(t % W);
    const int b = (int)((t / W) % kNumClasses);
    const int s = (int)(t / ((int64_t)W * kNumClasses));
    const int base = classbase[s * kNumClasses + b], n = classcnt[s * kNumClasses + b];
    const int* k = bkey + (size_t)s * L + base;
    const long long thr = (long long)(ts - 1) * tile;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)k[mid] < thr) lo = mid + 1; else hi = mid;
    }
    cum[t] = base + lo;
}

// ---------------------------------------------------------------------------
// The profile kernel.  A tile of PTS * THREADS grid points is processed by one CTA:
// thread t owns the points J0 + k THREADS + t, k = 0..PTS-1.
struct RowDesc {
    int N, nT, tile;
    float lnq, q1, q2, q3;      // expm1(-x)/(-x) ~ 1 + d (q1 + d (q2 + d q3)), x = d lnq
    const float* ln_tp;         // ln of the cut threshold t_p (outputs are t_p * sum of s_rel H)
    const int* cum;             // [kNumClasses][nT + 3]
    const int* bidx;            // [L] bucketed line indices
    const LineRec* rec;         // [L] their constants, in the same order
    const int* c;
    const float* f;
    const float* srel;
    const float* a;
    const float* kv;
    const int* jlo;
    const int* jhi;
    const int* ilo;
    const int* ihi;
    float* out;                 // [N]
};

// flag bits of the per-line records in shared memory
constexpr int kFlKloBits = 5;
constexpr int kFlMask = (1 << kFlKloBits) - 1;
constexpr int kFlChk = 1 << 10;      // points near the cut: test s_rel H >= 1
constexpr int kFlAlt = 1 << 11;      // far: "y" form; near: expm1 series for v
constexpr int kFlFull = 1 << 12;     // the window covers every slot of the tile
constexpr int kFlRat = 1 << 13;      // far: rational form sk / (|z|^2 - 3/2)
constexpr int kFlScaled = 1 << 14;   // far, rational: the line may be evaluated in units of sk (far_rat_pairs_scaled)

struct NearRec {
    float cf, f, klnq, a, srel, kv;
    int flags;
    int jlo, jhi;    // outer cut window (grid indices)
    int pad[3];
};

// far line, three forms (sk = s_rel a / sqrt(pi)).  v = G_k * (kv B) + kv E1 is the exact
// expm1 split of the frequency offset around the tile start.
//  * kFarRat, "rational": s_rel H = sk / (|z|^2 - 3/2), |z|^2 = v^2 + a^2.  Its relative
//    error against H is below (2 + 2a^2)/|z|^4 (the asymptotic series of H to order |z|^-4),
//    so it is used where that bound is <= 1e-6 over the whole tile: 3 FFMA + 1 reciprocal.
//    p = {kv B, kv E1, a^2 - 3/2, sk}.
//  * kFarExact: the one-level continued fraction without truncation, with
//    v' = sqrt2 v and D = v'^2 + 2a^2 - 1 = 2|z|^2 - 1:
//    s_rel H = (2 sk D + 4 sk) / (D^2 + 8 a^2): 5 FFMA + 1 reciprocal.
//  * kFarY: where D^2 could overflow FP32 (|v| >= 1e9 somewhere in the tile),
//    y = 1/D, s_rel H = sk y (2 + 4 y); there 8 a^2 y^2 is far below 1e-8.
//    p = {sqrt2 kv B, sqrt2 kv E1, 2a^2 - 1, 8a^2}, q = {2 sk, 4 sk} for both.
// The PTS points are evaluated without branches so that their dependency chains
// interleave; MASKED lines (partial coverage or points near the cut) select with a mask.
constexpr int kFarRat = 0, kFarExact = 1, kFarY = 2;

template <int PTS, int FORM, bool MASKED>
__device__ __forceinline__ void far_line(const float4 p, const float2 q, int klo, int khi, bool chk,
                                         const float (&G)[PTS], float (&part)[PTS]) {
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
        const float vp = fmaf(G[k], p.x, p.y);
        const float D = fmaf(vp, vp, p.z);
        float t, y;
        if (FORM == kFarRat) {
            y = rcp_approx(D);
            t = p.w;
        } else if (FORM == kFarY) {
            y = rcp_approx(D);
            t = fmaf(q.y, y, q.x);
        } else {
            y = rcp_approx(fmaf(D, D, p.w));
            t = fmaf(q.x, D, q.y);
        }
        if (MASKED) {
            const float l = t * y;
            bool ok = (k >= klo) & (k <= khi);
            if (chk) ok = ok & (l >= 1.f);
            part[k] += ok ? l : 0.f;
        } else {
            part[k] = fmaf(t, y, part[k]);
        }
    }
}

// packed FP32: two lanes per instruction, rounded like fmaf
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// plain line in the rational form, two points per reciprocal, in packed FP32.  The
// thread's points are taken as pairs (2j, 2j+1): v and D = v^2 + a^2 - 3/2 of both points
// in one packed FFMA each, r = 1/(D_0 D_1) and, with sr = sk r,
// sk/D_0 = sr D_1 and sk/D_1 = sr D_0 (about two ulps) in one packed FFMA into the pair's
// partial sums, held as {part_{2j+1}, part_{2j}}.  Per pair: three packed FFMAs and two
// FMULs on the FMA pipe (8 lane operations) and one reciprocal.  D_0 D_1 < 1e36 stays finite
// because the form is used only where |v| < 1e9 on the whole tile.
// u = {kv B, kv B, kv E1, kv E1}, w = {a^2 - 3/2, a^2 - 3/2, sk, sk} (duplicated so that
// each operand pair comes straight from one 16-byte shared-memory load).
template <int PTS>
__device__ __forceinline__ void far_rat_pairs(const float4 u, const float4 w, const float (&G)[PTS],
                                              float (&part)[PTS]) {
    static_assert(PTS % 2 == 0, "points are taken in pairs");
    const float2 B2 = make_float2(u.x, u.y), E2 = make_float2(u.z, u.w), C2 = make_float2(w.x, w.y);
    const float sk = w.z;
#pragma unroll
    for (int j = 0; j < PTS / 2; ++j) {
        const float2 v = ffma2(make_float2(G[2 * j], G[2 * j + 1]), B2, E2);
        const float2 D = ffma2(v, v, C2);
        const float P01 = D.x * D.y;
        float2 acc = make_float2(part[2 * j + 1], part[2 * j]);
        const float sr = sk * rcp_approx(P01);
        acc = ffma2(make_float2(sr, sr), D, acc);
        part[2 * j + 1] = acc.x;
        part[2 * j] = acc.y;
    }
}

// plain line in the rational form, in units of sk: with v' = v / sqrt(sk) and
// D' = v'^2 + (a^2 - 3/2)/sk = D/sk, the contribution sk/D is 1/D', so the factor sk leaves
// the inner loop: r = 1/(D'_0 D'_1), 1/D'_0 = r D'_1, 1/D'_1 = r D'_0.  Per pair: three
// packed FFMAs and one FMUL (7 lane operations) and one reciprocal.  Used for lines with
// sk <= 1e18 D_min and |v|_max <= 1e9 sqrt(sk) on the tile, so that every D' lies in
// [1e-18, 1e18] and the products stay normal FP32 numbers.
// u = {B', B', E', E'} = {kv B, kv B, kv E1, kv E1} / sqrt(sk), w = {c', c', -, -}.
template <int PTS>
__device__ __forceinline__ void far_rat_pairs_scaled(const float4 u, const float4 w, const float (&G)[PTS],
                                                     float (&part)[PTS]) {
    static_assert(PTS % 2 == 0, "points are taken in pairs");
    const float2 B2 = make_float2(u.x, u.y), E2 = make_float2(u.z, u.w), C2 = make_float2(w.x, w.y);
#pragma unroll
    for (int j = 0; j < PTS / 2; ++j) {
        const float2 v = ffma2(make_float2(G[2 * j], G[2 * j + 1]), B2, E2);
        const float2 D = ffma2(v, v, C2);
        const float r = rcp_approx(D.x * D.y);
        const float2 acc = ffma2(make_float2(r, r), D, make_float2(part[2 * j + 1], part[2 * j]));
        part[2 * j + 1] = acc.x;
        part[2 * j] = acc.y;
    }
}

// near line: exact offset d = (j - c) - f and the expm1 series for v; the tiers of H
// branch per point.  Lines that do not cover the whole tile are culled per warp in
// 32-point segments (a warp's lanes own 32 consecutive points of each slot).  The coverage
// and cut-test flags are runtime arguments: one copy of this code instead of four template
// copies measured 1.1 % faster on the 8-row table step (less instruction-cache pressure).
template <int PTS, int THREADS>
__device__ __forceinline__ void near_line(const NearRec& r, int seg0, bool series, bool full, bool chk,
                                          const float (&jf)[PTS], float q1, float q2, float q3, float lnq,
                                          float (&part)[PTS]) {
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
        if (!full) {
            const int lo = seg0 + k * THREADS;
            if (lo + 31 < r.jlo || lo > r.jhi) continue;
        }
        const float d = (jf[k] - r.cf) - r.f;
        float v;
        if (series) v = r.klnq * (d * fmaf(d, fmaf(d, fmaf(d, q3, q2), q1), 1.f));
        else v = r.kv * expm1f(-d * lnq);
        float l = r.srel * voigt_H_lean(v, r.a);
        if (chk) l = (l >= 1.f) ? l : 0.f;
        part[k] += l;
    }
}

// One tile of one row.  Called by the grid kernel (one tile per CTA, or S CTAs per tile that
// take every S-th chunk of the tile's candidate lines, sp = 0..S-1, when a call has too few
// tiles to fill the GPU) and by the persistent kernel (a loop over a work list).
template <int PREC, int PTS, int THREADS>
__device__ __forceinline__ void tile_body(const RowDesc& g, int tile, int sp = 0, int S = 1) {
    constexpr int TILE = PTS * THREADS;
    __shared__ float4 sFarA[THREADS];
    __shared__ float4 sFarB[THREADS];
    __shared__ NearRec sNear[THREADS];
    __shared__ int sCnt[6][THREADS / 32];

    const int J0 = tile * TILE;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // Kahan totals live in shared memory ([point][thread], conflict-free): they change once
    // per chunk, and keeping them out of registers lets more CTAs share an SM
    __shared__ float sSum[PREC == MPSA_PREC_FP32_COMPENSATED ? PTS : 1][THREADS];
    __shared__ float sComp[PREC == MPSA_PREC_FP32_COMPENSATED ? PTS : 1][THREADS];
    float jf[PTS], G[PTS], part[PTS];
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
        const int off = k * THREADS + tid;
        jf[k] = (float)(J0 + off);
        G[k] = expm1f(-(float)off * g.lnq);
        if (PREC == MPSA_PREC_FP32_COMPENSATED) {
            sSum[k][tid] = 0.f;
            sComp[k][tid] = 0.f;
        }
        part[k] = 0.f;
    }

    int chunk = 0;   // running chunk index over the classes: this CTA takes chunk % S == sp
    for (int b = 0; b < kNumClasses; ++b) {
        const int reach = 1 << b;
        int tlo = floordiv(J0 - reach + 1, TILE), thi = floordiv(J0 + TILE - 1 + reach - 1, TILE);
        tlo = max(tlo, -1);
        thi = min(thi, g.nT);
        if (tlo > thi) continue;
        const int* cum = g.cum + (size_t)b * (g.nT + 3);
        const int beg = cum[tlo + 1], end = cum[thi + 2];
        for (int base = beg; base < end; base += THREADS) {
            if (chunk++ % S != sp) continue;   // CTA-uniform
            // ---- set-up: one candidate line per thread
            const int pos = base + tid;
            bool isFar = false, isNear = false;
            float4 fa, fb;
            NearRec nr;
            if (pos < end) {
                const int4* rp = reinterpret_cast<const int4*>(g.rec + pos);
                const int4 r0 = __ldg(rp), r1 = __ldg(rp + 1), r2 = __ldg(rp + 2);
                const int jlo = r1.y, jhi = r1.z;
                if (jhi >= J0 && jlo <= J0 + TILE - 1) {
                    const int c = r0.x;
                    const float f = __int_as_float(r0.y), kv = __int_as_float(r0.z), a = __int_as_float(r0.w),
                                srel = __int_as_float(r1.x);
                    const int klo = max(0, (jlo - J0) / THREADS), khi = min(PTS - 1, (jhi - J0) / THREADS);
                    const int P0 = J0 + klo * THREADS, P1 = J0 + khi * THREADS + THREADS - 1;
                    const bool check = !(r1.w <= P0 && r2.x >= P1);
                    // distance from the centre x0 = c + f to the nearest point of the tile
                    // (far lines are evaluated at all points, masked to [klo, khi])
                    const int T0 = J0, T1 = J0 + TILE - 1;
                    float dist;
                    bool red;
                    if (c + 1 <= T0) { dist = (float)(T0 - c) - f; red = true; }
                    else if (c >= T1) { dist = f + (float)(c - T1); red = false; }
                    else { dist = 0.f; red = true; }
                    float vmin = 0.f;
                    if (dist >= (float)kFarDist)
                        vmin = red ? -kv * expm1f(-dist * g.lnq) : kv * expm1f(dist * g.lnq);
                    const int flags = klo | (khi << kFlKloBits) | (check ? kFlChk : 0) |
                                      ((klo == 0 && khi == PTS - 1) ? kFlFull : 0);
                    if (dist >= (float)kFarDist && vmin >= kFarV) {
                        isFar = true;
                        // a far line whose windows reach the grid's last point counts as covering
                        // the tile there: the points past the grid's end (last tile only) are
                        // evaluated but never stored, so narrow grids keep the unmasked forms
                        const int Te = min(T1, g.N - 1);
                        const int khf = jhi >= Te ? PTS - 1 : khi;
                        const bool chf = !(r1.w <= P0 && r2.x >= min(J0 + khf * THREADS + THREADS - 1, Te));
                        const int ff = klo | (khf << kFlKloBits) | (chf ? kFlChk : 0) |
                                       ((klo == 0 && khf == PTS - 1) ? kFlFull : 0);
                        const float D = (float)(J0 - c) - f;
                        const float x = D * g.lnq;
                        const float E1 = expm1f(-x), B = expf(-x);
                        const float A = a * a;
                        const float r2 = 1.41421356237309505f;
                        // the largest |v| on the tile (both ends) decides between the two forms
                        const float xe = ((float)(J0 + TILE - 1 - c) - f) * g.lnq;
                        const float vmax = fmaxf(fabsf(kv * E1), fabsf(kv * expm1f(-xe)));
                        const bool yform = vmax >= 1.0e9f;
                        const float sk = srel * a * kInvSqrtPi;
                        // rational form where (2 + 2a^2) / |z|^4 <= 1e-6 at the tile's nearest point
                        const float zmin2 = fmaf(vmin, vmin, A);
                        if (zmin2 * zmin2 >= 1.0e6f * fmaf(2.f, A, 2.f)) {
                            fa = make_float4(kv * B, kv * E1, A - 1.5f, sk);
                            // every D/sk of the tile within [1e-18, 1e18]: the form in units of sk
                            const bool scaled = sk <= 1.0e18f * (zmin2 - 1.5f) && vmax <= 1.0e9f * sqrtf(sk);
                            fb = make_float4(0.f, 0.f,
                                             __int_as_float(ff | kFlRat | (yform ? kFlAlt : 0) |
                                                            (scaled ? kFlScaled : 0)),
                                             0.f);
                        } else {
                            fa = make_float4(r2 * kv * B, r2 * kv * E1, fmaf(2.f, A, -1.f), 8.f * A);
                            fb = make_float4(2.f * sk, 4.f * sk, __int_as_float(ff | (yform ? kFlAlt : 0)), 0.f);
                        }
                    } else {
                        isNear = true;
                        const float dmax = fmaxf(fabsf((float)(P0 - c) - f), fabsf((float)(P1 - c) - f));
                        const bool series = dmax * g.lnq <= 0.05f;
                        nr.cf = (float)c;
                        nr.f = f;
                        nr.klnq = kv * g.lnq;
                        nr.a = a;
                        nr.srel = srel;
                        nr.kv = kv;
                        nr.flags = flags | (series ? kFlAlt : 0);
                        nr.jlo = jlo;
                        nr.jhi = jhi;
                        nr.pad[0] = nr.pad[1] = nr.pad[2] = 0;
                    }
                }
            }
            // far lines are compacted into five lists: plain rational in units of sk, plain
            // rational with two points per reciprocal (the few lines the scaled form cannot
            // take), plain "exact" and plain "y" forms, and masked (partial coverage or cut
            // test), so the hot loops dispatch nothing; near lines into a sixth
            constexpr int kNearCat = 5;
            int cat = -1;
            if (isFar) {
                const int fl = __float_as_int(fb.z);
                const bool plain = (fl & kFlFull) && !(fl & kFlChk);
                // rational lines with |v| >= 1e9 somewhere take the single-reciprocal masked path
                // rational lines: in units of sk where allowed (list 0), else two points per
                // reciprocal where |v| < 1e9 (list 1), else the single-reciprocal masked path
                cat = !plain ? 4
                             : ((fl & kFlRat) ? ((fl & kFlScaled) ? 0 : ((fl & kFlAlt) ? 4 : 1))
                                              : ((fl & kFlAlt) ? 3 : 2));
            } else if (isNear) {
                cat = kNearCat;
            }
            unsigned bm = 0u;
#pragma unroll
            for (int q = 0; q <= kNearCat; ++q) {
                const unsigned b = __ballot_sync(0xffffffffu, cat == q);
                if (cat == q) bm = b;
                if (lane == 0) sCnt[q][warp] = __popc(b);
            }
            __syncthreads();
            int off = 0, tot[kNearCat + 1] = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int w = 0; w < THREADS / 32; ++w) {
#pragma unroll
                for (int q = 0; q <= kNearCat; ++q) {
                    const int cnt = sCnt[q][w];
                    if (w < warp && q == cat) off += cnt;
                    tot[q] += cnt;
                }
            }
            const unsigned lt = (1u << lane) - 1u;
            if (cat >= 0 && cat < kNearCat) {
                int base2 = 0;
#pragma unroll
                for (int q = 0; q < kNearCat - 1; ++q)
                    if (q < cat) base2 += tot[q];
                const int p = base2 + off + __popc(bm & lt);
                if (cat == 0) {
                    const float rs = 1.f / sqrtf(fa.w), c1 = fa.z / fa.w;
                    sFarA[p] = make_float4(fa.x * rs, fa.x * rs, fa.y * rs, fa.y * rs);
                    sFarB[p] = make_float4(c1, c1, 0.f, 0.f);
                } else if (cat <= 1) {
                    sFarA[p] = make_float4(fa.x, fa.x, fa.y, fa.y);
                    sFarB[p] = make_float4(fa.z, fa.z, fa.w, fa.w);
                } else {
                    sFarA[p] = fa;
                    sFarB[p] = fb;
                }
            }
            if (cat == kNearCat) sNear[off + __popc(bm & lt)] = nr;
            const int nNear = tot[kNearCat];
            __syncthreads();

            // ---- evaluation: every thread, every compacted line, its PTS points
            {
                int r = 0;
                // two lines per iteration: half the loop overhead, and two independent
                // dependency chains per point for the scheduler
                for (; r + 1 < tot[0]; r += 2) {
                    const float4 ua = sFarA[r], wa = sFarB[r], ub = sFarA[r + 1], wb = sFarB[r + 1];
                    far_rat_pairs_scaled<PTS>(ua, wa, G, part);
                    far_rat_pairs_scaled<PTS>(ub, wb, G, part);
                }
                if (r < tot[0]) {
                    far_rat_pairs_scaled<PTS>(sFarA[r], sFarB[r], G, part);
                    ++r;
                }
                const int e1 = tot[0] + tot[1];
                for (; r + 1 < e1; r += 2) {
                    const float4 ua = sFarA[r], wa = sFarB[r], ub = sFarA[r + 1], wb = sFarB[r + 1];
                    far_rat_pairs<PTS>(ua, wa, G, part);
                    far_rat_pairs<PTS>(ub, wb, G, part);
                }
                if (r < e1) {
                    far_rat_pairs<PTS>(sFarA[r], sFarB[r], G, part);
                    ++r;
                }
                for (; r < e1 + tot[2]; ++r) {
                    const float4 q4 = sFarB[r];
                    far_line<PTS, kFarExact, false>(sFarA[r], make_float2(q4.x, q4.y), 0, PTS - 1, false, G, part);
                }
                for (; r < e1 + tot[2] + tot[3]; ++r) {
                    const float4 q4 = sFarB[r];
                    far_line<PTS, kFarY, false>(sFarA[r], make_float2(q4.x, q4.y), 0, PTS - 1, false, G, part);
                }
                for (; r < e1 + tot[2] + tot[3] + tot[4]; ++r) {
                    const float4 p = sFarA[r];
                    const float4 q4 = sFarB[r];
                    const float2 q = make_float2(q4.x, q4.y);
                    const int fl = __float_as_int(q4.z);
                    const int klo = fl & kFlMask, khi = (fl >> kFlKloBits) & kFlMask;
                    const bool chk = fl & kFlChk;
                    if (fl & kFlRat) far_line<PTS, kFarRat, true>(p, q, klo, khi, chk, G, part);
                    else if (fl & kFlAlt) far_line<PTS, kFarY, true>(p, q, klo, khi, chk, G, part);
                    else far_line<PTS, kFarExact, true>(p, q, klo, khi, chk, G, part);
                }
            }
            const int seg0 = J0 + warp * 32;
            for (int r = 0; r < nNear; ++r) {
                const NearRec nrr = sNear[r];
                const bool series = nrr.flags & kFlAlt;
                const bool full = nrr.flags & kFlFull, chk = nrr.flags & kFlChk;
                near_line<PTS, THREADS>(nrr, seg0, series, full, chk, jf, g.q1, g.q2, g.q3, g.lnq, part);
            }
            if (PREC == MPSA_PREC_FP32_COMPENSATED) {
                // fold the chunk's FP32 partial sums into the Kahan-compensated totals
#pragma unroll
                for (int k = 0; k < PTS; ++k) {
                    const float s0 = sSum[k][tid], c0 = sComp[k][tid];
                    const float y = part[k] - c0;
                    const float t = s0 + y;
                    sComp[k][tid] = (t - s0) - y;
                    sSum[k][tid] = t;
                    part[k] = 0.f;
                }
            }
            __syncthreads();
        }
    }
    const float tp = expf(*g.ln_tp);
#pragma unroll
    for (int k = 0; k < PTS; ++k) {
        const int j = J0 + k * THREADS + tid;
        const float tot = (PREC == MPSA_PREC_FP32_COMPENSATED) ? (sSum[k][tid] - sComp[k][tid]) : part[k];
        if (j < g.N) g.out[j] = tp * tot;
    }
}

// Grid form: one CTA per (row, tile); the rows of one call share the prep arrays.
struct TileArgs {
    int N, nT;
    int64_t L;
    float lnq, q1, q2, q3;
    const int* cum;
    const int* bidx;
    const LineRec* rec;
    const int* c;
    const float* f;
    const float* srel;
    const float* a;
    const float* kv;
    const int* jlo;
    const int* jhi;
    const int* ilo;
    const int* ihi;
    const float* ln_tp;
    float* out;
    int split;       // CTAs per tile (1: direct output)
    float* part;     // split > 1: partial sums [n_sel][split][N], added by k_split_sum
};

__device__ __forceinline__ RowDesc row_desc(const TileArgs& g, int s, int tile) {
    const size_t sL = (size_t)s * g.L;
    RowDesc r;
    r.N = g.N;
    r.nT = g.nT;
    r.tile = tile;
    r.lnq = g.lnq;
    r.q1 = g.q1;
    r.q2 = g.q2;
    r.q3 = g.q3;
    r.ln_tp = g.ln_tp + s;
    r.cum = g.cum + (size_t)s * kNumClasses * (g.nT + 3);
    r.bidx = g.bidx + sL;
    r.rec = g.rec + sL;
    r.c = g.c + sL;
    r.f = g.f + sL;
    r.srel = g.srel + sL;
    r.a = g.a + sL;
    r.kv = g.kv + sL;
    r.jlo = g.jlo + sL;
    r.jhi = g.jhi + sL;
    r.ilo = g.ilo + sL;
    r.ihi = g.ihi + sL;
    r.out = g.out + (size_t)s * g.N;
    return r;
}

#ifndef MPSA_TILES_MINB
#define MPSA_TILES_MINB 4
#endif
// SPLIT: g.split CTAs per tile, each writing its partial sums to g.part (a separate
// instantiation, so that the one-CTA-per-tile form compiles as it would without it)
template <int PREC, bool SPLIT>
__global__ void __launch_bounds__(kTileThreads, MPSA_TILES_MINB) k_tiles(TileArgs g) {
    RowDesc r = row_desc(g, blockIdx.y, kTile);
    if (SPLIT) {
        const int sp = blockIdx.x % g.split;
        r.out = g.part + ((size_t)blockIdx.y * g.split + sp) * g.N;
        tile_body<PREC, kPtsPerThread, kTileThreads>(r, blockIdx.x / g.split, sp, g.split);
    } else {
        tile_body<PREC, kPtsPerThread, kTileThreads>(r, blockIdx.x);
    }
}

// kappa[s][j] = sum over the split CTAs' partial sums (FP64 sum, one rounding to FP32)
__global__ void k_split_sum(int n_sel, int N, int split, const float* __restrict__ part, float* __restrict__ kappa) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_sel * N) return;
    const int s = (int)(t / N), j = (int)(t % N);
    double acc = 0.0;
    for (int q = 0; q < split; ++q) acc += part[((size_t)s * split + q) * N + j];
    kappa[t] = (float)acc;
}

// Persistent form: a fixed grid of CTAs pulls (row, tile) units from a work list
// (ordered by decreasing estimated cost) through one global counter.
template <int PREC, int PTS, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_tiles_persistent(const RowDesc* __restrict__ rows,
                                                                   const int2* __restrict__ units, int n_units,
                                                                   int* __restrict__ counter) {
    __shared__ int s_unit;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_unit;
        __syncthreads();
        if (u >= n_units) break;
        const int2 rt = units[u];
        const RowDesc r = rows[rt.x];
        tile_body<PREC, PTS, THREADS>(r, rt.y);
    }
}

// ---------------------------------------------------------------------------
// All-FP64 variant of the profile kernel (precision study): line terms of Eq. (l_nu_line),
// the exact frequency offset v = (c/lambda_j - nu0)/dnuD and H in FP64, plain FP64 sums.
// Same candidate lines and outer windows as the FP32 kernel; the cut threshold is the FP32
// one (t_p = exp(ln t_p)), so inclusion decisions differ only inside the edge slack band.
struct Tile64Args {
    TileArgs t;
    const int* sel;
    const double* pop;
    int pop_stride_;
    int n_sp;
    const int* sp_el;
    const int* sp_stage;
    const double* el;          // [n_el][kElStride] element records
    int n_el;
    double vturb;
    const double* lam_nm;      // line list
    const float* loggf;
    const float* E;
    const float* lgR;
    const float* lgS;
    const float* lgW;
    const int* species;
    double lam0_nm, lnq64;
};

// All-FP64 variant: one point per thread (256-point tiles, so that narrow grids still fill
// the GPU), line constants in FP64 per (line, tile), FP64 Voigt tiers.
constexpr int kTile64 = 256;
__global__ void __launch_bounds__(256) k_tiles64(Tile64Args g) {
    constexpr int THREADS = 256, PTS = 1, TILE = THREADS * PTS;
    static_assert(TILE == kTile64, "FP64 tile size");
    __shared__ double sS[THREADS], sA[THREADS], sNu[THREADS], sDnu[THREADS];
    __shared__ int sLo[THREADS], sHi[THREADS];
    __shared__ int sN;
    const int s = blockIdx.y, tile = blockIdx.x, tid = threadIdx.x;
    const RowDesc r = row_desc(g.t, s, kTile64);
    const int J0 = tile * TILE;
    const double* row = g.pop + (size_t)g.sel[s] * g.pop_stride_;
    const double T = row[kPopT], ne = row[kPopNe], nHI = row[kPopNHI], rho = row[kPopRho];
    const double tp = exp((double)*r.ln_tp);
    double nu[PTS], acc[PTS];
    for (int k = 0; k < PTS; ++k) {
        const int j = J0 + k * THREADS + tid;
        nu[k] = kC / (g.lam0_nm * exp((double)j * g.lnq64) * 1e-7);
        acc[k] = 0.0;
    }
    const double pre = sqrt(kPI) * kE * kE / (kME * kC);
    for (int b = 0; b < kNumClasses; ++b) {
        const int reach = 1 << b;
        int tlo = max(floordiv(J0 - reach + 1, TILE), -1), thi = min(floordiv(J0 + TILE - 1 + reach - 1, TILE), r.nT);
        if (tlo > thi) continue;
        const int* cum = r.cum + (size_t)b * (r.nT + 3);
        const int beg = cum[tlo + 1], end = cum[thi + 2];
        for (int base = beg; base < end; base += THREADS) {
            if (tid == 0) sN = 0;
            __syncthreads();
            const int pos = base + tid;
            if (pos < end) {
                const int q = r.bidx[pos];
                const int jlo = r.jlo[q], jhi = r.jhi[q];
                if (jhi >= J0 && jlo <= J0 + TILE - 1) {
                    const int sp = g.species[q];
                    const int e = g.sp_el[sp], st = g.sp_stage[sp];
                    const double lam = g.lam_nm[q] * 1e-7;
                    const double nu0 = kC / lam;
                    const double u = sqrt(2.0 * kKB * T / (g.el[e * kElStride + kElMass] * kAMU) + g.vturb * g.vturb);
                    const double dnu = nu0 * u / kC;
                    const double gam = pow(10.0, (double)g.lgR[q]) + pow(10.0, (double)g.lgS[q]) * ne +
                                       pow(10.0, (double)g.lgW[q]) * nHI;
                    const double NU = row[pop_nu(e, st)];
                    const double S = pre * pow(10.0, (double)g.loggf[q]) * NU / (rho * dnu) *
                                     exp(-(double)g.E[q] * kEV / (kKB * T)) * (-expm1(-kH * nu0 / (kKB * T)));
                    const int slot = atomicAdd(&sN, 1);
                    sS[slot] = S;
                    sA[slot] = gam / (4.0 * kPI * dnu);
                    sNu[slot] = nu0;
                    sDnu[slot] = 1.0 / dnu;
                    sLo[slot] = jlo;
                    sHi[slot] = jhi;
                }
            }
            __syncthreads();
            const int n = sN;
            for (int i = 0; i < n; ++i) {
                const double S = sS[i], a = sA[i], nu0 = sNu[i], inv_dnu = sDnu[i];
                const int lo = sLo[i], hi = sHi[i];
                for (int k = 0; k < PTS; ++k) {
                    const int j = J0 + k * THREADS + tid;
                    if (j < lo || j > hi) continue;
                    const double l = S * voigt_H64((nu[k] - nu0) * inv_dnu, a);
                    if (l >= tp) acc[k] += l;
                }
            }
            __syncthreads();
        }
    }
    for (int k = 0; k < PTS; ++k) {
        const int j = J0 + k * THREADS + tid;
        if (j < r.N) r.out[j] = (float)acc[k];
    }
}

int g_init_mask = 0;

__global__ void k_voigt_eval(int64_t n, const double* __restrict__ v, const double* __restrict__ a, bool fp64,
                             double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = fp64 ? voigt_H64(v[i], a[i]) : (double)voigt_H((float)v[i], (float)a[i]);
}

}  // namespace

int synth_module_init(int device) {
    if (device < 0 || device >= 31) return fail(MPSA_EINVAL, "device %d", device);
    if (g_init_mask & (1 << device)) return MPSA_OK;
    int rc = voigt_upload();
    if (rc != MPSA_OK) return rc;
    g_init_mask |= 1 << device;
    return MPSA_OK;
}

// Shared by synth_opacity and synth_spectrum: synthesis for rows `sel` of a
// population table `pop` onto grid (lam0, R, N); writes kappa [n_sel][N].
// Device buffers of the line preparation of n_sel rows (one grid, one tile size).
struct PrepBufs {
    int64_t L = 0;
    int n_sel = 0, N = 0, nT = 0, nb = 0, tile = kTile;
    double lnq = 0.0;
    int *c = nullptr, *bidx = nullptr, *bkey = nullptr, *blkcnt = nullptr, *classbase = nullptr, *classcnt = nullptr,
        *cum = nullptr;
    LineRec* rec = nullptr;
    float *f = nullptr, *lamcm = nullptr, *lnS = nullptr, *av = nullptr, *lnk0 = nullptr, *ln_tp = nullptr;
    RowConst* rc = nullptr;
    SpConst* spc = nullptr;
    long long* wpart = nullptr;
    MedState* med = nullptr;
    unsigned* ghist = nullptr;
    PrepOut po{};
};

// Allocate every prep buffer through `al` (stream-ordered scratch or persistent memory).
template <class Alloc>
int prep_alloc(PrepBufs& b, const mpsa_ctx* ctx, int n_sel, int N, double R, int tile, Alloc&& al) {
    b.L = ctx->L;
    b.n_sel = n_sel;
    b.N = N;
    b.tile = tile;
    b.nT = (N + tile - 1) / tile;
    b.nb = (int)((b.L + kPrepLines - 1) / kPrepLines);
    b.lnq = log1p(1.0 / R);
    const int64_t L = b.L;
    const size_t SL = (size_t)n_sel * L;
    int r;
    if ((r = al(&b.c, L)) || (r = al(&b.f, L)) || (r = al(&b.lamcm, L)) || (r = al(&b.rc, n_sel)) ||
        (r = al(&b.spc, (size_t)n_sel * ctx->n_sp)) || (r = al(&b.lnS, SL)) || (r = al(&b.av, SL)) ||
        (r = al(&b.lnk0, SL)) || (r = al(&b.ln_tp, n_sel)) || (r = al(&b.po.c, SL)) || (r = al(&b.po.f, SL)) ||
        (r = al(&b.po.srel, SL)) || (r = al(&b.po.a, SL)) || (r = al(&b.po.kv, SL)) || (r = al(&b.po.jlo, SL)) ||
        (r = al(&b.po.jhi, SL)) || (r = al(&b.po.ilo, SL)) || (r = al(&b.po.ihi, SL)) || (r = al(&b.po.cls, SL)) ||
        (r = al(&b.blkcnt, (size_t)n_sel * kNumClasses * b.nb)) || (r = al(&b.wpart, (size_t)n_sel * b.nb)) ||
        (r = al(&b.classbase, (size_t)n_sel * kNumClasses)) || (r = al(&b.classcnt, (size_t)n_sel * kNumClasses)) ||
        (r = al(&b.bidx, SL)) || (r = al(&b.bkey, SL)) || (r = al(&b.rec, SL)) ||
        (r = al(&b.cum, (size_t)n_sel * kNumClasses * (b.nT + 3))) || (r = al(&b.med, n_sel)) ||
        (r = al(&b.ghist, (size_t)n_sel * kMedBins)) || (r = al(&b.po.surv, SL)) || (r = al(&b.po.nsurv, n_sel)))
        return r;
    b.po.blkcnt = b.blkcnt;
    b.po.wpart = b.wpart;
    return MPSA_OK;
}

int ranges_launch(const PrepBufs& b, int tile, int* cum, cudaStream_t st);

// Line preparation of the rows d_sel of `pop` on the grid (lam0, R, N): placement, line terms,
// median continuum and cut threshold, cut windows, width-class buckets and tile ranges.
int prep_launch(const PrepBufs& b, const mpsa_ctx* ctx, const double* pop, const int* d_sel, double lam0_nm,
                float* kc_out, int64_t* evals, const mpsa_synth_opts* opts, cudaStream_t st) {
    const double cut = (opts && opts->cut > 0) ? opts->cut : 1e-3;
    const double kcf = (opts && opts->kc_factor > 0) ? opts->kc_factor : 1e-2;
    const int64_t L = b.L;
    const int n_sel = b.n_sel, n_sp = ctx->n_sp;
    const int lb = (int)((L + 255) / 256);
    k_place<<<lb, 256, 0, st>>>(L, ctx->d_lam, lam0_nm, b.lnq, b.c, b.f, b.lamcm);
    const int pop32 = (opts && opts->precision == MPSA_PREC_FP32_POP32) ? 1 : 0;
    k_consts<<<(n_sel * n_sp + 127) / 128, 128, 0, st>>>(n_sel, d_sel, n_sp, ctx->d_sp_el, ctx->d_sp_stage, ctx->n_el,
                                                           ctx->d_el, pop, ctx->vturb, pop32, b.rc, b.spc);
    k_kappa0<<<dim3(lb, (n_sel + kKappa0Rows - 1) / kKappa0Rows), 256, 0, st>>>(
        L, n_sel, ctx->d_species, ctx->d_loggf, ctx->d_E, ctx->d_lgR, ctx->d_lgS, ctx->d_lgW, b.lamcm, n_sp, b.rc,
        b.spc, b.lnS, b.av, b.lnk0);
    {
        // median of ln kappa0 per row: three radix levels, each a multi-CTA histogram and a pick
        const int per_row = (int)std::max<int64_t>(1, std::min<int64_t>(128, (L + 8191) / 8192));
        k_med_init<<<(n_sel * kMedBins + 255) / 256, 256, 0, st>>>(n_sel, L, b.med, b.ghist);
        for (int level = 0; level < 3; ++level) {
            k_med_hist<<<dim3(per_row, n_sel), 1024, 0, st>>>(L, b.lnk0, level, b.med, b.ghist);
            k_med_pick<<<n_sel, 1024, 0, st>>>(level, b.med, b.ghist, (float)log(kcf), (float)log(cut), b.ln_tp,
                                               kc_out);
        }
    }
    MPSA_CUDA_TRY(cudaMemsetAsync(b.po.nsurv, 0, (size_t)n_sel * sizeof(int), st));
    k_prep<<<dim3(b.nb, n_sel), kPrepThreads, 0, st>>>(L, b.N, (float)b.lnq, ctx->d_species, b.c, b.f, n_sp, b.spc,
                                                       b.lnS, b.av, b.lnk0, b.ln_tp, b.nb, b.po);
    {
        // the listed lines' count is known on the device only: about eight CTAs per SM in all,
        // each running over its row's list
        int dev = 0, sms = 0;
        MPSA_CUDA_TRY(cudaGetDevice(&dev));
        MPSA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int gx = std::max(1, std::min(b.nb, (8 * sms + n_sel - 1) / n_sel));
        k_windows<<<dim3(gx, n_sel), kPrepThreads, 0, st>>>(L, b.N, (float)b.lnq, ctx->d_species, b.c, b.f, n_sp, b.spc,
                                                            b.lnS, b.av, b.ln_tp, b.nb, b.po);
    }
    k_scan_class<<<dim3(kNumClasses, n_sel), 1024, 0, st>>>(b.nb, b.blkcnt, b.classcnt);
    k_scan_fin<<<n_sel, 1024, 0, st>>>(b.nb, b.classcnt, b.classbase, b.wpart, (long long*)evals);
    k_scatter<<<dim3(b.nb, n_sel), kPrepThreads, 0, st>>>(L, b.N, b.po.cls, b.c, b.blkcnt, b.classbase, b.nb, b.bidx,
                                                          b.bkey, b.po, b.rec);
    return ranges_launch(b, b.tile, b.cum, st);
}

int ranges_launch(const PrepBufs& b, int tile, int* cum, cudaStream_t st) {
    const int nT = (b.N + tile - 1) / tile;
    const int64_t nr = (int64_t)b.n_sel * kNumClasses * (nT + 3);
    k_ranges<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(b.n_sel, b.L, nT, tile, b.bkey, b.classbase, b.classcnt,
                                                          cum);
    MPSA_CUDA_TRY(cudaGetLastError());
    return MPSA_OK;
}

TileArgs tile_args(const PrepBufs& b, float* kappa) {
    TileArgs ta;
    ta.N = b.N;
    ta.nT = b.nT;
    ta.L = b.L;
    ta.lnq = (float)b.lnq;
    ta.q1 = (float)(-b.lnq / 2.0);
    ta.q2 = (float)(b.lnq * b.lnq / 6.0);
    ta.q3 = (float)(-b.lnq * b.lnq * b.lnq / 24.0);
    ta.cum = b.cum;
    ta.bidx = b.bidx;
    ta.rec = b.rec;
    ta.c = b.po.c;
    ta.f = b.po.f;
    ta.srel = b.po.srel;
    ta.a = b.po.a;
    ta.kv = b.po.kv;
    ta.jlo = b.po.jlo;
    ta.jhi = b.po.jhi;
    ta.ilo = b.po.ilo;
    ta.ihi = b.po.ihi;
    ta.ln_tp = b.ln_tp;
    ta.out = kappa;
    ta.split = 1;
    ta.part = nullptr;
    return ta;
}

int synth_rows(mpsa_ctx* ctx, const double* pop, int n_sel, const int* d_sel, double lam0_nm, double R, int N,
               float* kappa, float* kc_out, int64_t* evals, const mpsa_synth_opts* opts, cudaStream_t st) {
    const int prec = opts ? opts->precision : 0;
    if (prec != MPSA_PREC_FP32_COMPENSATED && prec != MPSA_PREC_FP32_NAIVE && prec != MPSA_PREC_FP64 &&
        prec != MPSA_PREC_FP32_POP32)
        return fail(MPSA_EINVAL, "synth: precision %d", prec);
    Scratch sc(st, ctx->pool);
    PrepBufs b;
    int r;
    const int tile = prec == MPSA_PREC_FP64 ? kTile64 : kTile;
    if ((r = prep_alloc(b, ctx, n_sel, N, R, tile, [&](auto** p, size_t n) { return sc.alloc(p, n); }))) return r;
    if ((r = prep_launch(b, ctx, pop, d_sel, lam0_nm, kc_out, evals, opts, st))) return r;
    const TileArgs ta = tile_args(b, kappa);
    prof_mark(ctx, MPSA_KERNEL_PROFILE, st);
    if (prec == MPSA_PREC_FP64) {
        Tile64Args g;
        g.t = ta;
        g.sel = d_sel;
        g.pop = pop;
        g.pop_stride_ = pop_stride(ctx->n_el);
        g.n_sp = ctx->n_sp;
        g.sp_el = ctx->d_sp_el;
        g.sp_stage = ctx->d_sp_stage;
        g.el = ctx->d_el;
        g.n_el = ctx->n_el;
        g.vturb = ctx->vturb;
        g.lam_nm = ctx->d_lam;
        g.loggf = ctx->d_loggf;
        g.E = ctx->d_E;
        g.lgR = ctx->d_lgR;
        g.lgS = ctx->d_lgS;
        g.lgW = ctx->d_lgW;
        g.species = ctx->d_species;
        g.lam0_nm = lam0_nm;
        g.lnq64 = b.lnq;
        k_tiles64<<<dim3(b.nT, n_sel), 256, 0, st>>>(g);
    } else {
        // a call with fewer tiles than two waves of the GPU (narrow windows) splits each tile's
        // candidate lines over several CTAs, up to 64, and adds their partial sums afterwards
        int dev = 0, sms = 0;
        MPSA_CUDA_TRY(cudaGetDevice(&dev));
        MPSA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int64_t ctas = (int64_t)b.nT * n_sel, want = 2ll * sms * MPSA_TILES_MINB;
        TileArgs tb = ta;
        tb.split = ctas >= want ? 1 : (int)std::min<int64_t>(64, (want + ctas - 1) / ctas);
        tb.part = nullptr;
        if (tb.split > 1 && (r = sc.alloc(&tb.part, (size_t)n_sel * tb.split * N))) return r;
        const dim3 grid((unsigned)(b.nT * tb.split), n_sel);
        const bool naive = prec == MPSA_PREC_FP32_NAIVE;
        if (tb.split > 1) {
            if (naive) k_tiles<MPSA_PREC_FP32_NAIVE, true><<<grid, kTileThreads, 0, st>>>(tb);
            else k_tiles<MPSA_PREC_FP32_COMPENSATED, true><<<grid, kTileThreads, 0, st>>>(tb);
        } else {
            if (naive) k_tiles<MPSA_PREC_FP32_NAIVE, false><<<grid, kTileThreads, 0, st>>>(tb);
            else k_tiles<MPSA_PREC_FP32_COMPENSATED, false><<<grid, kTileThreads, 0, st>>>(tb);
        }
        if (tb.split > 1) {
            const int64_t tot = (int64_t)n_sel * N;
            k_split_sum<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n_sel, N, tb.split, tb.part, kappa);
        }
    }
    prof_mark(ctx, MPSA_KERNEL_PROFILE, st);
    MPSA_CUDA_TRY(cudaGetLastError());
    return MPSA_OK;
}

int check_species(const mpsa_ctx* ctx, const char* who) {
    for (int i = 0; i < ctx->n_sp; ++i) {
        const int e = ctx->h_sp_el[i], st = ctx->h_sp_stage[i];
        if (e >= ctx->n_el) return fail(MPSA_EINVAL, "%s: species %d refers to element %d of %d", who, i, e, ctx->n_el);
        if (st >= (int)ctx->h_el[(size_t)e * kElStride + kElStages])
            return fail(MPSA_EINVAL, "%s: species %d is stage %d of element %d, which has %d stages", who, i, st, e,
                        (int)ctx->h_el[(size_t)e * kElStride + kElStages]);
    }
    return MPSA_OK;
}

int check_grid(const mpsa_lgrid* g, int* N) {
    const int64_t n = mpsa_grid_size(g);
    if (n < 1) return fail(MPSA_EINVAL, "invalid grid");
    if (n >= kMaxGrid - kTile) return fail(MPSA_EINVAL, "grid of %lld points exceeds %d", (long long)n, kMaxGrid - kTile);
    *N = (int)n;
    return MPSA_OK;
}

}  // namespace mpsa

using namespace mpsa;

extern "C" int synth_opacity(mpsa_ctx* ctx, const mpsa_lgrid* grid, int32_t n_sel, const int32_t* sel,
                             float* kappa_out, float* kappa_c_out, int64_t* evals_out, const mpsa_synth_opts* opts,
                             void* stream) {
    if (!ctx || !grid || !sel || !kappa_out) return fail(MPSA_EINVAL, "synth_opacity: NULL argument");
    if (ctx->L < 1 || ctx->n_sp < 1) return fail(MPSA_ESTATE, "synth_opacity: no line list loaded");
    if (!ctx->d_pop) return fail(MPSA_ESTATE, "synth_opacity: no atmosphere grid set");
    if (n_sel < 1) return fail(MPSA_EINVAL, "synth_opacity: n_sel = %d", n_sel);
    int N, r;
    if ((r = check_species(ctx, "synth_opacity"))) return r;
    const int rows = ctx->n_comp * ctx->n_points;
    for (int i = 0; i < n_sel; ++i)
        if (sel[i] < 0 || sel[i] >= rows) return fail(MPSA_EINVAL, "synth_opacity: sel[%d] = %d of %d rows", i, sel[i], rows);
    if ((r = check_grid(grid, &N))) return r;
    if ((size_t)n_sel * ctx->L >= (size_t)1 << 31)
        return fail(MPSA_EINVAL, "synth_opacity: n_sel * n_lines must stay below 2^31 (split the rows)");
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    int* d_sel;
    {
        Scratch s2(st, ctx->pool);
        if ((r = s2.alloc(&d_sel, n_sel))) return r;
        MPSA_CUDA_TRY(cudaMemcpyAsync(d_sel, sel, n_sel * sizeof(int), cudaMemcpyHostToDevice, st));
        r = synth_rows(ctx, ctx->d_pop, n_sel, d_sel, grid->lambda0_nm, grid->R, N, kappa_out, kappa_c_out, evals_out,
                       opts, st);
    }
    return r;
}

// ===========================================================================
// Batched form: many rows on several grids in one persistent, graph-captured launch.
//
// At creation every group's line preparation runs once; an autotuner times the
// persistent profile kernel for each candidate (points per thread, threads per CTA,
// CTAs per SM) on a sample of tiles and keeps the fastest per grid point; the
// (row, tile) work units are ordered by decreasing estimated cost (candidate lines
// per tile, largest first); then the whole pipeline (preparation of every group,
// one persistent profile launch over all units, the ODFs) is captured into a CUDA
// graph that mpsa_batch_run replays.
namespace mpsa {
namespace {

struct TuneCfg {
    int pts, threads, minb;
};
constexpr TuneCfg kCfgs[] = {{8, 256, 4}, {4, 256, 4}, {8, 128, 8}, {16, 128, 3}};
constexpr int kNumCfgs = sizeof(kCfgs) / sizeof(kCfgs[0]);

template <int PREC, int PTS, int THREADS, int MINB>
int persistent_launch_t(const RowDesc* rows, const int2* units, int n_units, int* counter, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    MPSA_CUDA_TRY(cudaGetDevice(&dev));
    MPSA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MPSA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tiles_persistent<PREC, PTS, THREADS, MINB>,
                                                                THREADS, 0));
    const int grid = std::max(1, std::min(n_units, sms * std::max(per_sm, 1)));
    k_tiles_persistent<PREC, PTS, THREADS, MINB><<<grid, THREADS, 0, st>>>(rows, units, n_units, counter);
    MPSA_CUDA_TRY(cudaGetLastError());
    return MPSA_OK;
}

int persistent_launch(int cfg, int prec, const RowDesc* rows, const int2* units, int n_units, int* counter,
                      cudaStream_t st) {
    MPSA_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), st));
    if (prec == MPSA_PREC_FP32_NAIVE) {
        switch (cfg) {
            case 0: return persistent_launch_t<1, 8, 256, 4>(rows, units, n_units, counter, st);
            case 1: return persistent_launch_t<1, 4, 256, 4>(rows, units, n_units, counter, st);
            case 2: return persistent_launch_t<1, 8, 128, 8>(rows, units, n_units, counter, st);
            default: return persistent_launch_t<1, 16, 128, 3>(rows, units, n_units, counter, st);
        }
    }
    switch (cfg) {
        case 0: return persistent_launch_t<0, 8, 256, 4>(rows, units, n_units, counter, st);
        case 1: return persistent_launch_t<0, 4, 256, 4>(rows, units, n_units, counter, st);
        case 2: return persistent_launch_t<0, 8, 128, 8>(rows, units, n_units, counter, st);
        default: return persistent_launch_t<0, 16, 128, 3>(rows, units, n_units, counter, st);
    }
}

// Estimated cost of a (row, tile) unit: the number of candidate lines of the tile.
__global__ void k_unit_cost(const RowDesc* __restrict__ rows, const int2* __restrict__ units, int n_units,
                            long long* __restrict__ cost) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_units) return;
    const int2 rt = units[u];
    const RowDesc r = rows[rt.x];
    const int TILE = r.tile, J0 = rt.y * TILE;
    long long n = 0;
    for (int b = 0; b < kNumClasses; ++b) {
        const int reach = 1 << b;
        int tlo = max(floordiv(J0 - reach + 1, TILE), -1), thi = min(floordiv(J0 + TILE - 1 + reach - 1, TILE), r.nT);
        if (tlo > thi) continue;
        const int* cum = r.cum + (size_t)b * (r.nT + 3);
        n += cum[thi + 2] - cum[tlo + 1];
    }
    cost[u] = n;
}

}  // namespace
}  // namespace mpsa

struct mpsa_batch {
    mpsa_ctx* ctx = nullptr;
    mpsa_synth_opts opts{};
    int prec = 0, cfg = 0;
    struct Group {
        mpsa_lgrid grid{};
        int N = 0, n_sel = 0;
        int* d_sel = nullptr;
        float *kappa = nullptr, *kc = nullptr;
        int64_t* evals = nullptr;
        mpsa::PrepBufs pb;
        int* cum = nullptr;   // tile ranges for the chosen tile size
        int K = 0, n_steps = 0, mean_kind = MPSA_MEAN_ARITH;
        int64_t* d_bounds = nullptr;
        double *d_cw = nullptr, *d_w = nullptr, *odf = nullptr;
    };
    std::vector<Group> groups;
    mpsa::RowDesc* d_rows = nullptr;
    int n_rows = 0;
    int2* d_units = nullptr;
    int n_units = 0;
    int* d_counter = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void*> allocs;
    double tune_ms_per_mpt[mpsa::kNumCfgs] = {0};
    int n_tuned = 0;
};

namespace mpsa {
namespace {

template <class T>
int balloc(mpsa_batch* b, T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T) + 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MPSA_ENOMEM, "mpsa_batch_create: cudaMalloc(%zu): %s", n * sizeof(T), cudaGetErrorString(e));
    }
    b->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return MPSA_OK;
}

// Row descriptors for every row of every group with the tile ranges `cums[g]` of tile size `tile`.
std::vector<RowDesc> row_descs(mpsa_batch* b, int tile, const std::vector<int*>& cums) {
    std::vector<RowDesc> rows;
    for (size_t g = 0; g < b->groups.size(); ++g) {
        auto& G = b->groups[g];
        const int nT = (G.N + tile - 1) / tile;
        for (int s = 0; s < G.n_sel; ++s) {
            TileArgs ta = tile_args(G.pb, G.kappa);
            ta.nT = nT;
            ta.cum = cums[g];
            RowDesc r;
            const size_t sL = (size_t)s * G.pb.L;
            r.N = G.N;
            r.nT = nT;
            r.tile = tile;
            r.lnq = ta.lnq;
            r.q1 = ta.q1;
            r.q2 = ta.q2;
            r.q3 = ta.q3;
            r.ln_tp = G.pb.ln_tp + s;
            r.cum = cums[g] + (size_t)s * kNumClasses * (nT + 3);
            r.bidx = G.pb.bidx + sL;
            r.rec = G.pb.rec + sL;
            r.c = G.pb.po.c + sL;
            r.f = G.pb.po.f + sL;
            r.srel = G.pb.po.srel + sL;
            r.a = G.pb.po.a + sL;
            r.kv = G.pb.po.kv + sL;
            r.jlo = G.pb.po.jlo + sL;
            r.jhi = G.pb.po.jhi + sL;
            r.ilo = G.pb.po.ilo + sL;
            r.ihi = G.pb.po.ihi + sL;
            r.out = G.kappa + (size_t)s * G.N;
            rows.push_back(r);
        }
    }
    return rows;
}

int batch_build(mpsa_batch* b, const mpsa_batch_group* gin, int n_groups, int autotune, cudaStream_t st) {
    mpsa_ctx* c = b->ctx;
    int r;
    // ---- groups: grids, rows, persistent prep buffers, ODF parameters
    for (int g = 0; g < n_groups; ++g) {
        const mpsa_batch_group& q = gin[g];
        mpsa_batch::Group G;
        G.grid = q.grid;
        if ((r = check_grid(&q.grid, &G.N))) return r;
        if (q.n_sel < 1 || !q.sel || !q.kappa_out) return fail(MPSA_EINVAL, "mpsa_batch_create: group %d rows/outputs", g);
        const int rows = c->n_comp * c->n_points;
        for (int i = 0; i < q.n_sel; ++i)
            if (q.sel[i] < 0 || q.sel[i] >= rows) return fail(MPSA_EINVAL, "mpsa_batch_create: group %d sel[%d]", g, i);
        if ((size_t)q.n_sel * c->L >= (size_t)1 << 31) return fail(MPSA_EINVAL, "mpsa_batch_create: group %d too large", g);
        G.n_sel = q.n_sel;
        G.kappa = q.kappa_out;
        G.kc = q.kappa_c_out;
        G.evals = q.evals_out;
        if ((r = balloc(b, &G.d_sel, q.n_sel))) return r;
        MPSA_CUDA_TRY(cudaMemcpy(G.d_sel, q.sel, q.n_sel * sizeof(int), cudaMemcpyHostToDevice));
        if ((r = prep_alloc(G.pb, c, q.n_sel, G.N, q.grid.R, kTile, [&](auto** p, size_t n) { return balloc(b, p, n); })))
            return r;
        if (q.K > 0) {
            if (!q.bounds || !q.widths || !q.odf_out) return fail(MPSA_EINVAL, "mpsa_batch_create: group %d ODF args", g);
            std::vector<double> cw(q.n_steps >= 1 && q.n_steps <= 32 ? q.n_steps + 1 : 1);
            if ((r = odf_check("mpsa_batch_create", q.n_sel, G.N, q.K, q.bounds, q.n_steps, q.widths, q.mean_kind,
                               cw.data())))
                return r;
            G.K = q.K;
            G.n_steps = q.n_steps;
            G.mean_kind = q.mean_kind;
            G.odf = q.odf_out;
            if ((r = balloc(b, &G.d_bounds, q.K + 1)) || (r = balloc(b, &G.d_cw, q.n_steps + 1)) ||
                (r = balloc(b, &G.d_w, q.n_steps)))
                return r;
            MPSA_CUDA_TRY(cudaMemcpy(G.d_bounds, q.bounds, (q.K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
            MPSA_CUDA_TRY(cudaMemcpy(G.d_cw, cw.data(), (q.n_steps + 1) * sizeof(double), cudaMemcpyHostToDevice));
            MPSA_CUDA_TRY(cudaMemcpy(G.d_w, q.widths, q.n_steps * sizeof(double), cudaMemcpyHostToDevice));
        }
        b->groups.push_back(G);
        b->n_rows += q.n_sel;
    }
    for (auto& G : b->groups)
        if ((r = prep_launch(G.pb, c, c->d_pop, G.d_sel, G.grid.lambda0_nm, G.kc, G.evals, &b->opts, st))) return r;
    MPSA_CUDA_TRY(cudaStreamSynchronize(st));
    if ((r = balloc(b, &b->d_rows, b->n_rows)) || (r = balloc(b, &b->d_counter, 1))) return r;

    // ---- autotune: time per grid point of each configuration on a sample of tiles
    b->cfg = 0;
    if (autotune) {
        cudaEvent_t e0, e1;
        MPSA_CUDA_TRY(cudaEventCreate(&e0));
        MPSA_CUDA_TRY(cudaEventCreate(&e1));
        double best = 1e300;
        for (int k = 0; k < kNumCfgs; ++k) {
            const int tile = kCfgs[k].pts * kCfgs[k].threads;
            std::vector<int*> cums;
            for (auto& G : b->groups) {
                const int nT = (G.N + tile - 1) / tile;
                int* cum;
                if ((r = balloc(b, &cum, (size_t)G.n_sel * kNumClasses * (nT + 3)))) return r;
                if ((r = ranges_launch(G.pb, tile, cum, st))) return r;
                cums.push_back(cum);
            }
            std::vector<RowDesc> rows = row_descs(b, tile, cums);
            // sample: at least 2048 (row, tile) units (all of them if there are fewer) spread
            // evenly over all units of the batch, so that rows weigh by their tile counts as in
            // the real launch and every CTA of the persistent launch runs several units (the
            // time then measures throughput, not the slowest unit)
            std::vector<int2> all;
            for (int i = 0; i < (int)rows.size(); ++i)
                for (int t = 0; t < rows[i].nT; ++t) all.push_back(make_int2(i, t));
            std::vector<int2> units;
            const size_t step = std::max<size_t>(1, all.size() / 2048);
            for (size_t u = step / 2; u < all.size(); u += step) units.push_back(all[u]);
            int2* du;
            if ((r = balloc(b, &du, units.size()))) return r;
            MPSA_CUDA_TRY(cudaMemcpy(b->d_rows, rows.data(), rows.size() * sizeof(RowDesc), cudaMemcpyHostToDevice));
            MPSA_CUDA_TRY(cudaMemcpy(du, units.data(), units.size() * sizeof(int2), cudaMemcpyHostToDevice));
            float ms_best = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                MPSA_CUDA_TRY(cudaEventRecord(e0, st));
                if ((r = persistent_launch(k, b->prec, b->d_rows, du, (int)units.size(), b->d_counter, st))) return r;
                MPSA_CUDA_TRY(cudaEventRecord(e1, st));
                MPSA_CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                MPSA_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                ms_best = std::min(ms_best, ms);
            }
            const double per_mpt = ms_best / ((double)units.size() * tile / 1e6);
            b->tune_ms_per_mpt[k] = per_mpt;
            if (per_mpt < best) {
                best = per_mpt;
                b->cfg = k;
            }
        }
        b->n_tuned = kNumCfgs;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }

    // ---- final tile ranges, row descriptors and the cost-ordered work list
    const int tile = kCfgs[b->cfg].pts * kCfgs[b->cfg].threads;
    std::vector<int*> cums;
    for (auto& G : b->groups) {
        const int nT = (G.N + tile - 1) / tile;
        if ((r = balloc(b, &G.cum, (size_t)G.n_sel * kNumClasses * (nT + 3)))) return r;
        if ((r = ranges_launch(G.pb, tile, G.cum, st))) return r;
        cums.push_back(G.cum);
    }
    std::vector<RowDesc> rows = row_descs(b, tile, cums);
    MPSA_CUDA_TRY(cudaMemcpy(b->d_rows, rows.data(), rows.size() * sizeof(RowDesc), cudaMemcpyHostToDevice));
    std::vector<int2> units;
    for (int i = 0; i < (int)rows.size(); ++i)
        for (int t = 0; t < rows[i].nT; ++t) units.push_back(make_int2(i, t));
    b->n_units = (int)units.size();
    if ((r = balloc(b, &b->d_units, units.size()))) return r;
    long long* dcost;
    if ((r = balloc(b, &dcost, units.size()))) return r;
    MPSA_CUDA_TRY(cudaMemcpy(b->d_units, units.data(), units.size() * sizeof(int2), cudaMemcpyHostToDevice));
    MPSA_CUDA_TRY(cudaStreamSynchronize(st));
    k_unit_cost<<<(b->n_units + 255) / 256, 256, 0, st>>>(b->d_rows, b->d_units, b->n_units, dcost);
    MPSA_CUDA_TRY(cudaGetLastError());
    std::vector<long long> cost(units.size());
    MPSA_CUDA_TRY(cudaMemcpyAsync(cost.data(), dcost, cost.size() * sizeof(long long), cudaMemcpyDeviceToHost, st));
    MPSA_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int> order(units.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<int2> sorted(units.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = units[order[i]];
    MPSA_CUDA_TRY(cudaMemcpy(b->d_units, sorted.data(), sorted.size() * sizeof(int2), cudaMemcpyHostToDevice));

    // ---- capture the pipeline into a CUDA graph
    if ((r = odf_setup())) return r;
    cudaStream_t cap;
    MPSA_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        return fail(MPSA_ECUDA, "mpsa_batch_create: begin capture: %s", cudaGetErrorString(e));
    }
    int rc = MPSA_OK;
    for (auto& G : b->groups) {
        if ((rc = prep_launch(G.pb, c, c->d_pop, G.d_sel, G.grid.lambda0_nm, G.kc, G.evals, &b->opts, cap))) break;
        if ((rc = ranges_launch(G.pb, tile, G.cum, cap))) break;
    }
    if (rc == MPSA_OK) rc = persistent_launch(b->cfg, b->prec, b->d_rows, b->d_units, b->n_units, b->d_counter, cap);
    if (rc == MPSA_OK)
        for (auto& G : b->groups)
            if (G.K > 0 && (rc = odf_launch(G.kappa, G.n_sel, G.N, G.K, G.d_bounds, G.n_steps, G.d_cw, G.d_w, G.odf, G.mean_kind, cap)))
                break;
    e = cudaStreamEndCapture(cap, &b->graph);
    cudaStreamDestroy(cap);
    if (rc != MPSA_OK) return rc;
    if (e != cudaSuccess) return fail(MPSA_ECUDA, "mpsa_batch_create: end capture: %s", cudaGetErrorString(e));
    MPSA_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return MPSA_OK;
}

}  // namespace
}  // namespace mpsa

extern "C" {

int mpsa_batch_create(mpsa_ctx* ctx, int32_t n_groups, const mpsa_batch_group* groups, const mpsa_synth_opts* opts,
                      int32_t autotune, void* stream, mpsa_batch** out) {
    if (!ctx || !groups || !out || n_groups < 1) return fail(MPSA_EINVAL, "mpsa_batch_create: bad argument");
    if (ctx->L < 1 || !ctx->d_pop) return fail(MPSA_ESTATE, "mpsa_batch_create: load a line list and a grid first");
    int rs;
    if ((rs = check_species(ctx, "mpsa_batch_create"))) return rs;
    const int prec = opts ? opts->precision : 0;
    if (prec != MPSA_PREC_FP32_COMPENSATED && prec != MPSA_PREC_FP32_NAIVE)
        return fail(MPSA_EINVAL, "mpsa_batch_create: precision %d", prec);
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    *out = nullptr;
    mpsa_batch* b = new mpsa_batch();
    b->ctx = ctx;
    if (opts) b->opts = *opts;
    b->prec = prec;
    const int r = batch_build(b, groups, n_groups, autotune, (cudaStream_t)stream);
    if (r != MPSA_OK) {
        mpsa_batch_destroy(b);
        return r;
    }
    *out = b;
    return MPSA_OK;
}

int mpsa_batch_run(mpsa_batch* b, void* stream) {
    if (!b || !b->exec) return fail(MPSA_EINVAL, "mpsa_batch_run: bad batch");
    MPSA_CUDA_TRY(cudaSetDevice(b->ctx->device));
    prof_mark(b->ctx, MPSA_KERNEL_PROFILE, (cudaStream_t)stream);
    MPSA_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    prof_mark(b->ctx, MPSA_KERNEL_PROFILE, (cudaStream_t)stream);
    return MPSA_OK;
}

int mpsa_batch_get_info(const mpsa_batch* b, mpsa_batch_info* out) {
    if (!b || !out) return fail(MPSA_EINVAL, "mpsa_batch_get_info: bad argument");
    out->pts_per_thread = kCfgs[b->cfg].pts;
    out->threads = kCfgs[b->cfg].threads;
    out->min_blocks = kCfgs[b->cfg].minb;
    out->n_rows = b->n_rows;
    out->n_units = b->n_units;
    out->n_tuned = b->n_tuned;
    for (int k = 0; k < 8; ++k) out->tune_ms_per_mpoint[k] = k < kNumCfgs ? b->tune_ms_per_mpt[k] : 0.0;
    return MPSA_OK;
}

int mpsa_voigt(mpsa_ctx* ctx, const double* v, const double* a, int64_t n, int32_t precision, double* out,
               void* stream) {
    if (!ctx || n < 0 || (n > 0 && (!v || !a || !out))) return fail(MPSA_EINVAL, "mpsa_voigt: bad argument");
    if (n == 0) return MPSA_OK;
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    const int threads = 256;
    const int64_t blocks = (n + threads - 1) / threads;
    if (blocks > 0x7fffffff) return fail(MPSA_EINVAL, "mpsa_voigt: n = %lld too large", (long long)n);
    k_voigt_eval<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(n, v, a, precision == MPSA_PREC_FP64, out);
    MPSA_CUDA_TRY(cudaGetLastError());
    return MPSA_OK;
}

void mpsa_batch_destroy(mpsa_batch* b) {
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void* p : b->allocs) cudaFree(p);
    delete b;
}

}  // extern "C"

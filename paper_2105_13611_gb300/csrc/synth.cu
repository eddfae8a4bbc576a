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
//   k_median       per row: lower median of ln kappa0 by radix selection -> ln t_p, kappa_c
//   k_prep         per (row, line): strength relative to t_p, cut windows (outer: no point
//                  beyond can pass the cut; inner: every point inside passes), width class
//   k_scan, k_scatter   stable counting sort of the kept lines by width class
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

namespace mpsa {

namespace {

constexpr float kLn10 = 2.302585092994046f;
constexpr float kFourPi = 12.566370614359172f;
constexpr float kFarV = 41.f;            // far formula valid for |v| >= 40
constexpr int kFarDist = 8 * kTile;      // far formula precise when the centre is this far away

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
                         const double* __restrict__ pop, double vturb, RowConst* __restrict__ rc,
                         SpConst* __restrict__ sc) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_sel * n_sp) return;
    const int s = t / n_sp, sp = t % n_sp;
    const double* row = pop + (size_t)sel[s] * pop_stride(n_el);
    const double T = row[kPopT];
    const int e = sp_el[sp], st = sp_stage[sp];
    const double m = el[e] * kAMU;
    const double u = sqrt(2.0 * kKB * T / m + vturb * vturb);
    const double NU = row[kPopHdr + 2 * e + st];
    const double pre = sqrt(kPI) * kE * kE / (kME * kC);
    SpConst o;
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
__global__ void k_kappa0(int64_t L, const int* __restrict__ species, const float* __restrict__ loggf,
                         const float* __restrict__ E, const float* __restrict__ lgR, const float* __restrict__ lgS,
                         const float* __restrict__ lgW, const float* __restrict__ lamcm, int n_sp,
                         const RowConst* __restrict__ rc, const SpConst* __restrict__ sc,
                         float* __restrict__ lnS_out, float* __restrict__ a_out, float* __restrict__ lnk0_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= L) return;
    const RowConst r = rc[s];
    const SpConst q = sc[(size_t)s * n_sp + species[i]];
    const float lam = lamcm[i];
    const float gamma = exp10f(lgR[i]) + exp10f(lgS[i]) * r.ne + exp10f(lgW[i]) * r.nHI;
    const float a = gamma * lam / (kFourPi * q.u);
    const float lnDnu = logf(q.u) - logf(lam);
    const float stim = -expm1f(-r.hc_kT_cm / lam);
    const float lnS = q.lnC + loggf[i] * kLn10 - E[i] * r.inv_kT_eV + logf(stim) - lnDnu;
    const size_t o = (size_t)s * L + i;
    lnS_out[o] = lnS;
    a_out[o] = a;
    lnk0_out[o] = lnS + logf(voigt_H(0.f, a));
}

// ---------------------------------------------------------------------------
// k_median: lower median (rank (L-1)/2) of ln kappa0 per row by 4-pass MSB radix
// selection on order-preserving keys of the FP32 bit patterns.
__device__ __forceinline__ unsigned fkey(float x) {
    unsigned b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unkey(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void __launch_bounds__(1024) k_median(int64_t L, const float* __restrict__ lnk0, float ln_kc_factor,
                                                 float ln_cut, float* __restrict__ ln_tp, float* __restrict__ kc_out) {
    __shared__ unsigned hist[256];
    __shared__ unsigned s_prefix, s_rank;
    const int s = blockIdx.x;
    const float* x = lnk0 + (size_t)s * L;
    if (threadIdx.x == 0) {
        s_prefix = 0;
        s_rank = (unsigned)((L - 1) / 2);
    }
    for (int level = 0; level < 4; ++level) {
        const int shift = 24 - 8 * level;
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const unsigned prefix = s_prefix;
        const unsigned pmask = level == 0 ? 0u : (0xffffffffu << (32 - 8 * level));
        for (int64_t i = threadIdx.x; i < L; i += blockDim.x) {
            unsigned k = fkey(x[i]);
            if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned rank = s_rank, acc = 0;
            int b = 0;
            for (; b < 255; ++b) {
                if (acc + hist[b] > rank) break;
                acc += hist[b];
            }
            s_rank = rank - acc;
            s_prefix = prefix | ((unsigned)b << shift);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float med = unkey(s_prefix);
        ln_tp[s] = med + ln_kc_factor + ln_cut;
        if (kc_out) kc_out[s] = expf(med + ln_kc_factor);
    }
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

__device__ void cut_speeds(float a, float r, float* v_out, float* v_in) {
    const float t_out = r * (1.f - 1e-4f), t_in = r * (1.f + 1e-4f);
    const float vmin = 1e-4f;
    {
        float lo = vmin, hi = v_bound(a, t_out);
        if (voigt_H(lo, a) < t_out) {
            hi = lo;
        } else {
            for (int it = 0; it < 40; ++it) {
                const float mid = sqrtf(lo * hi);
                if (voigt_H(mid, a) < t_out) hi = mid; else lo = mid;
            }
        }
        *v_out = hi;
    }
    if (voigt_H(0.f, a) < t_in) {
        *v_in = -1.f;
    } else {
        float lo = vmin, hi = v_bound(a, t_in);
        if (voigt_H(lo, a) < t_in) {
            *v_in = 0.f;
            return;
        }
        for (int it = 0; it < 40; ++it) {
            const float mid = sqrtf(lo * hi);
            if (voigt_H(mid, a) < t_in) hi = mid; else lo = mid;
        }
        *v_in = lo;
    }
}

// grid offsets d >= 0 at which |v| reaches vv, red side (d > 0: |v| = kv (1 - e^{-d lnq}))
// and blue side (|v| = kv (e^{d lnq} - 1)).
__device__ __forceinline__ float d_red(float vv, float kv, float lnq) {
    const float t = vv / kv;
    return t >= 1.f ? 1.0e9f : fminf(-log1pf(-t) / lnq, 1.0e9f);
}
__device__ __forceinline__ float d_blue(float vv, float kv, float lnq) { return fminf(log1pf(vv / kv) / lnq, 1.0e9f); }

constexpr unsigned char kDropped = 255;

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
};

__global__ void __launch_bounds__(256) k_prep(int64_t L, int N, float lnq, const int* __restrict__ species,
                                              const int* __restrict__ cpos, const float* __restrict__ fpos,
                                              int n_sp, const SpConst* __restrict__ sc,
                                              const float* __restrict__ lnS, const float* __restrict__ av,
                                              const float* __restrict__ lnk0, const float* __restrict__ ln_tp,
                                              int nb, PrepOut o) {
    __shared__ int cnt[kNumClasses];
    __shared__ long long wsum[8];
    const int s = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (threadIdx.x < kNumClasses) cnt[threadIdx.x] = 0;
    __syncthreads();
    long long w = 0;
    if (i < L) {
        const size_t q = (size_t)s * L + i;
        const float ltp = ln_tp[s];
        unsigned char cls = kDropped;
        int c = cpos[i];
        float f = fpos[i];
        float kv = sc[(size_t)s * n_sp + species[i]].kv;
        float a = av[q];
        float srel = 0.f;
        int jlo = 1, jhi = 0, ilo = 1, ihi = 0;
        if (lnk0[q] >= ltp) {
            const float rel = fminf(lnS[q] - ltp, 88.f);
            srel = expf(rel);
            const float r = expf(-rel);
            float vo, vi;
            cut_speeds(a, r, &vo, &vi);
            const float vo2 = vo * (1.f + 1e-5f);
            long long hi = (long long)c + (long long)floorf(fminf(f + d_red(vo2, kv, lnq), 1.0e9f)) + 2;
            long long lo = (long long)c + (long long)ceilf(fmaxf(f - d_blue(vo2, kv, lnq), -1.0e9f)) - 2;
            hi = hi > N - 1 ? N - 1 : hi;
            lo = lo < 0 ? 0 : lo;
            if (lo <= hi) {
                jlo = (int)lo;
                jhi = (int)hi;
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
                cls = (unsigned char)(32 - __clz(hw));
                w = (long long)(jhi - jlo + 1);
                atomicAdd(&cnt[cls], 1);
            }
        }
        o.c[q] = c;
        o.f[q] = f;
        o.srel[q] = srel;
        o.a[q] = a;
        o.kv[q] = kv;
        o.jlo[q] = jlo;
        o.jhi[q] = jhi;
        o.ilo[q] = ilo;
        o.ihi[q] = ihi;
        o.cls[q] = cls;
    }
    // block sum of window lengths
    for (int d = 16; d > 0; d >>= 1) w += __shfl_down_sync(0xffffffffu, w, d);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += wsum[k];
        o.wpart[(size_t)s * nb + blockIdx.x] = t;
    }
    if (threadIdx.x < kNumClasses) o.blkcnt[((size_t)s * kNumClasses + threadIdx.x) * nb + blockIdx.x] = cnt[threadIdx.x];
}

// k_scan: per row, exclusive scan of the per-block class counts (one warp per class),
// class base offsets, and the total number of profile evaluations.
__global__ void k_scan(int nb, int* __restrict__ blkcnt, int* __restrict__ classbase, int* __restrict__ classcnt,
                       const long long* __restrict__ wpart, long long* __restrict__ evals) {
    __shared__ int tot[kNumClasses];
    const int s = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = warp; b < kNumClasses; b += blockDim.x >> 5) {
        int* row = blkcnt + ((size_t)s * kNumClasses + b) * nb;
        int run = 0;
        for (int base = 0; base < nb; base += 32) {
            const int k = base + lane;
            int v = k < nb ? row[k] : 0, incl = v;
            for (int d = 1; d < 32; d <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            if (k < nb) row[k] = run + incl - v;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) tot[b] = run;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < kNumClasses; ++b) {
            classbase[s * kNumClasses + b] = acc;
            classcnt[s * kNumClasses + b] = tot[b];
            acc += tot[b];
        }
    }
    if (evals && warp == 0) {
        long long acc = 0;
        for (int k = lane; k < nb; k += 32) acc += wpart[(size_t)s * nb + k];
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
        if (lane == 0) evals[s] = acc;
    }
}

// k_scatter: stable placement of kept lines into class buckets (centre order preserved).
__global__ void __launch_bounds__(256) k_scatter(int64_t L, int N, const unsigned char* __restrict__ cls,
                                                 const int* __restrict__ cpos, const int* __restrict__ blkoff,
                                                 const int* __restrict__ classbase, int nb, int* __restrict__ bidx,
                                                 int* __restrict__ bkey) {
    __shared__ int wcnt[8][kNumClasses];
    const int s = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < 8 * kNumClasses; k += blockDim.x) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const int b = (i < L) ? (int)cls[(size_t)s * L + i] : (int)kDropped;
    const unsigned same = __match_any_sync(0xffffffffu, b);
    const unsigned lt = (1u << lane) - 1u;
    const int lrank = __popc(same & lt);
    if (b < kNumClasses && lrank == 0) wcnt[warp][b] = __popc(same);
    __syncthreads();
    if (b < kNumClasses) {
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wcnt[w][b];
        const int pos = classbase[s * kNumClasses + b] + blkoff[((size_t)s * kNumClasses + b) * nb + blockIdx.x] +
                        before + lrank;
        const int c = cpos[i];
        bidx[(size_t)s * L + pos] = (int)i;
        bkey[(size_t)s * L + pos] = c < -1 ? -1 : (c > N ? N : c);
    }
}

// k_ranges: cum[s][b][ts] = position of the first line of class b whose centre key is
// >= (ts - 1) * kTile, ts = 0 .. nT + 2 (tiles -1 .. nT, with off-grid centres clamped).
__global__ void k_ranges(int n_sel, int64_t L, int nT, const int* __restrict__ bkey,
                         const int* __restrict__ classbase, const int* __restrict__ classcnt, int* __restrict__ cum) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int W = nT + 3;
    if (t >= (int64_t)n_sel * kNumClasses * W) return;
    const int ts = (int)(t % W);
    const int b = (int)((t / W) % kNumClasses);
    const int s = (int)(t / ((int64_t)W * kNumClasses));
    const int base = classbase[s * kNumClasses + b], n = classcnt[s * kNumClasses + b];
    const int* k = bkey + (size_t)s * L + base;
    const long long thr = (long long)(ts - 1) * kTile;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)k[mid] < thr) lo = mid + 1; else hi = mid;
    }
    cum[t] = base + lo;
}

// ---------------------------------------------------------------------------
// The profile kernel.
struct TileArgs {
    int N, nT;
    int64_t L;
    float lnq, q1, q2, q3;      // expm1(-x)/(-x) ~ 1 + d (q1 + d (q2 + d q3)), x = d lnq
    const int* cum;
    const int* bidx;
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
};

struct NearRec {
    float cf, f, klnq, a, srel, kv;
    int flags;       // klo | khi << 3 | check << 6 | series << 7 | full << 8
    int jlo, jhi;    // outer cut window (grid indices)
    int pad[3];
};

// far line: v = G_k * kvB + kvE1 (exact expm1 decomposition around the tile start),
// H by the far tier with the 1/(1 + 8 a^2 y^2) factor only when a^2 is not negligible.
// The 8 points are evaluated without branches so that their dependency chains
// interleave; MASKED lines (partial coverage or points near the cut) select with a mask.
template <bool EPS, bool MASKED>
__device__ __forceinline__ void far_line(const float4 p, float A8, int klo, int khi, bool chk, const float (&G)[8],
                                         float (&part)[8]) {
#pragma unroll
    for (int k = 0; k < kPtsPerThread; ++k) {
        const float v = fmaf(G[k], p.x, p.y);
        const float y = rcp_approx(fmaf(2.f * v, v, p.z));
        float l = p.w * y * fmaf(4.f, y, 2.f);
        if (EPS) {
            const float e = A8 * y * y;
            l *= fmaf(e, e - 1.f, 1.f);
        }
        if (MASKED) {
            bool ok = (k >= klo) & (k <= khi);
            if (chk) ok = ok & (l >= 1.f);
            l = ok ? l : 0.f;
        }
        part[k] += l;
    }
}

// near line: exact offset d = (j - c) - f and the expm1 series for v; the tiers of H
// branch per point.  Lines that do not cover the whole tile are culled per warp in
// 32-point segments (a warp's lanes own 32 consecutive points of each slot).
template <bool FULL, bool CHK>
__device__ __forceinline__ void near_line(const NearRec& r, int seg0, bool series, const float (&jf)[8],
                                          float q1, float q2, float q3, float lnq, float (&part)[8]) {
#pragma unroll
    for (int k = 0; k < kPtsPerThread; ++k) {
        if (!FULL) {
            const int lo = seg0 + k * kTileThreads;
            if (lo + 31 < r.jlo || lo > r.jhi) continue;
        }
        const float d = (jf[k] - r.cf) - r.f;
        float v;
        if (series) v = r.klnq * (d * fmaf(d, fmaf(d, fmaf(d, q3, q2), q1), 1.f));
        else v = r.kv * expm1f(-d * lnq);
        float l = r.srel * voigt_H_lean(v, r.a);
        if (CHK) l = (l >= 1.f) ? l : 0.f;
        part[k] += l;
    }
}

#ifndef MPSA_TILES_MINB
#define MPSA_TILES_MINB 3
#endif
template <int PREC>
__global__ void __launch_bounds__(kTileThreads, MPSA_TILES_MINB) k_tiles(TileArgs g) {
    __shared__ float4 sFarA[kTileThreads];
    __shared__ float2 sFarB[kTileThreads];
    __shared__ NearRec sNear[kTileThreads];
    __shared__ int sCnt[2][kTileThreads / 32];

    const int s = blockIdx.y;
    const int tile = blockIdx.x;
    const int J0 = tile * kTile;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t sL = (size_t)s * g.L;

    float jf[kPtsPerThread], G[kPtsPerThread], sum[kPtsPerThread], comp[kPtsPerThread], part[kPtsPerThread];
#pragma unroll
    for (int k = 0; k < kPtsPerThread; ++k) {
        const int off = k * kTileThreads + tid;
        jf[k] = (float)(J0 + off);
        G[k] = expm1f(-(float)off * g.lnq);
        sum[k] = 0.f;
        comp[k] = 0.f;
        part[k] = 0.f;
    }

    for (int b = 0; b < kNumClasses; ++b) {
        const int reach = 1 << b;
        int tlo = floordiv(J0 - reach + 1, kTile), thi = floordiv(J0 + kTile - 1 + reach - 1, kTile);
        tlo = max(tlo, -1);
        thi = min(thi, g.nT);
        if (tlo > thi) continue;
        const int* cum = g.cum + ((size_t)s * kNumClasses + b) * (g.nT + 3);
        const int beg = cum[tlo + 1], end = cum[thi + 2];
        for (int base = beg; base < end; base += kTileThreads) {
            // ---- set-up: one candidate line per thread
            const int pos = base + tid;
            bool isFar = false, isNear = false;
            float4 fa;
            float2 fb;
            NearRec nr;
            if (pos < end) {
                const size_t q = sL + (size_t)g.bidx[sL + pos];
                const int jlo = g.jlo[q], jhi = g.jhi[q];
                if (jhi >= J0 && jlo <= J0 + kTile - 1) {
                    const int c = g.c[q];
                    const float f = g.f[q], kv = g.kv[q], a = g.a[q], srel = g.srel[q];
                    const int klo = max(0, (jlo - J0) >> 8), khi = min(kPtsPerThread - 1, (jhi - J0) >> 8);
                    const int P0 = J0 + klo * kTileThreads, P1 = J0 + khi * kTileThreads + kTileThreads - 1;
                    const bool check = !(g.ilo[q] <= P0 && g.ihi[q] >= P1);
                    // distance from the centre x0 = c + f to the nearest point of the tile
                    // (far lines are evaluated at all 8 points, masked to [klo, khi])
                    const int T0 = J0, T1 = J0 + kTile - 1;
                    float dist;
                    bool red;
                    if (c + 1 <= T0) { dist = (float)(T0 - c) - f; red = true; }
                    else if (c >= T1) { dist = f + (float)(c - T1); red = false; }
                    else { dist = 0.f; red = true; }
                    float vmin = 0.f;
                    if (dist >= (float)kFarDist)
                        vmin = red ? -kv * expm1f(-dist * g.lnq) : kv * expm1f(dist * g.lnq);
                    const int flags = klo | (khi << 3) | (check ? 64 : 0) | ((klo == 0 && khi == kPtsPerThread - 1) ? 256 : 0);
                    if (dist >= (float)kFarDist && vmin >= kFarV) {
                        isFar = true;
                        const float D = (float)(J0 - c) - f;
                        const float x = D * g.lnq;
                        const float E1 = expm1f(-x), B = expf(-x);
                        const float A = a * a;
                        fa = make_float4(kv * B, kv * E1, fmaf(2.f, A, -1.f), srel * a * kInvSqrtPi);
                        const bool eps = 8.f * A * (1.f / 9.0e6f) > 1e-8f;   // (2 |z|^2 - 1)^2 >= 9e6 here
                        fb = make_float2(8.f * A, __int_as_float(flags | (eps ? 128 : 0)));
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
                        nr.flags = flags | (series ? 128 : 0);
                        nr.jlo = jlo;
                        nr.jhi = jhi;
                        nr.pad[0] = nr.pad[1] = nr.pad[2] = 0;
                    }
                }
            }
            const unsigned bf = __ballot_sync(0xffffffffu, isFar), bn = __ballot_sync(0xffffffffu, isNear);
            if (lane == 0) {
                sCnt[0][warp] = __popc(bf);
                sCnt[1][warp] = __popc(bn);
            }
            __syncthreads();
            int offF = 0, offN = 0, nFar = 0, nNear = 0;
#pragma unroll
            for (int w = 0; w < kTileThreads / 32; ++w) {
                const int cf = sCnt[0][w], cn = sCnt[1][w];
                if (w < warp) { offF += cf; offN += cn; }
                nFar += cf;
                nNear += cn;
            }
            const unsigned lt = (1u << lane) - 1u;
            if (isFar) {
                const int p = offF + __popc(bf & lt);
                sFarA[p] = fa;
                sFarB[p] = fb;
            }
            if (isNear) sNear[offN + __popc(bn & lt)] = nr;
            __syncthreads();

            // ---- evaluation: every thread, every compacted line, its 8 points
            for (int r = 0; r < nFar; ++r) {
                const float4 p = sFarA[r];
                const float2 q = sFarB[r];
                const int fl = __float_as_int(q.y);
                const int klo = fl & 7, khi = (fl >> 3) & 7;
                const bool chk = fl & 64, eps = fl & 128;
                const bool plain = (fl & 256) && !chk;     // all 8 points, no cut test
                if (eps) {
                    if (plain) far_line<true, false>(p, q.x, klo, khi, chk, G, part);
                    else far_line<true, true>(p, q.x, klo, khi, chk, G, part);
                } else {
                    if (plain) far_line<false, false>(p, q.x, klo, khi, chk, G, part);
                    else far_line<false, true>(p, q.x, klo, khi, chk, G, part);
                }
            }
            const int seg0 = J0 + warp * 32;
            for (int r = 0; r < nNear; ++r) {
                const NearRec nrr = sNear[r];
                const bool series = nrr.flags & 128;
                const bool full = nrr.flags & 256, chk = nrr.flags & 64;
                if (full) {
                    if (chk) near_line<true, true>(nrr, seg0, series, jf, g.q1, g.q2, g.q3, g.lnq, part);
                    else near_line<true, false>(nrr, seg0, series, jf, g.q1, g.q2, g.q3, g.lnq, part);
                } else {
                    if (chk) near_line<false, true>(nrr, seg0, series, jf, g.q1, g.q2, g.q3, g.lnq, part);
                    else near_line<false, false>(nrr, seg0, series, jf, g.q1, g.q2, g.q3, g.lnq, part);
                }
            }
            if (PREC == MPSA_PREC_FP32_COMPENSATED) {
                // fold the chunk's FP32 partial sums into the Kahan-compensated totals
#pragma unroll
                for (int k = 0; k < kPtsPerThread; ++k) {
                    const float y = part[k] - comp[k];
                    const float t = sum[k] + y;
                    comp[k] = (t - sum[k]) - y;
                    sum[k] = t;
                    part[k] = 0.f;
                }
            }
            __syncthreads();
        }
    }
    const float tp = expf(g.ln_tp[s]);
    float* out = g.out + (size_t)s * g.N;
#pragma unroll
    for (int k = 0; k < kPtsPerThread; ++k) {
        const int j = J0 + k * kTileThreads + tid;
        const float tot = (PREC == MPSA_PREC_FP32_COMPENSATED) ? (sum[k] - comp[k]) : part[k];
        if (j < g.N) out[j] = tp * tot;
    }
}

int g_init_mask = 0;

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
int synth_rows(mpsa_ctx* ctx, const double* pop, int n_sel, const int* d_sel, double lam0_nm, double R, int N,
               float* kappa, float* kc_out, int64_t* evals, const mpsa_synth_opts* opts, cudaStream_t st) {
    const double cut = (opts && opts->cut > 0) ? opts->cut : 1e-3;
    const double kcf = (opts && opts->kc_factor > 0) ? opts->kc_factor : 1e-2;
    const int prec = opts ? opts->precision : 0;
    if (prec != MPSA_PREC_FP32_COMPENSATED && prec != MPSA_PREC_FP32_NAIVE)
        return fail(MPSA_EINVAL, "synth: precision %d", prec);
    const int64_t L = ctx->L;
    const int n_sp = ctx->n_sp;
    const double lnq = log1p(1.0 / R);
    const int nT = (N + kTile - 1) / kTile;
    const int nb = (int)((L + 255) / 256);
    Scratch sc(st);
    int *c, *bidx, *bkey, *blkcnt, *classbase, *classcnt, *cum;
    float *f, *lamcm, *lnS, *av, *lnk0, *ln_tp;
    RowConst* rc;
    SpConst* spc;
    long long* wpart;
    PrepOut po;
    int r;
    const size_t SL = (size_t)n_sel * L;
    if ((r = sc.alloc(&c, L)) || (r = sc.alloc(&f, L)) || (r = sc.alloc(&lamcm, L)) ||
        (r = sc.alloc(&rc, n_sel)) || (r = sc.alloc(&spc, (size_t)n_sel * n_sp)) || (r = sc.alloc(&lnS, SL)) ||
        (r = sc.alloc(&av, SL)) || (r = sc.alloc(&lnk0, SL)) || (r = sc.alloc(&ln_tp, n_sel)) ||
        (r = sc.alloc(&po.c, SL)) || (r = sc.alloc(&po.f, SL)) || (r = sc.alloc(&po.srel, SL)) ||
        (r = sc.alloc(&po.a, SL)) || (r = sc.alloc(&po.kv, SL)) || (r = sc.alloc(&po.jlo, SL)) ||
        (r = sc.alloc(&po.jhi, SL)) || (r = sc.alloc(&po.ilo, SL)) || (r = sc.alloc(&po.ihi, SL)) ||
        (r = sc.alloc(&po.cls, SL)) || (r = sc.alloc(&blkcnt, (size_t)n_sel * kNumClasses * nb)) ||
        (r = sc.alloc(&wpart, (size_t)n_sel * nb)) || (r = sc.alloc(&classbase, (size_t)n_sel * kNumClasses)) ||
        (r = sc.alloc(&classcnt, (size_t)n_sel * kNumClasses)) || (r = sc.alloc(&bidx, SL)) ||
        (r = sc.alloc(&bkey, SL)) || (r = sc.alloc(&cum, (size_t)n_sel * kNumClasses * (nT + 3))))
        return r;
    po.blkcnt = blkcnt;
    po.wpart = wpart;

    const int lb = (int)((L + 255) / 256);
    k_place<<<lb, 256, 0, st>>>(L, ctx->d_lam, lam0_nm, lnq, c, f, lamcm);
    k_consts<<<(n_sel * n_sp + 127) / 128, 128, 0, st>>>(n_sel, d_sel, n_sp, ctx->d_sp_el, ctx->d_sp_stage,
                                                           ctx->n_el, ctx->d_el, pop, ctx->vturb, rc, spc);
    k_kappa0<<<dim3(lb, n_sel), 256, 0, st>>>(L, ctx->d_species, ctx->d_loggf, ctx->d_E, ctx->d_lgR, ctx->d_lgS,
                                               ctx->d_lgW, lamcm, n_sp, rc, spc, lnS, av, lnk0);
    k_median<<<n_sel, 1024, 0, st>>>(L, lnk0, (float)log(kcf), (float)log(cut), ln_tp, kc_out);
    k_prep<<<dim3(nb, n_sel), 256, 0, st>>>(L, N, (float)lnq, ctx->d_species, c, f, n_sp, spc, lnS, av, lnk0,
                                            ln_tp, nb, po);
    k_scan<<<n_sel, 32 * 8, 0, st>>>(nb, blkcnt, classbase, classcnt, wpart, (long long*)evals);
    k_scatter<<<dim3(nb, n_sel), 256, 0, st>>>(L, N, po.cls, c, blkcnt, classbase, nb, bidx, bkey);
    const int64_t nr = (int64_t)n_sel * kNumClasses * (nT + 3);
    k_ranges<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(n_sel, L, nT, bkey, classbase, classcnt, cum);
    TileArgs ta;
    ta.N = N;
    ta.nT = nT;
    ta.L = L;
    ta.lnq = (float)lnq;
    ta.q1 = (float)(-lnq / 2.0);
    ta.q2 = (float)(lnq * lnq / 6.0);
    ta.q3 = (float)(-lnq * lnq * lnq / 24.0);
    ta.cum = cum;
    ta.bidx = bidx;
    ta.c = po.c;
    ta.f = po.f;
    ta.srel = po.srel;
    ta.a = po.a;
    ta.kv = po.kv;
    ta.jlo = po.jlo;
    ta.jhi = po.jhi;
    ta.ilo = po.ilo;
    ta.ihi = po.ihi;
    ta.ln_tp = ln_tp;
    ta.out = kappa;
    prof_mark(ctx, MPSA_KERNEL_PROFILE, st);
    if (prec == MPSA_PREC_FP32_NAIVE) k_tiles<MPSA_PREC_FP32_NAIVE><<<dim3(nT, n_sel), kTileThreads, 0, st>>>(ta);
    else k_tiles<MPSA_PREC_FP32_COMPENSATED><<<dim3(nT, n_sel), kTileThreads, 0, st>>>(ta);
    prof_mark(ctx, MPSA_KERNEL_PROFILE, st);
    MPSA_CUDA_TRY(cudaGetLastError());
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
    for (int i = 0; i < ctx->n_sp; ++i)
        if (ctx->h_sp_el[i] >= ctx->n_el)
            return fail(MPSA_EINVAL, "synth_opacity: species %d refers to element %d of %d", i, ctx->h_sp_el[i], ctx->n_el);
    const int rows = ctx->n_comp * ctx->n_points;
    for (int i = 0; i < n_sel; ++i)
        if (sel[i] < 0 || sel[i] >= rows) return fail(MPSA_EINVAL, "synth_opacity: sel[%d] = %d of %d rows", i, sel[i], rows);
    int N, r;
    if ((r = check_grid(grid, &N))) return r;
    if ((size_t)n_sel * ctx->L >= (size_t)1 << 31)
        return fail(MPSA_EINVAL, "synth_opacity: n_sel * n_lines must stay below 2^31 (split the rows)");
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    int* d_sel;
    {
        Scratch s2(st);
        if ((r = s2.alloc(&d_sel, n_sel))) return r;
        MPSA_CUDA_TRY(cudaMemcpyAsync(d_sel, sel, n_sel * sizeof(int), cudaMemcpyHostToDevice, st));
        r = synth_rows(ctx, ctx->d_pop, n_sel, d_sel, grid->lambda0_nm, grid->R, N, kappa_out, kappa_c_out, evals_out,
                       opts, st);
    }
    return r;
}

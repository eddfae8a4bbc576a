// build_odf: opacity distribution functions (paper Sect. 2.3 and App. E).
//
// For each (row, interval) one CTA finds the order statistics at the sub-bin
// boundaries and the sums of all values below them, then forms the step means
//   m_s = (S(c_s n) - S(c_{s-1} n)) / (w_s n),
//   S(u) = sum of the floor(u) smallest values + (u - floor(u)) * x_(floor(u)).
// S(k) for an order statistic theta = x_(k) is sum_{x < theta} x + (k - #{x < theta}) theta.
//
// Order statistics: MSB radix multi-select on the FP32 bit patterns (values are
// non-negative, so the bit order is the value order), four levels of 11, 8, 8
// and 4 bits (bits 30..20, 19..12, 11..4, 3..0).  Every histogram bin carries,
// in one 64-bit shared-memory atomic, the count (high 24 bits) and the sum of the
// bits below the bin's prefix (low 40 bits).  Values that share the exponent E
// are integers in units of 2^(max(E,1)-150), so every partial sum inside an
// exponent group is exact integer arithmetic; only the sum across exponent
// groups (256 of them) is done in FP64.  Pass 1 reads the interval from HBM;
// passes 2-4 re-read it (from L2) and histogram only the values whose prefix
// matches a target's.  Zeros are counted in registers (no atomics).
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"

namespace mpsa {

namespace {

constexpr int kOdfThreads = 1024;
constexpr int kMaxSteps = 32;
constexpr int kMaxTargets = kMaxSteps - 1;
constexpr int kL1Bins = 2048;
constexpr unsigned long long kOne = 1ull << 40;
constexpr unsigned long long kLowMask = kOne - 1;

struct Target {
    long long k;          // rank (0-based) of the order statistic
    int slot;             // distinct-prefix slot at the current level
    unsigned prefix;      // bits resolved so far
    long long cnt_lt;     // values below the current prefix range
    unsigned long long iv_lt;   // exact sum (group units) of values of the target's exponent group below it
    int total;            // 1 when k >= n (S is the total)
};

__device__ __forceinline__ unsigned long long group_base(unsigned E) { return E >= 1 ? (1ull << 23) : 0ull; }

__global__ void __launch_bounds__(kOdfThreads) k_odf(const float* __restrict__ kappa, int64_t N, int K,
                                                     const int64_t* __restrict__ bounds, int n_steps,
                                                     const double* __restrict__ cw, const double* __restrict__ w,
                                                     double* __restrict__ out) {
    extern __shared__ unsigned long long sm[];
    unsigned long long* h1 = sm;                                  // [2048]
    unsigned long long* h2 = sm + kL1Bins;                        // [kMaxTargets][256]
    __shared__ int cbefore[kL1Bins];
    __shared__ short slot1[kL1Bins];
    __shared__ unsigned long long gsum[256];
    __shared__ double gpre[257];
    __shared__ Target tg[kMaxTargets];
    __shared__ unsigned dpre[kMaxTargets];      // distinct prefixes of the current level
    __shared__ int n_distinct;
    __shared__ long long s_zero;
    __shared__ int wtot[32];

    const int k = blockIdx.x, row = blockIdx.y;
    const int64_t b0 = bounds[k], b1 = bounds[k + 1];
    const long long n = b1 - b0;
    const float* x = kappa + (size_t)row * N + b0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt = n_steps - 1;

    for (int i = tid; i < kL1Bins; i += kOdfThreads) { h1[i] = 0ull; slot1[i] = -1; }
    if (tid == 0) s_zero = 0;
    __syncthreads();

    // ---- pass 1: 11-bit histogram with exact low-bit sums
    long long zeros = 0;
    for (long long i = tid; i < n; i += kOdfThreads) {
        const unsigned bits = __float_as_uint(__ldg(x + i)) & 0x7fffffffu;
        if (bits == 0u) { ++zeros; continue; }
        atomicAdd(&h1[bits >> 20], kOne | (unsigned long long)(bits & 0xfffffu));
    }
    for (int d = 16; d > 0; d >>= 1) zeros += __shfl_down_sync(0xffffffffu, zeros, d);
    if (lane == 0 && zeros) atomicAdd((unsigned long long*)&s_zero, (unsigned long long)zeros);
    __syncthreads();
    if (tid == 0) h1[0] += (unsigned long long)s_zero << 40;
    __syncthreads();

    // ---- exclusive scan of level-1 counts (2 bins per thread)
    {
        const int c0 = (int)(h1[2 * tid] >> 40), c1 = (int)(h1[2 * tid + 1] >> 40);
        int v = c0 + c1, incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        if (lane == 31) wtot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int t = wtot[lane], ti = t;
            for (int d = 1; d < 32; d <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, ti, d);
                if (lane >= d) ti += y;
            }
            wtot[lane] = ti - t;
        }
        __syncthreads();
        const int ex = wtot[warp] + incl - v;
        cbefore[2 * tid] = ex;
        cbefore[2 * tid + 1] = ex + c0;
    }
    // exact per-exponent-group sums in group units
    if (tid < 256) {
        unsigned long long acc = 0;
        for (int m = 0; m < 8; ++m) {
            const unsigned long long h = h1[tid * 8 + m];
            const unsigned long long base = group_base(tid) + ((unsigned long long)m << 20);
            acc += (h >> 40) * base + (h & kLowMask);
        }
        gsum[tid] = acc;
    }
    // targets
    if (tid < nt) {
        Target t;
        const double u = cw[tid + 1] * (double)n;
        t.k = (long long)floor(u);
        t.total = t.k >= n;
        t.slot = -1;
        t.prefix = 0;
        t.cnt_lt = 0;
        t.iv_lt = 0;
        tg[tid] = t;
    }
    __syncthreads();
    if (warp == 0) {
        // FP64 exclusive prefix over the 256 exponent groups
        double loc[8], run = 0.0;
        for (int m = 0; m < 8; ++m) {
            const int E = lane * 8 + m;
            loc[m] = (double)gsum[E] * ldexp(1.0, (E >= 1 ? E : 1) - 150);
        }
        double tot = 0.0;
        for (int m = 0; m < 8; ++m) tot += loc[m];
        double incl = tot;
        for (int d = 1; d < 32; d <<= 1) {
            double y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        run = incl - tot;
        for (int m = 0; m < 8; ++m) {
            gpre[lane * 8 + m] = run;
            run += loc[m];
        }
        if (lane == 31) gpre[256] = run;
    }
    // locate each target's level-1 bin
    for (int t = 0; t < nt; ++t) {
        if (tg[t].total) continue;
        const long long kk = tg[t].k;
        for (int bb = 2 * tid; bb < 2 * tid + 2; ++bb) {
            const long long c = (long long)(h1[bb] >> 40);
            if (c > 0 && cbefore[bb] <= kk && kk < cbefore[bb] + c) {
                tg[t].prefix = (unsigned)bb << 20;
                tg[t].cnt_lt = cbefore[bb];
                // exact sum of the bins of the same exponent group below bb
                unsigned long long acc = 0;
                for (int m = bb & ~7; m < bb; ++m) {
                    const unsigned long long h = h1[m];
                    acc += (h >> 40) * (group_base(bb >> 3) + ((unsigned long long)(m & 7) << 20)) + (h & kLowMask);
                }
                tg[t].iv_lt = acc;
            }
        }
    }
    __syncthreads();

    // ---- levels 2..4
    const int shifts[3] = {12, 4, 0};
    const int widths[3] = {8, 8, 4};
    for (int lvl = 0; lvl < 3; ++lvl) {
        const int sh = shifts[lvl], wb = widths[lvl];
        const int hiShift = sh + wb;      // bits at and above hiShift are the resolved prefix
        const int nbins = 1 << wb;
        // distinct prefixes of the active targets
        if (tid == 0) {
            int nd = 0;
            for (int t = 0; t < nt; ++t) {
                if (tg[t].total) continue;
                int f = -1;
                for (int q = 0; q < nd; ++q)
                    if (dpre[q] == tg[t].prefix) f = q;
                if (f < 0) { dpre[nd] = tg[t].prefix; f = nd++; }
                tg[t].slot = f;
            }
            n_distinct = nd;
        }
        __syncthreads();
        const int nd = n_distinct;
        for (int i = tid; i < nd * 256; i += kOdfThreads) h2[i] = 0ull;
        if (lvl == 0)
            for (int q = tid; q < nd; q += kOdfThreads) slot1[dpre[q] >> 20] = (short)q;
        __syncthreads();
        if (nd > 0) {
            for (long long i = tid; i < n; i += kOdfThreads) {
                const unsigned bits = __float_as_uint(__ldg(x + i)) & 0x7fffffffu;
                if (bits == 0u || slot1[bits >> 20] < 0) continue;
                const unsigned pre = (bits >> hiShift) << hiShift;
                int q = -1;
                if (lvl == 0) q = slot1[bits >> 20];
                else
                    for (int r = 0; r < nd; ++r)
                        if (dpre[r] == pre) q = r;
                if (q < 0) continue;
                const unsigned sub = (bits >> sh) & (unsigned)(nbins - 1);
                const unsigned long long low = sh ? (bits & ((1u << sh) - 1u)) : 0u;
                atomicAdd(&h2[q * 256 + sub], kOne | low);
            }
        }
        __syncthreads();
        // zeros belong to the all-zero prefix
        if (tid < nd && dpre[tid] == 0u) h2[tid * 256] += (unsigned long long)s_zero << 40;
        __syncthreads();
        // resolve each target inside its slot (one thread per target; <= 256 bins)
        if (tid < nt && !tg[tid].total) {
            Target t = tg[tid];
            const unsigned long long* h = h2 + t.slot * 256;
            long long before = t.cnt_lt;
            const unsigned E = t.prefix >> 23;
            // integer value of the prefix (without the low bits) in group units
            const unsigned long long pbase = group_base(E) + (t.prefix & 0x7fffffu);
            for (int bb = 0; bb < nbins; ++bb) {
                const long long c = (long long)(h[bb] >> 40);
                if (t.k < before + c) {
                    t.prefix |= (unsigned)bb << sh;
                    break;
                }
                before += c;
                t.iv_lt += (unsigned long long)c * (pbase + ((unsigned long long)bb << sh)) + (h[bb] & kLowMask);
            }
            t.cnt_lt = before;
            tg[tid] = t;
        }
        __syncthreads();
    }

    // ---- step means
    if (tid < n_steps) {
        const int s = tid;
        auto S = [&](int bidx) -> double {   // S(c_bidx * n)
            if (bidx == 0) return 0.0;
            if (bidx == n_steps) return gpre[256];
            const Target& t = tg[bidx - 1];
            if (t.total) return gpre[256];
            const unsigned E = t.prefix >> 23;
            const double unit = ldexp(1.0, (E >= 1 ? (int)E : 1) - 150);
            const double theta = (double)__uint_as_float(t.prefix);
            const double below = gpre[E] + (double)t.iv_lt * unit;
            const double u = cw[bidx] * (double)n;
            return below + (double)(t.k - t.cnt_lt) * theta + (u - (double)t.k) * theta;
        };
        const double m = (S(s + 1) - S(s)) / (w[s] * (double)n);
        out[((size_t)row * K + k) * n_steps + s] = m;
    }
}

}  // namespace

}  // namespace mpsa

using namespace mpsa;

extern "C" int build_odf(mpsa_ctx* ctx, const float* kappa, int32_t n_rows, int64_t N, int32_t K,
                         const int64_t* bounds, int32_t n_steps, const double* widths, int32_t mean_kind,
                         double* odf_out, void* stream) {
    if (!ctx || !kappa || !bounds || !widths || !odf_out) return fail(MPSA_EINVAL, "build_odf: NULL argument");
    if (n_rows < 1 || N < 1 || K < 1) return fail(MPSA_EINVAL, "build_odf: n_rows %d N %lld K %d", n_rows, (long long)N, K);
    if (n_steps < 1 || n_steps > kMaxSteps) return fail(MPSA_EINVAL, "build_odf: n_steps = %d (1..%d)", n_steps, kMaxSteps);
    if (mean_kind != MPSA_MEAN_ARITH)
        return fail(MPSA_EINVAL, "build_odf: mean_kind %d not available (arithmetic only)", mean_kind);
    if (bounds[0] < 0 || bounds[K] > N) return fail(MPSA_EINVAL, "build_odf: bounds outside [0, N]");
    for (int k = 0; k < K; ++k) {
        const int64_t len = bounds[k + 1] - bounds[k];
        if (len < 1) return fail(MPSA_EINVAL, "build_odf: bounds not strictly increasing at %d", k);
        if (len >= (1 << 21)) return fail(MPSA_EINVAL, "build_odf: interval %d has %lld points (max 2^21-1)", k, (long long)len);
    }
    // cumulative widths: FP64 left-to-right partial sums, last forced to 1
    std::vector<double> cw(n_steps + 1);
    double acc = 0.0;
    cw[0] = 0.0;
    for (int s = 0; s < n_steps; ++s) {
        if (!(widths[s] > 0) || !isfinite(widths[s])) return fail(MPSA_EINVAL, "build_odf: widths[%d] = %g", s, widths[s]);
        acc = acc + widths[s];
        cw[s + 1] = acc;
    }
    if (fabs(acc - 1.0) > 1e-12) return fail(MPSA_EINVAL, "build_odf: widths sum to %.17g", acc);
    cw[n_steps] = 1.0;
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    int64_t* d_b;
    double *d_cw, *d_w;
    int r;
    if ((r = sc.alloc(&d_b, K + 1)) || (r = sc.alloc(&d_cw, n_steps + 1)) || (r = sc.alloc(&d_w, n_steps))) return r;
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_b, bounds, (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_cw, cw.data(), (n_steps + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_w, widths, n_steps * sizeof(double), cudaMemcpyHostToDevice, st));
    const size_t smem = (kL1Bins + (size_t)(n_steps - 1 > 0 ? n_steps - 1 : 1) * 256) * sizeof(unsigned long long);
    static unsigned attr_set = 0;   // one bit per device
    if (!(attr_set & (1u << (ctx->device & 31)))) {
        MPSA_CUDA_TRY(cudaFuncSetAttribute(k_odf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)((kL1Bins + kMaxTargets * 256) * sizeof(unsigned long long))));
        attr_set |= 1u << (ctx->device & 31);
    }
    prof_mark(ctx, MPSA_KERNEL_ODF, st);
    k_odf<<<dim3(K, n_rows), kOdfThreads, smem, st>>>(kappa, N, K, d_b, n_steps, d_cw, d_w, odf_out);
    prof_mark(ctx, MPSA_KERNEL_ODF, st);
    MPSA_CUDA_TRY(cudaGetLastError());
    return MPSA_OK;
}

// build_odf: opacity distribution functions (paper Sect. 2.3 and App. E).
//
// Two kernels.  k_odf_gather (further below) serves both kinds of mean with at most 12 steps
// on intervals of at most 65,536 points by a count pass and a gather pass; k_odf, the exact
// multi-select described here, serves every other case and the intervals the gather leaves.
//
// For each (row, interval) one CTA finds the order statistics at the sub-bin
// boundaries and the sums of all values below them, then forms the step means
//   m_s = (S(c_s n) - S(c_{s-1} n)) / (w_s n),
//   S(u) = sum of the floor(u) smallest values + (u - floor(u)) * x_(floor(u)).
// For an order statistic theta = x_(k): S(k) = sum_{x < theta} x + (k - #{x < theta}) theta.
//
// Order statistics: MSB radix multi-select on the FP32 bit patterns (values are
// non-negative, so the bit order is the value order) over four levels of 12, 7, 6
// and 6 bits (bits 30..19, 18..12, 11..6, 5..0).  Every histogram bin carries the
// count and the exact sum of the bits below the bin's prefix, the latter as two
// 32-bit sums (of bits >> 10 and of bits & 1023): 32-bit shared-memory atomics are
// native and keep their rate when many lanes hit one bin, while 64-bit ones are not.
// Values of one exponent E are integers in units of 2^(max(E,1)-150), so every partial
// sum inside an exponent group is exact integer arithmetic; only the sum across the 256
// exponent groups is FP64.
//
// Passes over the interval: pass 1 (from HBM) builds the level-1 histogram; pass 2
// (from L2) copies the values that fall into a target's level-1 bin into a
// shared-memory candidate buffer; levels 2-4 then run on that buffer.  If the
// candidates do not fit, the next level re-reads the interval instead.  Each warp
// reads 512 contiguous bytes per load; the 32 lanes of a warp aggregate their
// histogram adds by bin (match + reduce) so that one atomic per distinct bin is
// issued and no two lanes of a warp hit the same address.
//
// Geometric means (exp of the same integral of ln x) reuse the order statistics: one
// more pass (from L2) sums ln x of the positive values between consecutive distinct
// order statistics, exactly in 2^-30 fixed point, and
//   G(u) = sum_{0 < x < theta} ln x + (u - #{x < theta}) ln theta   (u at or above the zeros);
// a sub-bin that reaches into the zero values has geometric mean 0.
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace mpsa {

namespace {

constexpr int kOdfThreads = 512;
constexpr int kOdfWarps = kOdfThreads / 32;
constexpr int kMaxSteps = 32;
constexpr int kMaxTargets = kMaxSteps - 1;
constexpr int kL1Shift = 19;                       // level 1: bits 30..19
constexpr int kL1Bins = 1 << (31 - kL1Shift);      // 4096
constexpr int kL1PerGroup = 1 << (23 - kL1Shift);  // level-1 bins per exponent: 16
constexpr int kL2Bins = 128;                       // widest deeper level (7 bits)
constexpr int kMinSlots = 4;
#ifndef ODF_KCAND
#define ODF_KCAND 6144
#endif
constexpr int kCand = ODF_KCAND;                   // candidate buffer (32-bit patterns)
constexpr long long kMaxInterval = 1ll << 21;      // count < 2^24 and low-bit sums < 2^40 per bin
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxOdfRows = 65535;                // gridDim.y of the ODF launch
// The first output word of an interval that k_odf_gather leaves to k_odf: a NaN pattern that
// arithmetic never produces (its payload is not the canonical one).
constexpr unsigned long long kOdfRedo = 0x7ff40d0f0d0f0d0full;
constexpr int kMaxDevices = 64;

struct Target {
    long long k;                 // rank (0-based) of the order statistic
    long long cnt_lt;            // values below the current prefix range
    unsigned long long iv_lt;    // exact sum (group units) of the group's values below the prefix range
    long long cnt_in;            // values inside the current prefix range
    unsigned prefix;             // bits resolved so far
    int slot;                    // distinct-prefix slot at the current level
    int total;                   // 1 when k >= n (S is the total)
};

__device__ __forceinline__ unsigned long long group_base(unsigned E) { return E >= 1 ? (1ull << 23) : 0ull; }

// Visit every value of x[0..n) once, warp-coalesced: each warp owns a contiguous range of
// the 16-byte-aligned body and lane l reads float4 l, l+32, ... of it (512 contiguous bytes
// per warp and load), U loads in flight per lane before any is consumed.  The unaligned
// head and tail (< 4 values each) go to threads 0..3.  Every lane of a warp makes the same
// number of calls f(bits, valid), so warp-wide collectives inside f are safe.
template <class F>
__device__ __forceinline__ void for_each_value(const float* __restrict__ x, long long n, F&& f) {
    constexpr int U = 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned mis = (unsigned)(((uintptr_t)x >> 2) & 3u);
    long long head = mis ? (long long)(4u - mis) : 0;
    if (head > n) head = n;
    const float4* body = reinterpret_cast<const float4*>(x + head);
    const long long nv = (n - head) >> 2;
    const long long per = (((nv + kOdfWarps - 1) / kOdfWarps) + 31) & ~31ll;   // float4 per warp
    const long long w0 = (long long)warp * per, w1 = min(w0 + per, nv);
    for (long long it = w0; it < w0 + per; it += 32 * U) {
        float4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = it + 32 * u + lane;
            q[u] = i < w1 ? __ldg(body + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool v = it + 32 * u + lane < w1;
            f(__float_as_uint(q[u].x), v);
            f(__float_as_uint(q[u].y), v);
            f(__float_as_uint(q[u].z), v);
            f(__float_as_uint(q[u].w), v);
        }
    }
    const long long t0 = head + (nv << 2);
    f(tid < head ? __float_as_uint(__ldg(x + tid)) : 0u, tid < head);
    f(t0 + tid < n ? __float_as_uint(__ldg(x + t0 + tid)) : 0u, t0 + tid < n);
}

// A histogram of nb bins in shared memory: per bin the count and the sum of the values
// low parts (each < 2^20), kept exactly as two 32-bit sums of (low >> 10) and (low & 1023):
// an interval has fewer than 2^21 values, so neither sum can overflow.
struct Hist {
    unsigned* c;
    unsigned* hi;
    unsigned* lo;
    __device__ __forceinline__ void add(int k, unsigned n, unsigned shi, unsigned slo) const {
        atomicAdd(c + k, n);
        if (shi) atomicAdd(hi + k, shi);
        if (slo) atomicAdd(lo + k, slo);
    }
    __device__ __forceinline__ unsigned long long count(int k) const { return c[k]; }
    __device__ __forceinline__ unsigned long long low(int k) const {
        return ((unsigned long long)hi[k] << 10) + lo[k];
    }
    __device__ __forceinline__ void zero(int k) const { c[k] = 0u; hi[k] = 0u; lo[k] = 0u; }
};

// Histogram passes read the interval warp-coalesced (512 contiguous bytes per warp and
// load).  Neighbouring lanes then often hit the same bin; 32-bit shared atomics resolve
// that in hardware at full rate (a probe on this GPU measured 5e12 adds/s on one address),
// so the coalesced layout beats one contiguous chunk per thread, whose loads touch 32 lines
// per instruction (pass 1 of 8 rows: 0.17 ms against 0.27 ms).  Each lane still merges the
// runs inside its float4 before its atomics.

// Per-thread run merging of histogram adds: consecutive values of a thread that fall
// into the same bin are summed in registers and flushed with one set of atomics per run.
struct RunAdd {
    int key = -1;
    unsigned n = 0, shi = 0, slo = 0;
    __device__ __forceinline__ void add(const Hist& h, int k, unsigned low) {
        if (k != key) {
            if (key >= 0) h.add(key, n, shi, slo);
            key = k;
            n = shi = slo = 0u;
        }
        ++n;
        shi += low >> 10;
        slo += low & 1023u;
    }
    __device__ __forceinline__ void flush(const Hist& h) {
        if (key >= 0) h.add(key, n, shi, slo);
        key = -1;
    }
};

// Warp-aggregated append to the candidate buffer (one shared atomic per warp and call).
__device__ __forceinline__ void agg_append(unsigned* __restrict__ cand, int* n_cand, bool take, unsigned bits,
                                           int lane) {
    const unsigned m = __ballot_sync(kFull, take);
    if (m == 0u) return;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(n_cand, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (take) {
        const int pos = base + __popc(m & ((1u << lane) - 1u));
        if (pos < kCand) cand[pos] = bits;
    }
}

// Append every value x (bits with the sign cleared) of x[0..n) with take(x) to the candidate
// buffer.  Warp-coalesced like for_each_value; each lane marks the takes among its 16 loaded
// values, a warp scan gives every lane its offset, and one lane reserves the warp's total
// with a single atomic per 512 values (instead of one atomic round trip per warp and value).
template <class P>
__device__ __forceinline__ void collect_values(const float* __restrict__ x, long long n, unsigned* __restrict__ cand,
                                               int* n_cand, P&& take) {
    constexpr int U = 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned mis = (unsigned)(((uintptr_t)x >> 2) & 3u);
    long long head = mis ? (long long)(4u - mis) : 0;
    if (head > n) head = n;
    const float4* body = reinterpret_cast<const float4*>(x + head);
    const long long nv = (n - head) >> 2;
    const long long per = (((nv + kOdfWarps - 1) / kOdfWarps) + 31) & ~31ll;   // float4 per warp
    const long long w0 = (long long)warp * per, w1 = min(w0 + per, nv);
    for (long long it = w0; it < w0 + per; it += 32 * U) {
        unsigned b[4 * U];
        unsigned m = 0u;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = it + 32 * u + lane;
            const float4 q = i < w1 ? __ldg(body + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            b[4 * u] = __float_as_uint(q.x) & 0x7fffffffu;
            b[4 * u + 1] = __float_as_uint(q.y) & 0x7fffffffu;
            b[4 * u + 2] = __float_as_uint(q.z) & 0x7fffffffu;
            b[4 * u + 3] = __float_as_uint(q.w) & 0x7fffffffu;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool v = it + 32 * u + lane < w1;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (v && take(b[4 * u + c])) m |= 1u << (4 * u + c);
        }
        const int cnt = __popc(m);
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        if (total == 0) continue;
        int base = 0;
        if (lane == 31) base = atomicAdd(n_cand, total);
        int pos = __shfl_sync(kFull, base, 31) + incl - cnt;
#pragma unroll
        for (int e = 0; e < 4 * U; ++e)
            if ((m >> e) & 1u) {
                if (pos < kCand) cand[pos] = b[e];
                ++pos;
            }
    }
    const long long t0 = head + (nv << 2);
    const unsigned hb = tid < head ? __float_as_uint(__ldg(x + tid)) & 0x7fffffffu : 0u;
    agg_append(cand, n_cand, tid < head && take(hb), hb, lane);
    const unsigned tb = t0 + tid < n ? __float_as_uint(__ldg(x + t0 + tid)) & 0x7fffffffu : 0u;
    agg_append(cand, n_cand, t0 + tid < n && take(tb), tb, lane);
}

// ln x of a positive finite FP32 value given by its bits: x = 2^e m with m in
// [1/sqrt 2, sqrt 2), ln x = e ln 2 (FP64, exact e) + ln m (FP32 logf, |ln m| < 0.35),
// so the absolute error stays near 2e-8 whatever the exponent.
__device__ __forceinline__ double ln_f32_bits(unsigned bits) {
    int e = 0;
    if (bits < 0x00800000u) {   // subnormal: scale by 2^23 (exact)
        bits = __float_as_uint(__uint_as_float(bits) * 8388608.0f);
        e = -23;
    }
    e += (int)(bits >> 23) - 127;
    unsigned mb = (bits & 0x7fffffu) | 0x3f800000u;
    if (mb > 0x3fb504f3u) {   // m > sqrt 2: halve it
        mb -= 0x00800000u;
        e += 1;
    }
    return (double)e * 0.69314718055994530942 + (double)logf(__uint_as_float(mb));
}

// ln x of a positive finite FP32 value in fixed point, units of 2^-30 (|result| < 2^37):
// x = 2^e m with m in [1/sqrt 2, sqrt 2); e ln 2 from the integer round(ln 2 * 2^40) (error
// below 1e-10) plus ln m = logf(m) (|ln m| < 0.35, FP32 resolution about 3e-8).
constexpr long long kLn2Q40 = 762123384786ll;
constexpr long long kLnOffset = 1ll << 37;
__device__ __forceinline__ long long ln_q30(unsigned bits) {
    int e = 0;
    if (bits < 0x00800000u) {   // subnormal: scale by 2^23 (exact)
        bits = __float_as_uint(__uint_as_float(bits) * 8388608.0f);
        e = -23;
    }
    e += (int)(bits >> 23) - 127;
    unsigned mb = (bits & 0x7fffffu) | 0x3f800000u;
    if (mb > 0x3fb504f3u) {
        mb -= 0x00800000u;
        e += 1;
    }
    const long long el = ((long long)e * kLn2Q40 + 512) >> 10;
    return el + (long long)__float2int_rn(logf(__uint_as_float(mb)) * 1073741824.0f);
}

// One warp resolves one target inside its slot's 2^wb-bin histogram h (packed counts and
// low-bit sums): finds the sub-bin holding rank t.k and adds the counts and exact sums
// of all lower sub-bins.
__device__ __forceinline__ void resolve_warp(Target& t, const Hist& h, int wb, int sh, int lane) {
    const int nb = 1 << wb;
    const int per = nb >= 32 ? nb / 32 : 1;
    const unsigned E = t.prefix >> 23;
    const unsigned long long pbase = group_base(E) + (t.prefix & 0x7fffffu);
    long long cnt = 0;
    for (int m = 0; m < per; ++m) {
        const int b = lane * per + m;
        if (b < nb) cnt += (long long)h.count(b);
    }
    long long incl = cnt;
    for (int d = 1; d < 32; d <<= 1) {
        long long y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    const long long before = incl - cnt + t.cnt_lt;
    const bool mine = cnt > 0 && (t.k >= before) && (t.k < before + cnt);
    const unsigned owner = __ballot_sync(kFull, mine);
    const int ow = owner ? __ffs(owner) - 1 : 31;
    unsigned long long ivs = 0;
    long long cnt_below = 0;
    int found = 0;
    if (lane < ow) {
        for (int m = 0; m < per; ++m) {
            const int b = lane * per + m;
            if (b < nb) ivs += h.count(b) * (pbase + ((unsigned long long)b << sh)) + h.low(b);
        }
    } else if (lane == ow) {
        long long run = before;
        for (int m = 0; m < per; ++m) {
            const int b = lane * per + m;
            if (b >= nb) break;
            const long long c = (long long)h.count(b);
            if (t.k < run + c) { found = b; break; }
            run += c;
            ivs += (unsigned long long)c * (pbase + ((unsigned long long)b << sh)) + h.low(b);
        }
        cnt_below = run;
    }
    for (int d = 16; d > 0; d >>= 1) ivs += __shfl_down_sync(kFull, ivs, d);
    found = __shfl_sync(kFull, found, ow);
    cnt_below = __shfl_sync(kFull, cnt_below, ow);
    if (lane == 0) {
        t.iv_lt += ivs;
        t.cnt_lt = cnt_below;
        t.cnt_in = (long long)h.count(found);
        t.prefix |= (unsigned)found << sh;
    }
}

// CTAs per SM the kernel is compiled for.  Three fit the shared memory (71 KB each for 12
// steps) but force 40 registers and spills; with the batched candidate collection two CTAs
// (62 registers) are as fast for the arithmetic means and faster for the geometric ones.
#ifndef ODF_MINB
#define ODF_MINB 2
#endif
__global__ void __launch_bounds__(kOdfThreads, ODF_MINB) k_odf(const float* __restrict__ kappa, int64_t N, int K,
                                                     const int64_t* __restrict__ bounds, int n_steps,
                                                     const double* __restrict__ cw, const double* __restrict__ w,
                                                     double* __restrict__ out, int geom, int redo_only) {
    extern __shared__ __align__(16) unsigned sm[];
    const int nt = n_steps - 1;
    const int nslots = nt > kMinSlots ? nt : kMinSlots;
    // Two phases share the dynamic shared memory: until the targets are located it holds the
    // level-1 histogram and its prefix counts; from then on (both dead) the candidates, the
    // deeper histograms and the slot tables (64 KB for 12 steps).
    const Hist h1{sm, sm + kL1Bins, sm + 2 * kL1Bins};                 // [4096] each
    int* cincl = reinterpret_cast<int*>(sm + 3 * kL1Bins);             // [4096] inclusive prefix counts
    const int n2 = nslots * kL2Bins;
    unsigned* cand = sm;                                               // [kCand]
    unsigned* h2base = sm + kCand;
    const Hist h2{h2base, h2base + n2, h2base + 2 * n2};               // [nslots][128] each
    short* slot1 = reinterpret_cast<short*>(h2base + 3 * n2);          // [4096]: level-1 bin -> slot
    short* slot2 = slot1 + kL1Bins;                                    // [nslots][128]: 19-bit prefix -> slot
    __shared__ unsigned tbits[kL1Bins / 32];                 // bitmap of the targets' level-1 bins
    __shared__ unsigned long long gsum[256];
    __shared__ double gpre[257];
    __shared__ Target tg[kMaxTargets];
    __shared__ unsigned dpre[kMaxTargets];
    __shared__ int n_distinct, n_cand;
    __shared__ unsigned s_zero;
    __shared__ int wtot[kOdfWarps];
    __shared__ unsigned thr[kMaxTargets];       // geometric pass: distinct order statistics, ascending
    __shared__ double lsum[kMaxTargets + 1];    // geometric pass: inclusive prefix sums of ln x per bucket
    __shared__ unsigned gacc[5][kMaxTargets + 1];   // geometric pass: exact fixed-point sums per bucket
    __shared__ int n_thr;

    const int k = blockIdx.x, row = blockIdx.y;
    // after k_odf_gather: only the intervals it marked for this kernel (a uniform early exit)
    if (redo_only && *reinterpret_cast<const unsigned long long*>(out + ((size_t)row * K + k) * n_steps) != kOdfRedo)
        return;
    const int64_t b0 = bounds[k], b1 = bounds[k + 1];
    const long long n = b1 - b0;
    const float* x = kappa + (size_t)row * N + b0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int i = tid; i < kL1Bins; i += kOdfThreads) h1.zero(i);
    if (tid < kL1Bins / 32) tbits[tid] = 0u;
    if (tid == 0) { s_zero = 0u; n_cand = 0; }
    __syncthreads();

    // ---- pass 1 (HBM): level-1 histogram with exact low-bit sums (zeros land in bin 0)
    {
        unsigned zeros = 0;
        RunAdd run;
        for_each_value(x, n, [&](unsigned bits, bool valid) {
            if (!valid) return;
            bits &= 0x7fffffffu;
            zeros += bits == 0u ? 1u : 0u;
            run.add(h1, (int)(bits >> kL1Shift), bits & ((1u << kL1Shift) - 1u));
        });
        run.flush(h1);
        zeros = __reduce_add_sync(kFull, zeros);
        if (lane == 0 && zeros) atomicAdd(&s_zero, zeros);
    }
    __syncthreads();

    // ---- inclusive scan of the level-1 counts (8 bins per thread)
    {
        int c[8], v = 0;
        for (int m = 0; m < 8; ++m) { c[m] = (int)h1.count(8 * tid + m); v += c[m]; }
        int incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            int y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        if (lane == 31) wtot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int t = lane < kOdfWarps ? wtot[lane] : 0, ti = t;
            for (int d = 1; d < 32; d <<= 1) {
                int y = __shfl_up_sync(kFull, ti, d);
                if (lane >= d) ti += y;
            }
            if (lane < kOdfWarps) wtot[lane] = ti - t;
        }
        __syncthreads();
        int run = wtot[warp] + incl - v;
        for (int m = 0; m < 8; ++m) { run += c[m]; cincl[8 * tid + m] = run; }
    }
    if (tid < 256) {
        unsigned long long acc = 0;
        for (int m = 0; m < kL1PerGroup; ++m) {
            const int b = tid * kL1PerGroup + m;
            acc += h1.count(b) * (group_base(tid) + ((unsigned long long)m << kL1Shift)) + h1.low(b);
        }
        gsum[tid] = acc;
    }
    __syncthreads();
    if (warp == 0) {
        // FP64 exclusive prefix over the 256 exponent groups (the only FP64 reduction)
        double loc[8];
        double tot = 0.0;
        for (int m = 0; m < 8; ++m) {
            const int E = lane * 8 + m;
            loc[m] = (double)gsum[E] * ldexp(1.0, (E >= 1 ? E : 1) - 150);
            tot += loc[m];
        }
        double incl = tot;
        for (int d = 1; d < 32; d <<= 1) {
            double y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        double run = incl - tot;
        for (int m = 0; m < 8; ++m) {
            gpre[lane * 8 + m] = run;
            run += loc[m];
        }
        if (lane == 31) gpre[256] = run;
    } else if (warp == 1 && lane < nt) {
        // each target's level-1 bin: the first bin whose inclusive count exceeds its rank
        Target t;
        // u = c_s n as one rounded FP64 product (no fused multiply-add), so that the rank is
        // the floor of the correctly rounded product whatever the compiler contracts
        t.k = (long long)floor(__dmul_rn(cw[lane + 1], (double)n));
        t.total = t.k >= n;
        t.slot = -1;
        t.prefix = 0;
        t.cnt_lt = 0;
        t.cnt_in = 0;
        t.iv_lt = 0;
        if (!t.total) {
            int lo = 0, hi = kL1Bins - 1;   // smallest bb with cincl[bb] > k
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((long long)cincl[mid] > t.k) hi = mid;
                else lo = mid + 1;
            }
            const int bb = lo;
            const long long cnt = (long long)h1.count(bb);
            t.prefix = (unsigned)bb << kL1Shift;
            t.cnt_lt = (long long)cincl[bb] - cnt;
            t.cnt_in = cnt;
            unsigned long long acc = 0;
            const unsigned E = (unsigned)bb / kL1PerGroup;
            for (int m = bb & ~(kL1PerGroup - 1); m < bb; ++m) {
                acc += h1.count(m) * (group_base(E) + ((unsigned long long)(m & (kL1PerGroup - 1)) << kL1Shift)) +
                       h1.low(m);
            }
            t.iv_lt = acc;
        }
        tg[lane] = t;
    }
    __syncthreads();

    // ---- levels 2..4.  The counts of the current target prefixes are known from the last
    // histogram; once they fit the candidate buffer, one pass (from L2) collects those
    // values and every remaining level runs on the buffer.  Until then each level is a
    // histogram pass over the interval (from L2) restricted to the target prefixes, found
    // with O(1) prefix -> slot tables (slot1 at 12 resolved bits, slot2 at 20).
    // the level phase starts: h1 and cincl are dead, their memory now holds the level data
    for (int i = tid; i < kL1Bins; i += kOdfThreads) slot1[i] = -1;
    __syncthreads();
    const int shifts[3] = {12, 6, 0};
    const int widths[3] = {7, 6, 6};
    bool have_cand = false;
    int nc = 0;
    int nd_prev = 0;
    for (int lvl = 0; lvl < 3; ++lvl) {
        const int sh = shifts[lvl], wb = widths[lvl];
        const int hiShift = sh + wb;
        const int nbins = 1 << wb;
        if (warp == 0) {
            // distinct target prefixes -> slots (lane t holds target t)
            const bool act = lane < nt && !tg[lane].total;
            const unsigned p = act ? tg[lane].prefix : 0xffffffffu;
            const unsigned grp = __match_any_sync(kFull, p);
            const int first = __ffs(grp) - 1;
            const bool leader = act && first == lane;
            const unsigned lm = __ballot_sync(kFull, leader);
            const int slot = __popc(lm & ((1u << first) - 1u));
            if (act) tg[lane].slot = slot;
            long long in = 0;
            if (leader) {
                dpre[slot] = p;
                in = tg[lane].cnt_in - (p == 0u ? (long long)s_zero : 0ll);
                if (lvl == 0) atomicOr(&tbits[p >> (kL1Shift + 5)], 1u << ((p >> kL1Shift) & 31u));
            }
            for (int d = 16; d > 0; d >>= 1) in += __shfl_down_sync(kFull, in, d);
            if (lane == 0) {
                n_distinct = __popc(lm);
                n_cand = (!have_cand && in <= kCand) ? 0 : -1;   // 0: collect in this level
            }
        }
        __syncthreads();
        const int nd = n_distinct;
        if (nd == 0) break;
        const bool collect = n_cand == 0;
        // prefix -> slot tables for the current depth
        if (lvl == 0) {
            for (int q = tid; q < nd; q += kOdfThreads) slot1[dpre[q] >> kL1Shift] = (short)q;
        } else if (lvl == 1) {
            for (int i = tid; i < nd_prev * kL2Bins; i += kOdfThreads) slot2[i] = -1;
        }
        __syncthreads();
        if (lvl == 1)
            for (int q = tid; q < nd; q += kOdfThreads) {
                const int q1 = slot1[dpre[q] >> kL1Shift];
                if (q1 >= 0) slot2[q1 * kL2Bins + ((dpre[q] >> 12) & (kL2Bins - 1))] = (short)q;
            }
        for (int i = tid; i < nd * kL2Bins; i += kOdfThreads) h2.zero(i);
        __syncthreads();
        // slot of a value at the current depth, or -1 (zeros are never in a slot)
        auto slot_of = [&](unsigned bits) -> int {
            if (bits == 0u) return -1;
            const int q1 = slot1[bits >> kL1Shift];
            if (q1 < 0 || lvl == 0) return q1;
            if (lvl == 1) return slot2[q1 * kL2Bins + ((bits >> 12) & (kL2Bins - 1))];
            const unsigned pre = (bits >> hiShift) << hiShift;
            int q = -1;
            for (int r = 0; r < nd; ++r)
                if (dpre[r] == pre) q = r;
            return q;
        };
        if (collect) {
            if (lvl == 0) {
                collect_values(x, n, cand, &n_cand, [&](unsigned bits) {
                    return bits != 0u && ((tbits[bits >> (kL1Shift + 5)] >> ((bits >> kL1Shift) & 31u)) & 1u);
                });
            } else {
                collect_values(x, n, cand, &n_cand, [&](unsigned bits) { return slot_of(bits) >= 0; });
            }
            __syncthreads();
            nc = min(n_cand, kCand);
            have_cand = true;
        }
        if (have_cand) {
            for (int i0 = 0; i0 < nc; i0 += kOdfThreads) {
                const int i = i0 + tid;
                const unsigned bits = i < nc ? cand[i] : 0u;
                const int q = i < nc ? slot_of(bits) : -1;
                const unsigned sub = (bits >> sh) & (unsigned)(nbins - 1);
                const unsigned low = sh ? (bits & ((1u << sh) - 1u)) : 0u;
                if (q >= 0) h2.add(q * kL2Bins + (int)sub, 1u, low >> 10, low & 1023u);
            }
        } else {
            RunAdd run;
            for_each_value(x, n, [&](unsigned bits, bool valid) {
                bits &= 0x7fffffffu;
                const int q = valid ? slot_of(bits) : -1;
                if (q < 0) return;
                const unsigned sub = (bits >> sh) & (unsigned)(nbins - 1);
                const unsigned low = sh ? (bits & ((1u << sh) - 1u)) : 0u;
                run.add(h2, q * kL2Bins + (int)sub, low);
            });
            run.flush(h2);
        }
        __syncthreads();
        if (tid < nd && dpre[tid] == 0u) h2.c[tid * kL2Bins] += s_zero;
        __syncthreads();
        for (int t = warp; t < nt; t += kOdfWarps) {
            if (tg[t].total) continue;
            Target tt = tg[t];
            const Hist hs{h2.c + tt.slot * kL2Bins, h2.hi + tt.slot * kL2Bins, h2.lo + tt.slot * kL2Bins};
            resolve_warp(tt, hs, wb, sh, lane);
            if (lane == 0) tg[t] = tt;
        }
        nd_prev = nd;
        __syncthreads();
    }

    if (geom) {
        if (tid == 0) {
            int m = 0;
            for (int t = 0; t < nt; ++t) {
                if (tg[t].total) continue;
                const unsigned p = tg[t].prefix;
                bool dup = false;
                for (int q = 0; q < m; ++q) dup |= thr[q] == p;
                if (dup) continue;
                int i = m++;
                while (i > 0 && thr[i - 1] > p) { thr[i] = thr[i - 1]; --i; }
                thr[i] = p;
            }
            n_thr = m;
        }
        for (int i = tid; i < 5 * (kMaxTargets + 1); i += kOdfThreads) (&gacc[0][0])[i] = 0u;
        __syncthreads();
        const int m = n_thr;
        // bucket of x = number of order statistics <= x; values below thr[j] sit in buckets 0..j.
        // ln x is summed exactly in fixed point (ln_q30 + 2^37 >= 0, in five 32-bit parts per
        // bucket: count and four 10-bit digits of the run sums), with runs merged per lane.
        int rkey = -1;
        unsigned rn = 0;
        unsigned long long rsum = 0;
        auto flush = [&]() {
            if (rkey < 0) return;
            atomicAdd(&gacc[0][rkey], rn);
            atomicAdd(&gacc[1][rkey], (unsigned)(rsum & 1023u));
            atomicAdd(&gacc[2][rkey], (unsigned)((rsum >> 10) & 1023u));
            atomicAdd(&gacc[3][rkey], (unsigned)((rsum >> 20) & 1023u));
            atomicAdd(&gacc[4][rkey], (unsigned)(rsum >> 30));
        };
        for_each_value(x, n, [&](unsigned bits, bool valid) {
            bits &= 0x7fffffffu;
            if (!valid || bits == 0u) return;
            int b = 0;
            for (int q = 0; q < m; ++q) b += bits >= thr[q];
            if (b != rkey) {
                flush();
                rkey = b;
                rn = 0;
                rsum = 0;
            }
            ++rn;
            rsum += (unsigned long long)(ln_q30(bits) + kLnOffset);
        });
        flush();
        __syncthreads();
        if (tid <= m) {
            const unsigned long long tot = (unsigned long long)gacc[1][tid] + ((unsigned long long)gacc[2][tid] << 10) +
                                           ((unsigned long long)gacc[3][tid] << 20) +
                                           ((unsigned long long)gacc[4][tid] << 30);
            const long long lq = (long long)tot - (long long)gacc[0][tid] * kLnOffset;
            lsum[tid] = (double)lq * 0x1p-30;
        }
        __syncthreads();
        if (tid == 0)
            for (int q = 1; q <= m; ++q) lsum[q] += lsum[q - 1];
        __syncthreads();
        if (tid < n_steps) {
            const int s = tid;
            auto G = [&](int bidx, double u) -> double {
                if (bidx == 0) return 0.0;
                if (bidx == n_steps) return lsum[m];
                const Target& t = tg[bidx - 1];
                if (t.total) return lsum[m];
                int j = 0;
                while (j < m - 1 && thr[j] != t.prefix) ++j;
                const double frac = u - (double)t.cnt_lt;
                return lsum[j] + (frac != 0.0 ? frac * ln_f32_bits(t.prefix) : 0.0);
            };
            const double a = __dmul_rn(cw[s], (double)n);
            const double b = __dmul_rn(cw[s + 1], (double)n);
            double r = 0.0;
            if (!(a < (double)s_zero)) r = exp((G(s + 1, b) - G(s, a)) / (w[s] * (double)n));
            out[((size_t)row * K + k) * n_steps + s] = r;
        }
        return;
    }

    // ---- step means
    if (tid < n_steps) {
        const int s = tid;
        auto S = [&](int bidx) -> double {
            if (bidx == 0) return 0.0;
            if (bidx == n_steps) return gpre[256];
            const Target& t = tg[bidx - 1];
            if (t.total) return gpre[256];
            const unsigned E = t.prefix >> 23;
            const double unit = ldexp(1.0, (E >= 1 ? (int)E : 1) - 150);
            const double theta = (double)__uint_as_float(t.prefix);
            const double below = gpre[E] + (double)t.iv_lt * unit;
            const double u = __dmul_rn(cw[bidx], (double)n);   // rounded product: no contraction into u - cnt_lt
            return below + (u - (double)t.cnt_lt) * theta;
        };
        out[((size_t)row * K + k) * n_steps + s] = (S(s + 1) - S(s)) / (w[s] * (double)n);
    }
}

// ---------------------------------------------------------------------------
// k_odf_gather: ODFs of intervals of at most 65,536 points with at most 12 steps (the ODFs of
// the paper: 328 intervals x 12 steps), count then gather; arithmetic or geometric means.
//
// Pass 1 (HBM) counts the values of each 14-bit prefix of the FP32 pattern (bits 30..17: the
// exponent and six mantissa bits, 64 bins per octave) with one shared-memory add per value and
// no other work, so it runs at the rate of the loads.  A scan of the counts gives the bin of
// every boundary rank (a target bin) and the number of values below that bin.  A byte table
// then maps each bin to its gap (the bins between two consecutive target bins, numbered from
// 0) or marks it as a target bin.  Pass 2 (from L2) adds each value of a gap to a lane-private
// FP32 column of that gap in shared memory (columns [bank][warp][gap][lane]: no two lanes share
// an address, so no atomics; two banks give every lane two independent read-add-write chains)
// and sets a bit for each value in a target bin; those few (1-3 % of the values on the table
// workload) go to their target bin's region of a candidate list.  All values of a target bin
// share the exponent, so one warp per target bin finds each order statistic by two radix
// levels over its candidates (bits 16..8, then 7..0) and sums the candidates below it exactly,
// as integers in units of the exponent's ulp.
//
// Sums: a column holds at most 64 values (65,536 points over 512 threads and two banks), a
// relative error below 63 * 2^-24 = 3.8e-6 even if every rounding errs the same way, about
// 1e-7 in practice.  The columns of a gap are added as FP32 pairs (hi, lo) with error-free
// two-sums (FP64 adds run at 1/64 of the FP32 rate on this part), then converted to FP64.  An
// interval whose target bins hold more values than the candidate list, or that is longer than
// 65,536 points, gets kOdfRedo in its first output word and is recomputed by k_odf, which also
// serves more steps.  Geometric means (GEOM) add ln x in the same columns as exact 64-bit
// fixed-point sums (ln_q30, as k_odf) and count the zeros; their step means follow k_odf's.
constexpr int kGThreads = 512;
constexpr int kGWarps = kGThreads / 32;
constexpr int kGShift = 17;                              // bin = bits 30..17
constexpr int kGBins = 1 << (31 - kGShift);              // 16384
constexpr int kGMaxN = 1 << 16;
constexpr int kGMaxSteps = 12;
constexpr int kGGaps = kGMaxSteps;                       // gaps 0..n_slots, n_slots <= 11
constexpr int kGBanks = 2;
constexpr int kGCand = 8192;                             // candidate list (32-bit patterns)
constexpr int kGColWords = kGWarps * kGGaps * 32;        // one bank of columns [warp][gap][lane]
constexpr int kGTableWords = kGBins / 4;                 // one byte per bin
constexpr size_t kGSmem = ((size_t)kGTableWords + kGCand + (size_t)kGBanks * kGColWords) * sizeof(unsigned);  // 96 KB
constexpr int kGU = 4;                                   // float4 loads in flight per thread
static_assert(kGSmem >= (size_t)kGBins * sizeof(unsigned), "the counts must fit the dynamic shared memory");
static_assert((kGMaxSteps - 1) * 512 <= kGBanks * kGColWords, "selection histograms reuse the columns");

__device__ __forceinline__ unsigned gbin(unsigned bits) { return (bits >> kGShift) & (kGBins - 1); }

// (hi, lo) += a, with the rounding error of hi + a kept exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float a) {
    const float s = hi + a;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (a - bp);
    hi = s;
}

template <bool GEOM>
__global__ void __launch_bounds__(kGThreads, 2) k_odf_gather(const float* __restrict__ kappa, int64_t N, int K,
                                                             const int64_t* __restrict__ bounds, int n_steps,
                                                             const double* __restrict__ cw,
                                                             const double* __restrict__ w, double* __restrict__ out) {
    extern __shared__ __align__(16) unsigned sm[];
    __shared__ int s_tbase[kGThreads];    // values below each thread's 32 bins
    __shared__ int s_kt[kGMaxSteps];      // rank of each boundary (>= n: the total)
    __shared__ int s_tbin[kGMaxSteps];    // its bin
    __shared__ int s_blt[kGMaxSteps];     // values below its bin
    __shared__ int s_bcnt[kGMaxSteps];    // values in its bin
    __shared__ int s_tslot[kGMaxSteps];   // its slot (distinct target bin), -1 for the total
    __shared__ int s_sbin[kGMaxSteps], s_slt[kGMaxSteps];   // per slot: bin, values below it
    __shared__ int s_coff[kGMaxSteps + 1], s_ccur[kGMaxSteps];   // per slot: candidate region, cursor
    __shared__ unsigned s_theta[kGMaxSteps];
    __shared__ int s_cb[kGMaxSteps];      // values below the order statistic
    __shared__ double s_sb[kGMaxSteps];   // sum of its slot's values below it
    __shared__ double s_G[kGGaps], s_T[kGMaxSteps], s_P[kGMaxSteps + 1];
    // geometric means: exact sums of ln x in units of 2^-30 (ln_q30), and the zero count
    __shared__ long long s_G64[GEOM ? kGGaps : 1], s_T64[GEOM ? kGMaxSteps : 1], s_sb64[GEOM ? kGMaxSteps : 1];
    __shared__ long long s_P64[GEOM ? kGMaxSteps + 1 : 1];
    __shared__ int s_zero;
    __shared__ int s_wsum[kGWarps];
    __shared__ int s_nslots;

    const int k = blockIdx.x, row = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t b0 = bounds[k];
    const int64_t len = bounds[k + 1] - b0;
    double* o = out + ((size_t)row * K + k) * n_steps;
    if (len > kGMaxN) {   // uniform: left to k_odf
        if (tid == 0) *reinterpret_cast<unsigned long long*>(o) = kOdfRedo;
        return;
    }
    const int n = (int)len, nt = n_steps - 1;
    const float* x = kappa + (size_t)row * N + b0;
    unsigned* cnt = sm;                                                          // pass 1: [kGBins]
    unsigned char* tbl = reinterpret_cast<unsigned char*>(sm);                   // pass 2: [kGBins]
    unsigned* cand = sm + kGTableWords;                                          // [kGCand]
    float* col = reinterpret_cast<float*>(sm + kGTableWords + kGCand);           // [kGBanks][kGColWords]

    // u = c_s n as one rounded FP64 product, as in k_odf and the oracle
    if (tid < nt) s_kt[tid] = (int)floor(__dmul_rn(cw[tid + 1], (double)n));
    if (tid == 0) s_zero = 0;
    for (int i = tid; i < kGBins / 4; i += kGThreads) reinterpret_cast<uint4*>(cnt)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();

    // the 16-byte-aligned body as float4, strided over the CTA (512 contiguous bytes per warp
    // and load); the unaligned head and tail (< 4 values each) go to threads 0..3
    const int mis = (int)(((uintptr_t)x >> 2) & 3u);
    const int head = min(mis ? 4 - mis : 0, n);
    const float4* body = reinterpret_cast<const float4*>(x + head);
    const int nv = (n - head) >> 2;
    const int tail0 = head + 4 * nv;

    // ---- pass 1 (HBM): counts
    for (int i0 = 0; i0 < nv; i0 += kGU * kGThreads) {
        float4 q[kGU];
#pragma unroll
        for (int u = 0; u < kGU; ++u) {
            const int i = i0 + u * kGThreads + tid;
            q[u] = i < nv ? __ldg(body + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kGU; ++u)
            if (i0 + u * kGThreads + tid < nv) {
                atomicAdd(cnt + gbin(__float_as_uint(q[u].x)), 1u);
                atomicAdd(cnt + gbin(__float_as_uint(q[u].y)), 1u);
                atomicAdd(cnt + gbin(__float_as_uint(q[u].z)), 1u);
                atomicAdd(cnt + gbin(__float_as_uint(q[u].w)), 1u);
            }
    }
    if (tid < head) atomicAdd(cnt + gbin(__float_as_uint(__ldg(x + tid))), 1u);
    if (tid < n - tail0) atomicAdd(cnt + gbin(__float_as_uint(__ldg(x + tail0 + tid))), 1u);
    __syncthreads();

    // ---- scan: thread tid owns bins [32 tid, 32 tid + 32) (rotated reads: no bank conflicts)
    {
        int tot = 0;
        const uint4* c4 = reinterpret_cast<const uint4*>(cnt) + tid * 8;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint4 q = c4[(j + lane) & 7];
            tot += (int)(q.x + q.y + q.z + q.w);
        }
        int incl = tot;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        int below = incl - tot;
        for (int v = 0; v < warp; ++v) below += s_wsum[v];
        s_tbase[tid] = below;
    }
    __syncthreads();
    // one warp per boundary rank: the thread range holding it (the last base <= rank), then its
    // bin among that thread's 32 (a warp scan) and the values below the bin
    if (warp < nt) {
        const int t = warp, kt = s_kt[t];
        if (kt < n) {
            int lo = 0, hi = kGThreads - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_tbase[mid] <= kt) lo = mid;
                else hi = mid - 1;
            }
            const int c = (int)cnt[lo * 32 + lane];
            int ci = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(kFull, ci, d);
                if (lane >= d) ci += y;
            }
            const int rel = kt - s_tbase[lo];
            const unsigned m = __ballot_sync(kFull, rel < ci);
            if (lane == (m ? __ffs(m) - 1 : 31)) {
                s_tbin[t] = lo * 32 + lane;
                s_blt[t] = s_tbase[lo] + ci - c;
                s_bcnt[t] = c;
            }
        }
    }
    __syncthreads();
    // distinct target bins -> slots and candidate regions (warp 0, lane t = target t; the bins
    // are non-decreasing in t, so a slot starts where a target's bin differs from the previous one)
    if (warp == 0) {
        const bool act = lane < nt && s_kt[lane] < n;
        const int bin = act ? s_tbin[lane] : -1;
        const int prev = __shfl_up_sync(kFull, bin, 1);
        const bool start = act && (lane == 0 || prev != bin);
        const unsigned starts = __ballot_sync(kFull, start);
        const int slot = act ? __popc(starts & ((2u << lane) - 1u)) - 1 : -1;
        if (lane < nt) s_tslot[lane] = slot;
        const int c = start ? s_bcnt[lane] : 0;
        int ci = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, ci, d);
            if (lane >= d) ci += y;
        }
        if (start) {
            s_sbin[slot] = bin;
            s_slt[slot] = s_blt[lane];
            s_coff[slot] = ci - c;
            s_ccur[slot] = ci - c;
        }
        if (lane == 31) {
            s_coff[__popc(starts)] = ci;
            s_nslots = __popc(starts);
        }
    }
    __syncthreads();
    const int ns = s_nslots;
    if (s_coff[ns] > kGCand) {   // uniform: left to k_odf
        if (tid == 0) *reinterpret_cast<unsigned long long*>(o) = kOdfRedo;
        return;
    }
    // ---- code table over the dead counts: gap index, or 0x80 | slot for a target bin
    {
        const int bA = tid * 32;
        int g = 0;
        for (int j = 0; j < ns; ++j) g += s_sbin[j] < bA;
        uint4 v0, v1;
        if (g < ns && s_sbin[g] < bA + 32) {
            unsigned wd[8];
            int nx = s_sbin[g];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                unsigned code;
                if (bA + j == nx) {
                    code = 0x80u | (unsigned)g;
                    ++g;
                    nx = g < ns ? s_sbin[g] : 0x7fffffff;
                } else {
                    code = (unsigned)g;
                }
                if ((j & 3) == 0) wd[j >> 2] = 0u;
                wd[j >> 2] |= code << (8 * (j & 3));
            }
            v0 = make_uint4(wd[0], wd[1], wd[2], wd[3]);
            v1 = make_uint4(wd[4], wd[5], wd[6], wd[7]);
        } else {
            const unsigned wv = (unsigned)g * 0x01010101u;
            v0 = v1 = make_uint4(wv, wv, wv, wv);
        }
        uint4* t4 = reinterpret_cast<uint4*>(tbl) + tid * 2;
        t4[0] = v0;
        t4[1] = v1;
    }
    for (int i = tid; i < kGBanks * kGColWords / 4; i += kGThreads)
        reinterpret_cast<uint4*>(col)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();

    // ---- pass 2 (L2): gap columns and candidates.  The loads of the next iteration are issued
    // before the current one is processed (the pass waits on L2 latency); all 8 codes of an
    // iteration are read before any column is written, and the two banks take alternate
    // values, so each lane's read-add-write steps form two independent chains.
    {
        float* colA = col + warp * (kGGaps * 32) + lane;
        float* colB = colA + kGColWords;
        long long* colL = reinterpret_cast<long long*>(col) + warp * (kGGaps * 32) + lane;
        int zeros = 0;
        auto to_cand = [&](unsigned bits) {
            const int pos = atomicAdd(&s_ccur[tbl[bits >> kGShift] & 0x7fu], 1);
            cand[pos] = bits;   // inside the slot's region: its size is the bin's count
        };
        constexpr int P2U = 2;
        float4 q[P2U], qn[P2U];
        auto load2 = [&](float4* dst, int j0) {
#pragma unroll
            for (int u = 0; u < P2U; ++u) {
                const int i = j0 + u * kGThreads + tid;
                dst[u] = i < nv ? __ldcs(body + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        load2(q, 0);
#pragma unroll
        for (int u = 0; u < P2U; ++u) qn[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i0 = 0; i0 < nv; i0 += P2U * kGThreads) {
            if (i0 + P2U * kGThreads < nv) load2(qn, i0 + P2U * kGThreads);
            float v[4 * P2U];
            unsigned cd[4 * P2U];
#pragma unroll
            for (int u = 0; u < P2U; ++u) {
                const bool ok = i0 + u * kGThreads + tid < nv;
                const float qq[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const unsigned bits = __float_as_uint(qq[c]) & 0x7fffffffu;
                    v[4 * u + c] = __uint_as_float(bits);
                    cd[4 * u + c] = ok ? tbl[bits >> kGShift] : 0xffu;
                }
            }
            if constexpr (!GEOM) {
#pragma unroll
                for (int e = 0; e < 4 * P2U; e += 2) {
                    const unsigned ca = cd[e], cb = cd[e + 1];
                    float a = 0.f, b = 0.f;
                    if (ca < (unsigned)kGGaps) a = colA[ca * 32];
                    if (cb < (unsigned)kGGaps) b = colB[cb * 32];
                    if (ca < (unsigned)kGGaps) colA[ca * 32] = a + v[e];
                    if (cb < (unsigned)kGGaps) colB[cb * 32] = b + v[e + 1];
                }
            } else {
                // ln x of the positive values in fixed point (exact 64-bit sums); zeros counted
#pragma unroll
                for (int e = 0; e < 4 * P2U; ++e) {
                    const unsigned bits = __float_as_uint(v[e]);
                    if (cd[e] != 0xffu && bits == 0u) ++zeros;
                    if (cd[e] < (unsigned)kGGaps && bits != 0u) colL[cd[e] * 32] += ln_q30(bits);
                }
            }
            unsigned cm = 0u;
#pragma unroll
            for (int e = 0; e < 4 * P2U; ++e)
                if (cd[e] >= 0x80u && cd[e] != 0xffu) cm |= 1u << e;
            while (cm) {   // rare: reload the value (an L1/L2 hit) rather than keep it
                const int e = __ffs(cm) - 1;
                cm &= cm - 1u;
                const int i = i0 + (e >> 2) * kGThreads + tid;
                to_cand(__float_as_uint(__ldg(x + head + 4 * i + (e & 3))) & 0x7fffffffu);
            }
#pragma unroll
            for (int u = 0; u < P2U; ++u) q[u] = qn[u];
        }
        auto one = [&](unsigned bits) {
            bits &= 0x7fffffffu;
            const unsigned code = tbl[bits >> kGShift];
            if (GEOM && bits == 0u) ++zeros;
            if (code < (unsigned)kGGaps) {
                if constexpr (!GEOM) colA[code * 32] += __uint_as_float(bits);
                else if (bits != 0u) colL[code * 32] += ln_q30(bits);
            } else {
                to_cand(bits);
            }
        };
        if (tid < head) one(__float_as_uint(__ldg(x + tid)));
        if (tid < n - tail0) one(__float_as_uint(__ldg(x + tail0 + tid)));
        if (GEOM) {
            zeros = __reduce_add_sync(kFull, zeros);
            if (lane == 0 && zeros) atomicAdd(&s_zero, zeros);
        }
    }
    __syncthreads();

    // ---- gap sums (one warp per gap): FP32 two-sums over the 32 columns of a lane, then over
    // the lanes, then FP64
    if (GEOM && warp <= ns) {
        const long long* cl = reinterpret_cast<const long long*>(col);
        long long sg = 0;
        for (int v = 0; v < kGWarps; ++v) sg += cl[v * (kGGaps * 32) + warp * 32 + lane];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) sg += __shfl_down_sync(kFull, sg, d);
        if (lane == 0) s_G64[warp] = sg;
    }
    if (!GEOM && warp <= ns) {
        float hi = 0.f, lo = 0.f;
#pragma unroll 4
        for (int v = 0; v < kGBanks * kGWarps; ++v) two_sum_add(hi, lo, col[v * (kGGaps * 32) + warp * 32 + lane]);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const float h2 = __shfl_down_sync(kFull, hi, d), l2 = __shfl_down_sync(kFull, lo, d);
            two_sum_add(hi, lo, h2);
            lo += l2;
        }
        if (lane == 0) s_G[warp] = (double)hi + (double)lo;
    }
    __syncthreads();

    // ---- one warp per slot: its total and the order statistics of its targets (the columns
    // are dead: their memory holds one 512-bin histogram per slot)
    if (warp < ns) {
        const int j = warp;
        const unsigned B = (unsigned)s_sbin[j];
        const unsigned E = B >> (23 - kGShift);
        const int eff = E >= 1 ? (int)E : 1;
        const unsigned impl = E >= 1 ? 0x800000u : 0u;
        const int c0 = s_coff[j], c1 = s_coff[j + 1];
        unsigned* h = reinterpret_cast<unsigned*>(col) + j * 512;
        unsigned long long ts = 0;   // mantissa integers: < 2^24 * 2^16
        for (int i = c0 + lane; i < c1; i += 32) ts += (cand[i] & 0x7fffffu) | impl;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) ts += __shfl_down_sync(kFull, ts, d);
        if (lane == 0) s_T[j] = ldexp((double)ts, eff - 150);
        if (GEOM) {
            long long tl = 0;
            for (int i = c0 + lane; i < c1; i += 32) {
                const unsigned c = cand[i];
                if (c) tl += ln_q30(c);
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) tl += __shfl_down_sync(kFull, tl, d);
            if (lane == 0) s_T64[j] = tl;
        }
        for (int t = 0; t < nt; ++t) {
            if (s_tslot[t] != j) continue;   // uniform over the warp
            const int r = s_kt[t] - s_slt[j];   // rank inside the bin (below its count)
            // level A: bits 16..8
            for (int i = lane; i < 512; i += 32) h[i] = 0u;
            __syncwarp();
            for (int i = c0 + lane; i < c1; i += 32) atomicAdd(h + ((cand[i] >> 8) & 511u), 1u);
            __syncwarp();
            int cl = 0;
#pragma unroll
            for (int m = 0; m < 16; ++m) cl += (int)h[lane * 16 + m];
            int ci = cl;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(kFull, ci, d);
                if (lane >= d) ci += y;
            }
            unsigned ow = __ballot_sync(kFull, r >= ci - cl && r < ci);
            int owner = ow ? __ffs(ow) - 1 : 0;
            int a = 0, cA = 0;
            if (lane == owner) {
                int run = ci - cl, m = 0;
                for (; m < 15; ++m) {
                    const int c = (int)h[lane * 16 + m];
                    if (r < run + c) break;
                    run += c;
                }
                a = lane * 16 + m;
                cA = run;
            }
            a = __shfl_sync(kFull, a, owner);
            cA = __shfl_sync(kFull, cA, owner);
            __syncwarp();
            // level B: bits 7..0 of the values in level-A bin a
            for (int i = lane; i < 256; i += 32) h[i] = 0u;
            __syncwarp();
            for (int i = c0 + lane; i < c1; i += 32) {
                const unsigned c = cand[i];
                if (((c >> 8) & 511u) == (unsigned)a) atomicAdd(h + (c & 255u), 1u);
            }
            __syncwarp();
            const int r2 = r - cA;
            cl = 0;
#pragma unroll
            for (int m = 0; m < 8; ++m) cl += (int)h[lane * 8 + m];
            ci = cl;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(kFull, ci, d);
                if (lane >= d) ci += y;
            }
            ow = __ballot_sync(kFull, r2 >= ci - cl && r2 < ci);
            owner = ow ? __ffs(ow) - 1 : 0;
            int bb = 0, cB = 0;
            if (lane == owner) {
                int run = ci - cl, m = 0;
                for (; m < 7; ++m) {
                    const int c = (int)h[lane * 8 + m];
                    if (r2 < run + c) break;
                    run += c;
                }
                bb = lane * 8 + m;
                cB = run;
            }
            bb = __shfl_sync(kFull, bb, owner);
            cB = __shfl_sync(kFull, cB, owner);
            const unsigned theta = (B << kGShift) | ((unsigned)a << 8) | (unsigned)bb;
            unsigned long long sb = 0;
            for (int i = c0 + lane; i < c1; i += 32) {
                const unsigned c = cand[i];
                if (c < theta) sb += (c & 0x7fffffu) | impl;
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) sb += __shfl_down_sync(kFull, sb, d);
            if (GEOM) {
                long long sl = 0;
                for (int i = c0 + lane; i < c1; i += 32) {
                    const unsigned c = cand[i];
                    if (c && c < theta) sl += ln_q30(c);
                }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) sl += __shfl_down_sync(kFull, sl, d);
                if (lane == 0) s_sb64[t] = sl;
            }
            if (lane == 0) {
                s_theta[t] = theta;
                s_cb[t] = s_slt[j] + cA + cB;
                s_sb[t] = ldexp((double)sb, eff - 150);
            }
            __syncwarp();
        }
    }
    __syncthreads();

    if constexpr (GEOM) {
        // ---- geometric step means: G(u) = sum_{0<x<theta} ln x + (u - #{x<theta}) ln theta (the
        // ln sums exact in units of 2^-30, scanned over the slots in 64-bit integers); a sub-bin
        // whose rank range starts among the zeros has geometric mean 0, as in k_odf
        if (warp == 0) {
            const long long gj = lane <= ns ? s_G64[lane] : 0;
            const long long v = gj + (lane < ns ? s_T64[lane] : 0);
            long long inc = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long y = __shfl_up_sync(kFull, inc, d);
                if (lane >= d) inc += y;
            }
            if (lane < ns) s_P64[lane] = inc - v + gj;
            if (lane == ns) s_P64[ns] = inc;
        }
        __syncthreads();
        if (tid < n_steps) {
            auto G = [&](int bidx, double u) -> double {
                if (bidx == 0) return 0.0;
                if (bidx == n_steps || s_kt[bidx - 1] >= n) return (double)s_P64[ns] * 0x1p-30;
                const int t = bidx - 1;
                const double frac = u - (double)s_cb[t];
                return (double)(s_P64[s_tslot[t]] + s_sb64[t]) * 0x1p-30 +
                       (frac != 0.0 ? frac * ln_f32_bits(s_theta[t]) : 0.0);
            };
            const double a = __dmul_rn(cw[tid], (double)n);
            const double b = __dmul_rn(cw[tid + 1], (double)n);
            double r = 0.0;
            if (!(a < (double)s_zero)) r = exp((G(tid + 1, b) - G(tid, a)) / (w[tid] * (double)n));
            o[tid] = r;
        }
        return;
    }
    // ---- step means: S(u) = (sum below theta) + (u - #below) theta at each boundary; s_P[j] is
    // the sum of everything below slot j's bin (an FP64 scan over the slots in warp 0), s_P[ns]
    // the total
    if (warp == 0) {
        const double gj = lane <= ns ? s_G[lane] : 0.0;
        const double v = gj + (lane < ns ? s_T[lane] : 0.0);
        double inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double y = __shfl_up_sync(kFull, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane < ns) s_P[lane] = inc - v + gj;
        if (lane == ns) s_P[ns] = inc;
    }
    __syncthreads();
    if (tid < n_steps) {
        auto S = [&](int bidx) -> double {
            if (bidx == 0) return 0.0;
            if (bidx == n_steps || s_kt[bidx - 1] >= n) return s_P[ns];
            const int t = bidx - 1;
            const double u = __dmul_rn(cw[bidx], (double)n);
            return s_P[s_tslot[t]] + s_sb[t] + (u - (double)s_cb[t]) * (double)__uint_as_float(s_theta[t]);
        };
        o[tid] = (S(tid + 1) - S(tid)) / (w[tid] * (double)n);
    }
}

size_t odf_smem_bytes(int n_steps) {
    const int nt = n_steps - 1;
    const int nslots = nt > kMinSlots ? nt : kMinSlots;
    const size_t setup = 4 * (size_t)kL1Bins * sizeof(unsigned);
    const size_t levels = (kCand + 3 * (size_t)nslots * kL2Bins) * sizeof(unsigned) +
                          (kL1Bins + (size_t)nslots * kL2Bins) * sizeof(short);
    return setup > levels ? setup : levels;
}

}  // namespace

}  // namespace mpsa

using namespace mpsa;

namespace mpsa {

int odf_check(const char* who, int n_rows, int64_t N, int K, const int64_t* bounds, int n_steps,
              const double* widths, int mean_kind, double* cw) {
    if (n_rows < 1 || N < 1 || K < 1) return fail(MPSA_EINVAL, "%s: n_rows %d N %lld K %d", who, n_rows, (long long)N, K);
    // one CTA per (interval, row): the rows are the grid's y dimension
    if (n_rows > kMaxOdfRows) return fail(MPSA_EINVAL, "%s: n_rows = %d (at most %d per call)", who, n_rows, kMaxOdfRows);
    if (n_steps < 1 || n_steps > kMaxSteps) return fail(MPSA_EINVAL, "%s: n_steps = %d (1..%d)", who, n_steps, kMaxSteps);
    if (mean_kind != MPSA_MEAN_ARITH && mean_kind != MPSA_MEAN_GEOM)
        return fail(MPSA_EINVAL, "%s: mean_kind %d (0 arithmetic, 1 geometric)", who, mean_kind);
    if (bounds[0] < 0 || bounds[K] > N) return fail(MPSA_EINVAL, "%s: bounds outside [0, N]", who);
    for (int k = 0; k < K; ++k) {
        const int64_t len = bounds[k + 1] - bounds[k];
        if (len < 1) return fail(MPSA_EINVAL, "%s: bounds not strictly increasing at %d", who, k);
        if (len >= kMaxInterval)
            return fail(MPSA_EINVAL, "%s: interval %d has %lld points (max 2^21-1)", who, k, (long long)len);
    }
    // cumulative widths: FP64 left-to-right partial sums, the last forced to 1
    double acc = 0.0;
    cw[0] = 0.0;
    for (int s = 0; s < n_steps; ++s) {
        if (!(widths[s] > 0) || !isfinite(widths[s])) return fail(MPSA_EINVAL, "%s: widths[%d] = %g", who, s, widths[s]);
        acc = acc + widths[s];
        cw[s + 1] = acc;
    }
    if (fabs(acc - 1.0) > 1e-12) return fail(MPSA_EINVAL, "%s: widths sum to %.17g", who, acc);
    cw[n_steps] = 1.0;
    return MPSA_OK;
}

int odf_setup() {
    int dev = 0;
    MPSA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(MPSA_EINVAL, "build_odf: device %d", dev);
    // once per device (thread-safe): the kernel's dynamic shared-memory limit
    static std::once_flag once[kMaxDevices];
    static cudaError_t err[kMaxDevices];
    std::call_once(once[dev], [&] {
        err[dev] = cudaFuncSetAttribute(k_odf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)odf_smem_bytes(kMaxSteps));
        if (err[dev] == cudaSuccess)
            err[dev] = cudaFuncSetAttribute(k_odf_gather<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem);
        if (err[dev] == cudaSuccess)
            err[dev] = cudaFuncSetAttribute(k_odf_gather<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem);
    });
    if (err[dev] != cudaSuccess)
        return fail(MPSA_ECUDA, "build_odf: cudaFuncSetAttribute: %s", cudaGetErrorString(err[dev]));
    return MPSA_OK;
}

int odf_launch(const float* kappa, int n_rows, int64_t N, int K, const int64_t* d_bounds, int n_steps,
               const double* d_cw, const double* d_w, double* d_out, int mean_kind, cudaStream_t st) {
    int r;
    if ((r = odf_setup())) return r;
    // at most 12 steps: count then gather, and the exact multi-select only for the intervals the
    // gather leaves (too long, or too many candidates); otherwise the multi-select for every
    // interval
    const bool gather = n_steps <= kGMaxSteps;
    if (gather) {
        if (mean_kind == MPSA_MEAN_GEOM)
            k_odf_gather<true><<<dim3(K, n_rows), kGThreads, kGSmem, st>>>(kappa, N, K, d_bounds, n_steps, d_cw, d_w, d_out);
        else
            k_odf_gather<false><<<dim3(K, n_rows), kGThreads, kGSmem, st>>>(kappa, N, K, d_bounds, n_steps, d_cw, d_w, d_out);
        MPSA_CUDA_TRY(cudaGetLastError());
    }
    k_odf<<<dim3(K, n_rows), kOdfThreads, odf_smem_bytes(n_steps), st>>>(kappa, N, K, d_bounds, n_steps, d_cw, d_w,
                                                                         d_out, mean_kind == MPSA_MEAN_GEOM, gather);
    MPSA_CUDA_TRY(cudaGetLastError());
    return MPSA_OK;
}

}  // namespace mpsa

extern "C" int build_odf(mpsa_ctx* ctx, const float* kappa, int32_t n_rows, int64_t N, int32_t K,
                         const int64_t* bounds, int32_t n_steps, const double* widths, int32_t mean_kind,
                         double* odf_out, void* stream) {
    if (!ctx || !kappa || !bounds || !widths || !odf_out) return fail(MPSA_EINVAL, "build_odf: NULL argument");
    std::vector<double> cw(n_steps >= 1 && n_steps <= kMaxSteps ? n_steps + 1 : 1);
    int r;
    if ((r = odf_check("build_odf", n_rows, N, K, bounds, n_steps, widths, mean_kind, cw.data()))) return r;
    MPSA_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st, ctx->pool);
    int64_t* d_b;
    double *d_cw, *d_w;
    if ((r = sc.alloc(&d_b, K + 1)) || (r = sc.alloc(&d_cw, n_steps + 1)) || (r = sc.alloc(&d_w, n_steps))) return r;
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_b, bounds, (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_cw, cw.data(), (n_steps + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_w, widths, n_steps * sizeof(double), cudaMemcpyHostToDevice, st));
    prof_mark(ctx, MPSA_KERNEL_ODF, st);
    r = odf_launch(kappa, n_rows, N, K, d_b, n_steps, d_cw, d_w, odf_out, mean_kind, st);
    prof_mark(ctx, MPSA_KERNEL_ODF, st);
    return r;
}

// ---------------------------------------------------------------------------
// build_odf_noalloc: build_odf without any device allocation.
//
// build_odf stages the interval bounds and the sub-bin widths in stream-ordered
// scratch (the context's pool).  This entry point stages them instead in the fixed
// file-scope array below, for callers that must not allocate device memory: a
// process whose device memory is entirely owned by another framework's caching
// allocator, or a latency-critical loop where an allocation (or a cudaFree that
// may synchronise the device) is not allowed.  The array is resident on every
// device that loads the library, until the process exits.
namespace mpsa {
namespace {

constexpr int kNoAllocMaxIntervals = 65536;
constexpr size_t kNoAllocBytes =
    (size_t)(kNoAllocMaxIntervals + 1) * sizeof(int64_t) + (size_t)(2 * kMaxSteps + 1) * sizeof(double);
static __device__ __align__(256) unsigned char g_odf_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array, looked up once per device (std::call_once, so
// first calls from several host threads are safe).  In host code the symbol name is
// only a host-side stand-in; the address comes from cudaGetSymbolAddress with the
// device current.  The address is kept for the life of the process: it does not
// survive a cudaDeviceReset, after which this entry point must not be called.
static void* g_noalloc_ptr[kMaxDevices];
static cudaError_t g_noalloc_err[kMaxDevices];
static std::once_flag g_noalloc_once[kMaxDevices];

int noalloc_scratch(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return fail(MPSA_EINVAL, "build_odf_noalloc: device %d", device);
    std::call_once(g_noalloc_once[device], [&] {
        void* p = nullptr;
        g_noalloc_err[device] = cudaGetSymbolAddress(&p, g_odf_noalloc_scratch);
        if (g_noalloc_err[device] == cudaSuccess) g_noalloc_ptr[device] = p;
    });
    if (g_noalloc_err[device] != cudaSuccess || !g_noalloc_ptr[device])
        return fail(MPSA_ECUDA, "build_odf_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(g_noalloc_err[device]));
    *out = static_cast<unsigned char*>(g_noalloc_ptr[device]);
    return MPSA_OK;
}

}  // namespace
}  // namespace mpsa

extern "C" int build_odf_noalloc(int32_t device, const float* kappa, int32_t n_rows, int64_t N, int32_t K,
                                 const int64_t* bounds, int32_t n_steps, const double* widths, int32_t mean_kind,
                                 double* odf_out, void* stream) {
    if (!kappa || !bounds || !widths || !odf_out) return fail(MPSA_EINVAL, "build_odf_noalloc: NULL argument");
    // the fixed array's limit first: bounds[K] is read by the shared checks below
    if (K > kNoAllocMaxIntervals)
        return fail(MPSA_EINVAL, "build_odf_noalloc: K = %d intervals exceeds the fixed scratch limit of %d", K,
                    kNoAllocMaxIntervals);
    double cw[kMaxSteps + 1];
    int r;
    if ((r = odf_check("build_odf_noalloc", n_rows, N, K, bounds, n_steps, widths, mean_kind, cw))) return r;
    MPSA_CUDA_TRY(cudaSetDevice(device));
    unsigned char* base;
    if ((r = noalloc_scratch(device, &base))) return r;
    // layout: bounds [K+1] int64 | cumulative widths [n_steps+1] | widths [n_steps]
    int64_t* d_b = reinterpret_cast<int64_t*>(base);
    double* d_cw = reinterpret_cast<double*>(base + (size_t)(kNoAllocMaxIntervals + 1) * sizeof(int64_t));
    double* d_w = d_cw + (kMaxSteps + 1);
    cudaStream_t st = (cudaStream_t)stream;
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_b, bounds, (K + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_cw, cw, (n_steps + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
    MPSA_CUDA_TRY(cudaMemcpyAsync(d_w, widths, n_steps * sizeof(double), cudaMemcpyHostToDevice, st));
    return odf_launch(kappa, n_rows, N, K, d_b, n_steps, d_cw, d_w, odf_out, mean_kind, st);
}

// Shared definitions of the GB300 line-opacity library: physical constants,
// error handling, the context structure and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mpsa.h"

namespace mpsa {

// CODATA 2018, cgs.
constexpr double kC = 2.99792458e10;             // speed of light [cm s^-1]
constexpr double kH = 6.62607015e-27;            // Planck constant [erg s]
constexpr double kKB = 1.380649e-16;             // Boltzmann constant [erg K^-1]
constexpr double kME = 9.1093837015e-28;         // electron mass [g]
constexpr double kE = 4.803204712570263e-10;     // elementary charge [statC]
constexpr double kAMU = 1.66053906660e-24;       // atomic mass unit [g]
constexpr double kEV = 1.602176634e-12;          // electron volt [erg]
constexpr double kPI = 3.14159265358979323846;

// Layout of one population-table row (FP64): T, P, n_e, n_HI, rho, then N/U of
// stages I .. V of every element (0 for stages an element does not have).
constexpr int kMaxStages = 5;
constexpr int kPopT = 0, kPopP = 1, kPopNe = 2, kPopNHI = 3, kPopRho = 4, kPopHdr = 5;
__host__ __device__ inline int pop_stride(int n_el) { return kPopHdr + kMaxStages * n_el; }
__host__ __device__ inline int pop_nu(int e, int stage) { return kPopHdr + kMaxStages * e + stage; }

// Element record of the equation of state (FP64, kElStride values per element): mass [amu],
// log eps (H = 12), number of stages (1..5), ionisation energies chi_0..chi_3 [eV] (stage j ->
// j + 1) and the partition-function coefficients ln U_j(T) = c0 + c1 x + c2 x^2 of stages
// 0..4, x = ln(T / 5040 K).
constexpr int kElMass = 0, kElLogEps = 1, kElStages = 2, kElChi = 3, kElLnU = 7, kElStride = 22;

// Grid points per tile of the profile kernel and threads per tile.
constexpr int kTileThreads = 256;
constexpr int kPtsPerThread = 8;
constexpr int kTile = kTileThreads * kPtsPerThread;   // 2048
constexpr int kNumClasses = 26;                       // window half-width classes 2^0 .. 2^25
constexpr int kMaxGrid = 1 << 24;                     // grid indices exact in FP32

void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);

#define MPSA_CUDA_TRY(expr)                                                          \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return ::mpsa::fail(e_ == cudaErrorMemoryAllocation ? MPSA_ENOMEM : MPSA_ECUDA, \
                                "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// Stream-ordered scratch buffer: allocated on the call's stream from the context's
// memory pool (cudaMallocFromPoolAsync; the device's default pool without a pool) and
// released with cudaFreeAsync on the same stream.
struct Scratch {
    std::vector<void*> ptrs;
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;
    explicit Scratch(cudaStream_t s, cudaMemPool_t p = nullptr) : stream(s), pool(p) {}
    template <class T>
    int alloc(T** p, size_t n) {
        void* q = nullptr;
        cudaError_t e = pool ? cudaMallocFromPoolAsync(&q, n * sizeof(T) + 16, pool, stream)
                             : cudaMallocAsync(&q, n * sizeof(T) + 16, stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(MPSA_ENOMEM, "cudaMallocAsync(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
        }
        ptrs.push_back(q);
        *p = static_cast<T*>(q);
        return MPSA_OK;
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, stream);
    }
};

}  // namespace mpsa

struct mpsa_ctx {
    int device = 0;
    // stream-ordered scratch of every call: a pool of this context that keeps freed memory
    // cached (release threshold: unlimited) until mpsa_destroy, so that repeated calls do
    // not map and unmap their gigabytes of line-preparation scratch each time
    cudaMemPool_t pool = nullptr;
    // element table of the equation of state (device), [n_el][kElStride] records
    int n_el = 0;
    double* d_el = nullptr;
    std::vector<double> h_el;        // host copy, same layout
    // species table
    int n_sp = 0;
    int32_t* d_sp_el = nullptr;
    int32_t* d_sp_stage = nullptr;
    std::vector<int32_t> h_sp_el, h_sp_stage;
    // line list (device, ascending lambda)
    int64_t L = 0;
    double* d_lam = nullptr;
    float* d_loggf = nullptr;
    float* d_E = nullptr;
    float* d_lgR = nullptr;
    float* d_lgS = nullptr;
    float* d_lgW = nullptr;
    int32_t* d_species = nullptr;
    // population table (device FP64) [n_comp * n_points][pop_stride]
    int n_points = 0, n_comp = 0;
    double* d_pop = nullptr;
    double vturb = 0.0;
    std::vector<double> h_abund;     // [n_comp][n_el]
    // kernel timing (mpsa_profile_enable)
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev[4];   // start/stop pairs per kernel
};

namespace mpsa {
// Record a timing event for kernel `which` on `st` when profiling is enabled.
inline void prof_mark(mpsa_ctx* c, int which, cudaStream_t st) {
    if (!c || !c->prof) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, st);
    c->prof_ev[which].push_back(e);
}
}  // namespace mpsa

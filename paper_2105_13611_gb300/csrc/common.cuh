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
// stages I and II of every element.
constexpr int kPopT = 0, kPopP = 1, kPopNe = 2, kPopNHI = 3, kPopRho = 4, kPopHdr = 5;
__host__ __device__ inline int pop_stride(int n_el) { return kPopHdr + 2 * n_el; }

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

// Stream-ordered scratch buffer: allocated with cudaMallocAsync on the call's
// stream and released with cudaFreeAsync on the same stream.
struct Scratch {
    std::vector<void*> ptrs;
    cudaStream_t stream = nullptr;
    explicit Scratch(cudaStream_t s) : stream(s) {}
    template <class T>
    int alloc(T** p, size_t n) {
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, n * sizeof(T) + 16, stream);
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
    // element table (device: 5 arrays of n_el doubles, packed)
    int n_el = 0;
    double* d_el = nullptr;          // [5][n_el]: mass_amu, chi_eV, U1, U2, log_eps
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
    std::vector<cudaEvent_t> prof_ev[3];   // start/stop pairs per kernel
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

// Internal declarations shared by the translation units of libpsweep.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include "psweep.h"

namespace ps {

// Thread-local message behind ps_last_error().
void set_error(const char* fmt, ...);
void clear_error();

inline int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return PS_ERR_CUDA;
}

#define PS_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return ps::cuda_fail(e_, #call); \
    } while (0)

#define PS_ARG(cond, ...)                              \
    do {                                               \
        if (!(cond)) {                                 \
            ps::set_error(__VA_ARGS__);                \
            return PS_ERR_ARG;                         \
        }                                              \
    } while (0)

// Device-side status bits latched by kernels (atomicOr), read by the host.
enum : uint32_t {
    DEV_CAPACITY = 1u,  // hash table or block pool full
    DEV_TIMEOUT = 2u,   // bounded probe loop gave up
};

// Camera in float for device use (level intrinsics already applied).
struct CamF {
    float xi, fx, fy, cx, cy, k1, k2, p1, p2, r2_max;
    float lim;           // -min(xi, 1/xi): sphere-z validity bound
    int width, height;
};

CamF to_camf(const ps_camera& c);

// Ring of pre-created CUDA events recording stage boundaries of successive
// calls (measurement only; see psweep_profile in psweep.h).
struct StageProfiler {
    int stages = 0, cap = 0, n = 0;
    cudaEvent_t* ev = nullptr;  // [cap][stages + 1]
    int enable(int n_stages, int capacity);
    void release();
    // boundary b (0..stages) of the current call; no-op when off or full
    void mark(int b, cudaStream_t s) {
        if (n < cap) cudaEventRecord(ev[n * (stages + 1) + b], s);
    }
    void end_call() {
        if (n < cap) ++n;
    }
    int read(double* ms, int32_t* calls);
};

}  // namespace ps

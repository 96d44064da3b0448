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
    DEV_STATE = 4u,     // a work counter ran past its end (overlapping calls on one handle)
};

// First word of every handle the library hands out, so that
// ps_sync_status can tell the handle types apart.
enum : uint32_t {
    MAGIC_SWEEP = 0x50535750u,  // "PSWP"
    MAGIC_TSDF = 0x50535444u,   // "PSTD"
    MAGIC_BATCH = 0x50534241u,  // "PSBA"
};

// Latched-status readers of each handle type (synchronise the stream, read
// and clear the status word, map its bits to a PS_* code).
int sweep_sync_status(psweep_t* h, cudaStream_t s);
int tsdf_sync_status(tsdf_t* t, cudaStream_t s);
int batch_sync_status(psbatch_t* b, cudaStream_t s);

// Checked build (compiled with -DPS_CHECK): bounds checks at the accesses
// whose address comes from data (image gathers from projected coordinates,
// pool slots from the hash table, queue items) set a bit in a device word of
// the translation unit and skip the access.  In the normal build the checks
// compile to nothing.  ps_check_read() collects and clears the bits.
enum : uint32_t {
    CHK_GATHER = 1u,  // image gather outside the image
    CHK_PIXEL = 2u,   // pixel index outside the image
    CHK_POOL = 4u,    // voxel-block pool slot outside the pool
    CHK_ITEM = 8u,    // work item outside its level or queue
};
#ifdef PS_CHECK
#define PS_CHECKED 1
#else
#define PS_CHECKED 0
#endif
namespace {
__device__ unsigned g_check_bits;  // one per translation unit
}
// True when cond holds; in the checked build a failure records `bit`.
#define PS_DCHECK(cond, bit) \
    (!PS_CHECKED || (cond) || (atomicOr(&ps::g_check_bits, (unsigned)(bit)), false))
// Host reader of this translation unit's check word (reads and clears it).
#define PS_DEFINE_CHECK_READER(fn)                                                \
    unsigned fn() {                                                               \
        unsigned v = 0;                                                           \
        if (!PS_CHECKED) return 0;                                                \
        if (cudaMemcpyFromSymbol(&v, ps::g_check_bits, sizeof(v)) != cudaSuccess) \
            return 0xffffffffu;                                                   \
        const unsigned z = 0;                                                     \
        cudaMemcpyToSymbol(ps::g_check_bits, &z, sizeof(z));                      \
        return v;                                                                 \
    }
unsigned check_bits_sweep();
unsigned check_bits_tsdf();
unsigned check_bits_batch16();
unsigned check_bits_batch24();
unsigned check_bits_diff();

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

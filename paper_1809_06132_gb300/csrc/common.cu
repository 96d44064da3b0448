// Error reporting and version of libpsweep.so.
#include <cstring>

#include "internal.cuh"

namespace ps {

thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

int StageProfiler::enable(int n_stages, int capacity) {
    release();
    if (capacity <= 0) return PS_OK;
    stages = n_stages;
    ev = new cudaEvent_t[(size_t)capacity * (n_stages + 1)];
    for (int i = 0; i < capacity * (n_stages + 1); ++i) {
        cudaError_t e = cudaEventCreate(&ev[i]);
        if (e != cudaSuccess) {
            for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
            delete[] ev;
            ev = nullptr;
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    cap = capacity;
    n = 0;
    return PS_OK;
}

void StageProfiler::release() {
    if (ev) {
        for (int i = 0; i < cap * (stages + 1); ++i) cudaEventDestroy(ev[i]);
        delete[] ev;
    }
    ev = nullptr;
    cap = n = 0;
}

int StageProfiler::read(double* ms, int32_t* calls) {
    for (int s = 0; s < stages; ++s) ms[s] = 0.0;
    for (int c = 0; c < n; ++c) {
        for (int s = 0; s < stages; ++s) {
            cudaEvent_t a = ev[c * (stages + 1) + s], b = ev[c * (stages + 1) + s + 1];
            cudaError_t e = cudaEventSynchronize(b);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
            float t = 0.f;
            e = cudaEventElapsedTime(&t, a, b);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
            ms[s] += t;
        }
    }
    if (calls) *calls = n;
    n = 0;
    return PS_OK;
}

}  // namespace ps

extern "C" const char* ps_last_error(void) { return ps::g_err; }

extern "C" const char* ps_version(void) {
    return PS_CHECKED ? "psweep-gb300 0.1 (sm_103a, checked)" : "psweep-gb300 0.1 (sm_103a)";
}

extern "C" int ps_sync_status(void* handle, void* stream) {
    ps::clear_error();
    PS_ARG(handle != nullptr, "ps_sync_status: handle is NULL");
    uint32_t magic = 0;
    std::memcpy(&magic, handle, sizeof(magic));
    cudaStream_t s = (cudaStream_t)stream;
    switch (magic) {
        case ps::MAGIC_SWEEP: return ps::sweep_sync_status(static_cast<psweep_t*>(handle), s);
        case ps::MAGIC_TSDF: return ps::tsdf_sync_status(static_cast<tsdf_t*>(handle), s);
        case ps::MAGIC_BATCH: return ps::batch_sync_status(static_cast<psbatch_t*>(handle), s);
        default: break;
    }
    ps::set_error("ps_sync_status: not a handle of this library");
    return PS_ERR_ARG;
}

extern "C" int ps_check_read(uint32_t* bits) {
    ps::clear_error();
    PS_ARG(bits != nullptr, "ps_check_read: bits is NULL");
    PS_CUDA(cudaDeviceSynchronize());
    *bits = ps::check_bits_sweep() | ps::check_bits_tsdf() | ps::check_bits_batch16() | ps::check_bits_batch24() |
            ps::check_bits_diff();
    return PS_OK;
}

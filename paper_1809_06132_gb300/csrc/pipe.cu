// Frame pipeline: host frames through three CUDA streams (copy in; sweep
// and fusion; copy out) with two frames in flight, so that the host<->device
// copies and the host-side staging of frames n + 1 and n - 1 overlap the
// GPU work of frame n.  The paper runs depth estimation and fusion on
// separate computers at the same time (Sec. IV-A); on one GPU the sweep
// fills every SM, so fusion follows each sweep on the compute stream and the
// overlap that remains is the copies'.
#include <cstring>

#include "sweep_dev.cuh"

struct ps_pipe_s {
    psweep_t* h = nullptr;
    tsdf_t* t = nullptr;
    cudaStream_t s_in = nullptr, s_sweep = nullptr, s_out = nullptr;
    int n_img = 0;
    size_t img_bytes[1 + PS_MAX_CAMS] = {};
    size_t depth_bytes = 0;
    uint8_t* dev_img[2][1 + PS_MAX_CAMS] = {};
    uint8_t* host_img[2][1 + PS_MAX_CAMS] = {};  // pinned staging
    float* dev_depth[2] = {};
    float* host_depth[2] = {};                    // pinned staging
    float* user_out[2] = {};
    bool pending[2] = {};
    cudaEvent_t ev_in[2] = {}, ev_depth[2] = {}, ev_done[2] = {};
    long long n_pushed = 0;
};

namespace {

void free_pipe(ps_pipe_t* p) {
    if (!p) return;
    if (p->s_in) cudaStreamSynchronize(p->s_in);
    if (p->s_sweep) cudaStreamSynchronize(p->s_sweep);
    if (p->s_out) cudaStreamSynchronize(p->s_out);
    for (int k = 0; k < 2; ++k) {
        for (int i = 0; i < p->n_img; ++i) {
            cudaFree(p->dev_img[k][i]);
            cudaFreeHost(p->host_img[k][i]);
        }
        cudaFree(p->dev_depth[k]);
        cudaFreeHost(p->host_depth[k]);
        if (p->ev_in[k]) cudaEventDestroy(p->ev_in[k]);
        if (p->ev_depth[k]) cudaEventDestroy(p->ev_depth[k]);
        if (p->ev_done[k]) cudaEventDestroy(p->ev_done[k]);
    }
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_sweep) cudaStreamDestroy(p->s_sweep);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    delete p;
}

// Wait for the frame in `slot` and hand its depth map to the caller's buffer.
int retire(ps_pipe_t* p, int slot) {
    if (!p->pending[slot]) return PS_OK;
    PS_CUDA(cudaEventSynchronize(p->ev_done[slot]));
    if (p->user_out[slot]) std::memcpy(p->user_out[slot], p->host_depth[slot], p->depth_bytes);
    p->pending[slot] = false;
    return PS_OK;
}

}  // namespace

extern "C" int ps_pipe_create(psweep_t* h, tsdf_t* t, ps_pipe_t** out) {
    ps::clear_error();
    PS_ARG(out != nullptr, "ps_pipe_create: out is NULL");
    *out = nullptr;
    PS_ARG(h != nullptr, "ps_pipe_create: sweep handle is NULL");
    ps_pipe_t* p = new ps_pipe_t();
    p->h = h;
    p->t = t;
    p->n_img = 1 + h->n_cams;
    for (int i = 0; i < p->n_img; ++i) {
        const ps_camera& c = i == 0 ? h->ref : h->cams[i - 1];
        p->img_bytes[i] = (size_t)c.width * c.height;
    }
    p->depth_bytes = sizeof(float) * (size_t)h->ref.width * h->ref.height;
#define PP_TRY(call)                                                           \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            free_pipe(p);                                                      \
            ps::set_error("%s: %s", #call, cudaGetErrorString(e_));            \
            return e_ == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA; \
        }                                                                      \
    } while (0)
    PP_TRY(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking));
    PP_TRY(cudaStreamCreateWithFlags(&p->s_sweep, cudaStreamNonBlocking));
    PP_TRY(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        for (int i = 0; i < p->n_img; ++i) {
            PP_TRY(cudaMalloc(&p->dev_img[k][i], p->img_bytes[i]));
            PP_TRY(cudaMallocHost(&p->host_img[k][i], p->img_bytes[i]));
        }
        PP_TRY(cudaMalloc(&p->dev_depth[k], p->depth_bytes));
        PP_TRY(cudaMallocHost(&p->host_depth[k], p->depth_bytes));
        PP_TRY(cudaEventCreateWithFlags(&p->ev_in[k], cudaEventDisableTiming));
        PP_TRY(cudaEventCreateWithFlags(&p->ev_depth[k], cudaEventDisableTiming));
        PP_TRY(cudaEventCreateWithFlags(&p->ev_done[k], cudaEventDisableTiming));
    }
#undef PP_TRY
    *out = p;
    return PS_OK;
}

extern "C" int ps_pipe_push(ps_pipe_t* p, const uint8_t* const* host_images, const ps_box* boxes, int32_t n_boxes,
                            const ps_pose* world_to_ref, const double* local_center, float* host_depth_out) {
    ps::clear_error();
    PS_ARG(p != nullptr && host_images != nullptr, "ps_pipe_push: pipeline or images NULL");
    PS_ARG(p->t == nullptr || world_to_ref != nullptr, "ps_pipe_push: world_to_ref is NULL");
    for (int i = 0; i < p->n_img; ++i) PS_ARG(host_images[i] != nullptr, "ps_pipe_push: host_images[%d] is NULL", i);
    const int slot = (int)(p->n_pushed & 1);
    // the slot's previous frame (two pushes ago) must be finished before its buffers are reused
    int st = retire(p, slot);
    if (st) return st;
    // copy in
    const uint8_t* dev[1 + PS_MAX_CAMS];
    for (int i = 0; i < p->n_img; ++i) {
        std::memcpy(p->host_img[slot][i], host_images[i], p->img_bytes[i]);
        PS_CUDA(cudaMemcpyAsync(p->dev_img[slot][i], p->host_img[slot][i], p->img_bytes[i], cudaMemcpyHostToDevice,
                                p->s_in));
        dev[i] = p->dev_img[slot][i];
    }
    PS_CUDA(cudaEventRecord(p->ev_in[slot], p->s_in));
    // sweep, then fusion, in frame order on the compute stream (the handles'
    // buffers are reused and the volume is updated in order).  Fusion is
    // short and runs right behind its sweep: on a stream of its own it could
    // be held behind the next frame's persistent sweep launch, delaying the
    // slot's release and so the next frame's input copy.
    PS_CUDA(cudaStreamWaitEvent(p->s_sweep, p->ev_in[slot], 0));
    st = psweep_depth(p->h, dev, boxes, n_boxes, p->dev_depth[slot], nullptr, p->s_sweep);
    if (st) return st;
    if (p->t) {
        st = tsdf_integrate(p->t, p->dev_depth[slot], world_to_ref, local_center, p->s_sweep);
        if (st) return st;
    }
    PS_CUDA(cudaEventRecord(p->ev_depth[slot], p->s_sweep));
    // copy out on the output stream
    PS_CUDA(cudaStreamWaitEvent(p->s_out, p->ev_depth[slot], 0));
    if (host_depth_out)
        PS_CUDA(cudaMemcpyAsync(p->host_depth[slot], p->dev_depth[slot], p->depth_bytes, cudaMemcpyDeviceToHost,
                                p->s_out));
    PS_CUDA(cudaEventRecord(p->ev_done[slot], p->s_out));
    p->user_out[slot] = host_depth_out;
    p->pending[slot] = true;
    ++p->n_pushed;
    return PS_OK;
}

extern "C" int ps_pipe_flush(ps_pipe_t* p) {
    ps::clear_error();
    PS_ARG(p != nullptr, "ps_pipe_flush: pipeline is NULL");
    // oldest first
    const int first = (int)(p->n_pushed & 1);
    int st = retire(p, first);
    if (st) return st;
    return retire(p, first ^ 1);
}

extern "C" void ps_pipe_destroy(ps_pipe_t* p) { free_pipe(p); }

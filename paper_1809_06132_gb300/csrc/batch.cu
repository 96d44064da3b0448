// Batched plane sweeps (host side): queue construction, device tables,
// per-run staging, CUDA graph replay, completion timing and the autotuner.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <set>
#include <vector>

#include "batch_dev.cuh"

namespace ps {
const void* batch_kernel_th16(int kp);
const void* batch_kernel_th24(int kp);
}  // namespace ps

using namespace ps;

struct psbatch_s {
    uint32_t magic = MAGIC_BATCH;  // first word: handle type for ps_sync_status
    int n = 0;
    std::vector<psweep_t*> sw;
    ps_batch_opts opts{};
    const void* kernel = nullptr;
    int grid = 0;
    size_t smem = 0;
    std::vector<int> n_images;  // 1 + n_cams per sweep
    std::vector<int> q_counts;  // items per kind
    // device tables (static)
    JobD* jobs = nullptr;
    LevelD* levels = nullptr;
    int4* queue = nullptr;
    int n_queue = 0;
    float* partial = nullptr;
    // zeroed per run: head, abort, status, pad, then counters and tile counts
    int* zero = nullptr;
    size_t zero_bytes = 0;
    unsigned long long* times = nullptr;  // [1 + n]
    // per-run staging: JobIO[n] then up to 256 boxes per sweep
    void* stage_host[2] = {};
    void* stage_dev = nullptr;
    size_t stage_bytes = 0;
    cudaEvent_t stage_free[2] = {};
    int slot = 0;
    bool ran = false;
    cudaGraphExec_t exec[2] = {};
};

namespace {

constexpr int MAX_BOXES = 256;

void free_batch(psbatch_t* b) {
    if (!b) return;
    cudaFree(b->jobs);
    cudaFree(b->levels);
    cudaFree(b->queue);
    cudaFree(b->partial);
    cudaFree(b->zero);
    cudaFree(b->times);
    cudaFree(b->stage_dev);
    for (int i = 0; i < 2; ++i) {
        cudaFreeHost(b->stage_host[i]);
        if (b->stage_free[i]) cudaEventDestroy(b->stage_free[i]);
        if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
    }
    delete b;
}

// Relative cost of one sweep item of a level (plane-camera halo samples).
double item_cost(const LevelD& D, int th) {
    return (double)D.chunk * D.n_cams * (TW + 2 * D.rho) * (th + 2 * D.rho);
}

int launch(psbatch_t* b, cudaStream_t s) {
    PS_CUDA(cudaMemcpyAsync(b->stage_dev, b->stage_host[b->slot], b->stage_bytes, cudaMemcpyHostToDevice, s));
    PS_CUDA(cudaMemsetAsync(b->zero, 0, b->zero_bytes, s));
    PS_CUDA(cudaMemsetAsync(b->times, 0xff, sizeof(unsigned long long) * (1 + b->n), s));
    BatchArgs A;
    A.jobs = b->jobs;
    A.levels = b->levels;
    A.io = static_cast<const JobIO*>(b->stage_dev);
    A.boxes = reinterpret_cast<const ps_box*>(static_cast<const char*>(b->stage_dev) + sizeof(JobIO) * b->n);
    A.queue = b->queue;
    A.n_queue = b->n_queue;
    A.head = b->zero;
    A.abort = b->zero + 1;
    A.status = reinterpret_cast<unsigned*>(b->zero + 2);
    A.ctr = b->zero + 4;
    A.t = b->times;
    A.limit_ns = (unsigned long long)b->opts.wait_limit_ms * 1000000ull;
    void* args[] = {&A};
    PS_CUDA(cudaLaunchKernel(b->kernel, dim3(b->grid), dim3(NT), args, b->smem, s));
    return PS_OK;
}

}  // namespace

extern "C" int psbatch_create(psweep_t* const* sweeps, int32_t n, const ps_batch_opts* opts, psbatch_t** out) {
    clear_error();
    PS_ARG(out != nullptr, "psbatch_create: out is NULL");
    *out = nullptr;
    PS_ARG(sweeps != nullptr && n >= 1 && n <= 4096, "psbatch_create: need 1..4096 sweep handles");
    ps_batch_opts o{};
    if (opts) o = *opts;
    if (o.tile_h == 0) o.tile_h = 24;
    if (o.kp == 0) o.kp = 2;
    if (o.plane_chunk == 0) o.plane_chunk = PLANE_CHUNK;
    if (o.wait_limit_ms == 0) o.wait_limit_ms = 2000;
    PS_ARG(o.tile_h == 16 || o.tile_h == 24, "psbatch_create: tile_h must be 16 or 24");
    PS_ARG(o.kp == 1 || o.kp == 2, "psbatch_create: kp must be 1 or 2");
    PS_ARG(o.plane_chunk >= 1 && o.plane_chunk <= 4096, "psbatch_create: plane_chunk must be in 1..4096");
    PS_ARG(o.order == PS_BATCH_SHORTEST_FIRST || o.order == PS_BATCH_GIVEN_ORDER, "psbatch_create: bad order");
    PS_ARG(o.grid >= 0, "psbatch_create: grid must be >= 0");
    PS_ARG(o.wait_limit_ms >= 1 && o.wait_limit_ms <= 60000, "psbatch_create: wait_limit_ms must be in 1..60000");
    {
        std::set<const psweep_t*> seen;
        for (int i = 0; i < n; ++i) {
            PS_ARG(sweeps[i] != nullptr, "psbatch_create: sweeps[%d] is NULL", i);
            PS_ARG(seen.insert(sweeps[i]).second, "psbatch_create: sweeps[%d] appears twice", i);
        }
    }
    const int th = o.tile_h;
    psbatch_t* b = new psbatch_t();
    b->n = n;
    b->sw.assign(sweeps, sweeps + n);
    b->opts = o;
    b->kernel = th == 16 ? batch_kernel_th16(o.kp) : batch_kernel_th24(o.kp);
#define PB_TRY(call)                                                           \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            free_batch(b);                                                     \
            set_error("%s: %s", #call, cudaGetErrorString(e_));                \
            return e_ == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA; \
        }                                                                      \
    } while (0)

    // levels, jobs, scratch layout
    std::vector<LevelD> lv((size_t)n * PS_MAX_LEVELS);
    std::vector<JobD> jobs(n);
    std::vector<double> cost(n, 0.0);
    size_t partial_floats = 0;
    std::vector<size_t> partial_off((size_t)n * PS_MAX_LEVELS, 0);
    int tile_ints = 0;
    std::vector<int> tile_off((size_t)n * PS_MAX_LEVELS, 0);
    for (int i = 0; i < n; ++i) {
        const psweep_t* h = sweeps[i];
        b->n_images.push_back(1 + h->n_cams);
        JobD& J = jobs[i];
        std::memset(&J, 0, sizeof(J));
        J.n_cams = h->n_cams;
        J.n_levels = h->n_levels;
        J.image_half = h->image_half;
        J.ref_w = h->ref.width;
        for (int j = 0; j < h->n_cams; ++j) J.cam_w[j] = h->cams[j].width;
        for (int l = 0; l < h->n_levels; ++l) {
            LevelD& D = lv[(size_t)i * PS_MAX_LEVELS + l];
            fill_level(h, l, th, balanced_chunk(h->n_planes[l], o.plane_chunk), D);
            if (D.n_chunks > 1) {
                partial_off[(size_t)i * PS_MAX_LEVELS + l] = partial_floats;
                partial_floats += (size_t)7 * th * TW * D.n_items;
            }
            tile_off[(size_t)i * PS_MAX_LEVELS + l] = tile_ints;
            tile_ints += D.n_tiles;
            J.tiles_total += D.n_tiles;
            cost[i] += item_cost(D, th) * D.n_items;
            const ps_level& L = h->levels[l];
            PrepD& P = J.prep[l];
            P.s = L.kind == PS_LEVEL_DOWNSAMPLE ? L.factor : 0;
            P.x0 = h->cx0[l];
            P.y0 = h->cy0[l];
            P.Wl = h->lW[l];
            P.Hl = h->lH[l];
            P.rho = L.window / 2;
            P.ref = h->ref_img[l];
            P.stats = h->stats[l];
            P.n_ref_items = (P.Hl + PREP_ROWS - 1) / PREP_ROWS;
            P.cam_s = L.kind == PS_LEVEL_DOWNSAMPLE ? L.factor : 1;
            int quad_items = 0;
            for (int j = 0; j < h->n_cams; ++j) {
                P.cam_Wl[j] = h->lcam[l][j].width;
                P.cam_Hl[j] = h->lcam[l][j].height;
                P.quad[j] = h->quad[l][j];
                quad_items += (P.cam_Hl[j] + PREP_ROWS - 1) / PREP_ROWS;
            }
            P.prep_target = quad_items + P.n_ref_items;  // statistics items cover the same rows as Q_REF
        }
        fill_merge(h, &lv[(size_t)i * PS_MAX_LEVELS], J.M);
        J.filter = h->filter.enable ? 1 : 0;
        J.cont_half = h->filter.window / 2;
        J.gamma = (float)h->filter.gamma;
        J.delta = (float)h->filter.delta;
        J.merged = h->merged;
        J.merge_items = (h->ref.height + MERGE_ROWS - 1) / MERGE_ROWS;
        if (o.drill_unmet_wait) J.tiles_total += 1;  // no run ever finishes this many tiles
    }
    if (partial_floats) PB_TRY(cudaMalloc(&b->partial, sizeof(float) * partial_floats));
    const size_t ctr_ints = 4 + (size_t)n * C_N;
    b->zero_bytes = sizeof(int) * (ctr_ints + tile_ints);
    PB_TRY(cudaMalloc(&b->zero, b->zero_bytes));
    for (int i = 0; i < n; ++i)
        for (int l = 0; l < sweeps[i]->n_levels; ++l) {
            LevelD& D = lv[(size_t)i * PS_MAX_LEVELS + l];
            if (D.n_chunks > 1) D.partial = b->partial + partial_off[(size_t)i * PS_MAX_LEVELS + l];
            D.done = b->zero + ctr_ints + tile_off[(size_t)i * PS_MAX_LEVELS + l];
            D.tiles_done = b->zero + 4 + i * C_N + C_TILES;
            D.status = reinterpret_cast<unsigned*>(b->zero + 2);
        }

    // launch shape
    {
        size_t smem = 0;
        for (int i = 0; i < n; ++i)
            for (int l = 0; l < sweeps[i]->n_levels; ++l) {
                const int r = lv[(size_t)i * PS_MAX_LEVELS + l].rho, nc = sweeps[i]->n_cams;
                smem = std::max(smem, th == 16 ? (o.kp == 1 ? sweep_smem<16, 1>(r, nc) : sweep_smem<16, 2>(r, nc))
                                               : (o.kp == 1 ? sweep_smem<24, 1>(r, nc) : sweep_smem<24, 2>(r, nc)));
            }
        b->smem = smem;
        int dev = 0, sms = 0, optin = 0, per_sm = 0;
        cudaFuncAttributes fa;
        PB_TRY(cudaGetDevice(&dev));
        PB_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        PB_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        PB_TRY(cudaFuncGetAttributes(&fa, b->kernel));
        if (smem + fa.sharedSizeBytes > (size_t)optin) {
            free_batch(b);
            PS_ARG(false, "psbatch_create: a work item needs %zu bytes of shared memory (device: %d)",
                   smem + fa.sharedSizeBytes, optin);
        }
        PB_TRY(cudaFuncSetAttribute(b->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        PB_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b->kernel, NT, smem));
        if (per_sm < 1) {
            free_batch(b);
            PS_ARG(false, "psbatch_create: the batch kernel does not fit one SM");
        }
        const int fit = sms;  // one CTA per SM: each CTA allocates all of its SM's tensor memory
        b->grid = o.grid > 0 ? std::min(o.grid, fit) : fit;
    }

    // queue: level images of every sweep, then statistics, then per sweep its
    // sweep items followed (after a delay of one grid of items) by its merge
    // and continuity rows
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    if (o.order == PS_BATCH_SHORTEST_FIRST)
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] < cost[c]; });
    std::vector<int4> q;
    b->q_counts.assign(6, 0);
    auto push = [&](int4 e) {
        q.push_back(e);
        ++b->q_counts[e.x & 15];
    };
    for (int i : order)
        for (int l = 0; l < sweeps[i]->n_levels; ++l)
            for (int r = 0; r < jobs[i].prep[l].n_ref_items; ++r) push(qitem(Q_REF, i, l, 0, r));
    for (int i : order)
        for (int l = 0; l < sweeps[i]->n_levels; ++l)
            for (int j = 0; j < sweeps[i]->n_cams; ++j)
                for (int r = 0; r * PREP_ROWS < jobs[i].prep[l].cam_Hl[j]; ++r) push(qitem(Q_QUAD, i, l, j, r));
    for (int i : order)
        for (int l = 0; l < sweeps[i]->n_levels; ++l)
            for (int r = 0; r < jobs[i].prep[l].n_ref_items; ++r) push(qitem(Q_STATS, i, l, 0, r));
    struct Pending {
        size_t at;
        int job, kind;
    };
    std::vector<Pending> pend;
    auto flush = [&](bool all) {
        for (;;) {
            auto it = std::min_element(pend.begin(), pend.end(),
                                       [](const Pending& a, const Pending& c) { return a.at < c.at; });
            if (it == pend.end() || (!all && it->at > q.size())) return;
            const Pending p = *it;
            pend.erase(it);
            for (int r = 0; r < jobs[p.job].merge_items; ++r) push(qitem(p.kind, p.job, 0, 0, r));
            if (p.kind == Q_MERGE && jobs[p.job].filter) pend.push_back({q.size() + (size_t)b->grid, p.job, Q_CONT});
        }
    };
    for (int i : order) {
        const psweep_t* h = sweeps[i];
        int lo[PS_MAX_LEVELS] = {0, 1};
        if (h->n_levels == 2 && item_cost(lv[(size_t)i * PS_MAX_LEVELS + 1], th) >
                                    item_cost(lv[(size_t)i * PS_MAX_LEVELS + 0], th))
            std::swap(lo[0], lo[1]);
        for (int k = 0; k < h->n_levels; ++k) {
            const int l = lo[k];
            for (int it = 0; it < lv[(size_t)i * PS_MAX_LEVELS + l].n_items; ++it) {
                push(qitem(Q_SWEEP, i, l, 0, it));
                flush(false);
            }
        }
        pend.push_back({q.size() + (size_t)b->grid, i, Q_MERGE});
    }
    flush(true);
    b->n_queue = (int)q.size();

    PB_TRY(cudaMalloc(&b->jobs, sizeof(JobD) * n));
    PB_TRY(cudaMemcpy(b->jobs, jobs.data(), sizeof(JobD) * n, cudaMemcpyHostToDevice));
    PB_TRY(cudaMalloc(&b->levels, sizeof(LevelD) * lv.size()));
    PB_TRY(cudaMemcpy(b->levels, lv.data(), sizeof(LevelD) * lv.size(), cudaMemcpyHostToDevice));
    PB_TRY(cudaMalloc(&b->queue, sizeof(int4) * q.size()));
    PB_TRY(cudaMemcpy(b->queue, q.data(), sizeof(int4) * q.size(), cudaMemcpyHostToDevice));
    PB_TRY(cudaMalloc(&b->times, sizeof(unsigned long long) * (1 + n)));
    b->stage_bytes = sizeof(JobIO) * n + sizeof(ps_box) * (size_t)MAX_BOXES * n;
    PB_TRY(cudaMalloc(&b->stage_dev, b->stage_bytes));
    for (int i = 0; i < 2; ++i) {
        PB_TRY(cudaMallocHost(&b->stage_host[i], b->stage_bytes));
        std::memset(b->stage_host[i], 0, b->stage_bytes);
        PB_TRY(cudaEventCreateWithFlags(&b->stage_free[i], cudaEventDisableTiming));
    }
    PB_TRY(cudaDeviceSynchronize());
#undef PB_TRY
    *out = b;
    return PS_OK;
}

extern "C" void psbatch_destroy(psbatch_t* b) { free_batch(b); }

extern "C" int psbatch_run(psbatch_t* b, const uint8_t* const* images, const ps_box* boxes, const int32_t* n_boxes,
                           float* const* depth_out, void* stream) {
    clear_error();
    PS_ARG(b != nullptr && images != nullptr && depth_out != nullptr, "psbatch_run: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    PS_ARG(!b->opts.use_graph || s != nullptr, "psbatch_run: graph replay needs a non-NULL stream");
    const int slot = b->slot;
    // the staging slot is free once the run that last read it has finished
    PS_CUDA(cudaEventSynchronize(b->stage_free[slot]));
    JobIO* io = static_cast<JobIO*>(b->stage_host[slot]);
    ps_box* bx = reinterpret_cast<ps_box*>(io + b->n);
    int img = 0, box_in = 0, box_out = 0;
    for (int i = 0; i < b->n; ++i) {
        std::memset(&io[i], 0, sizeof(JobIO));
        for (int k = 0; k < b->n_images[i]; ++k) {
            PS_ARG(images[img] != nullptr, "psbatch_run: image %d of sweep %d is NULL", k, i);
            io[i].img[k] = images[img++];
        }
        PS_ARG(depth_out[i] != nullptr, "psbatch_run: depth_out[%d] is NULL", i);
        io[i].depth = depth_out[i];
        const int nb = n_boxes ? n_boxes[i] : 0;
        PS_ARG(nb >= 0 && nb <= MAX_BOXES, "psbatch_run: n_boxes[%d] must be in 0..%d", i, MAX_BOXES);
        PS_ARG(nb == 0 || boxes != nullptr, "psbatch_run: boxes is NULL");
        io[i].n_boxes = nb;
        io[i].box0 = box_out;
        for (int k = 0; k < nb; ++k) bx[box_out++] = boxes[box_in++];
    }
    if (b->opts.use_graph) {
        if (!b->exec[slot]) {
            cudaGraph_t g = nullptr;
            PS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            int st = launch(b, s);
            cudaError_t e = cudaStreamEndCapture(s, &g);
            if (st) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return cuda_fail(e, "psbatch_run: stream capture");
            e = cudaGraphInstantiate(&b->exec[slot], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "psbatch_run: graph instantiation");
        }
        PS_CUDA(cudaGraphLaunch(b->exec[slot], s));
    } else {
        int st = launch(b, s);
        if (st) return st;
    }
    PS_CUDA(cudaEventRecord(b->stage_free[slot], s));
    b->slot ^= 1;
    b->ran = true;
    return PS_OK;
}

extern "C" int psbatch_status(psbatch_t* b) {
    clear_error();
    PS_ARG(b != nullptr, "psbatch_status: handle is NULL");
    if (!b->ran) return PS_OK;
    PS_CUDA(cudaEventSynchronize(b->stage_free[b->slot ^ 1]));
    unsigned st = 0;
    PS_CUDA(cudaMemcpy(&st, b->zero + 2, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st & DEV_TIMEOUT) {
        set_error("psbatch: a work item's wait gave up; the rest of the batch was skipped");
        return PS_ERR_TIMEOUT;
    }
    if (st & DEV_STATE) {
        set_error("psbatch: a tile's plane chunks were counted more often than it has chunks");
        return PS_ERR_STATE;
    }
    return PS_OK;
}

namespace ps {
// The batch's status word is cleared by every run, so it holds the last
// run's outcome.
int batch_sync_status(psbatch_t* b, cudaStream_t s) {
    PS_CUDA(cudaStreamSynchronize(s));
    return psbatch_status(b);
}
}  // namespace ps

extern "C" int psbatch_timing(psbatch_t* b, double* done_ms, double* span_ms) {
    clear_error();
    PS_ARG(b != nullptr, "psbatch_timing: handle is NULL");
    PS_ARG(b->ran, "psbatch_timing: the batch has not run");
    int st = psbatch_status(b);
    if (st) return st;
    std::vector<unsigned long long> t(1 + b->n);
    PS_CUDA(cudaMemcpy(t.data(), b->times, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost));
    double span = 0.0;
    for (int i = 0; i < b->n; ++i) {
        const double ms = (double)(t[1 + i] - t[0]) * 1e-6;
        if (done_ms) done_ms[i] = ms;
        span = std::max(span, ms);
    }
    if (span_ms) *span_ms = span;
    return PS_OK;
}

extern "C" int psbatch_queue_stats(psbatch_t* b, int32_t* counts) {
    clear_error();
    PS_ARG(b != nullptr && counts != nullptr, "psbatch_queue_stats: NULL argument");
    for (int k = 0; k < 6; ++k) counts[k] = b->q_counts[k];
    return PS_OK;
}

extern "C" int psbatch_autotune(psweep_t* const* sweeps, int32_t n, const uint8_t* const* images,
                                const ps_box* boxes, const int32_t* n_boxes, float* const* depth_out,
                                const ps_batch_opts* candidates, int32_t n_cand, int32_t reps, int32_t* best,
                                double* ms_out, void* stream) {
    clear_error();
    PS_ARG(candidates != nullptr && n_cand >= 1 && reps >= 1 && reps <= 1000 && best != nullptr &&
               ms_out != nullptr,
           "psbatch_autotune: need candidates, 1..1000 reps, best and ms_out");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    PS_CUDA(cudaEventCreate(&e0));
    PS_CUDA(cudaEventCreate(&e1));
    int st = PS_OK;
    *best = -1;
    for (int c = 0; c < n_cand && st == PS_OK; ++c) {
        psbatch_t* b = nullptr;
        st = psbatch_create(sweeps, n, &candidates[c], &b);
        if (st) break;
        std::vector<double> ms;
        for (int r = 0; r <= reps && st == PS_OK; ++r) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "psbatch_autotune");
                break;
            }
            st = psbatch_run(b, images, boxes, n_boxes, depth_out, stream);
            if (st) break;
            e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "psbatch_autotune");
                break;
            }
            if (r > 0) ms.push_back(t);  // the first run is untimed (and instantiates a graph)
        }
        if (st == PS_OK) st = psbatch_status(b);
        psbatch_destroy(b);
        if (st) break;
        std::sort(ms.begin(), ms.end());
        ms_out[c] = ms[ms.size() / 2];
        if (*best < 0 || ms_out[c] < ms_out[*best]) *best = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// Batched plane sweeps: the device side of psbatch_run.
//
// Every step of psweep_depth for every sweep of a batch runs as a work item
// of one persistent kernel.  Items come from a device queue in a fixed order
// built on the host:
//   Q_REF    rows of a level's reference image
//   Q_QUAD   rows of a level's quad image of one matching camera
//   Q_STATS  rows of a level's reference window statistics (after Q_REF)
//   Q_SWEEP  one tile x plane-chunk item of the sweep (after Q_QUAD, Q_STATS)
//   Q_MERGE  rows of the merged full-resolution map (after every tile)
//   Q_CONT   rows of the continuity filter and boxes (after every Q_MERGE)
// An item whose inputs come from other items waits for a per-sweep counter
// with a bounded spin.  The queue lists every item after all the items it
// waits for, and a CTA only takes an item after every earlier item has been
// taken by a running CTA, so the earliest unfinished item never waits: every
// wait ends.  A wait that still exceeds the time limit latches DEV_TIMEOUT,
// sets the abort flag, and the remaining items are skipped.
#pragma once

#include "sweep_dev.cuh"

namespace ps {

constexpr int PREP_ROWS = 16;   // level rows per Q_REF / Q_QUAD / Q_STATS item
constexpr int MERGE_ROWS = 16;  // output rows per Q_MERGE / Q_CONT item
constexpr int SPIN_LIMIT_ITERS = 1 << 22;  // a dependency wait gives up after its time limit or this many polls

enum : int { Q_REF = 0, Q_QUAD, Q_STATS, Q_SWEEP, Q_MERGE, Q_CONT };

// Per-sweep counters, zeroed per run.
enum : int { C_REF0 = 0, C_REF1, C_PREP0, C_PREP1, C_TILES, C_MERGE, C_OUT, C_N = 8 };

// Queue entry: x = kind | level << 4 | camera << 8, y = sweep, z = index.
__host__ __device__ inline int4 qitem(int kind, int job, int level, int cam, int idx) {
    return make_int4(kind | (level << 4) | (cam << 8), job, idx, 0);
}

// Level images of one level of one sweep.
struct PrepD {
    int s, x0, y0;   // reference: block size (0 = crop) and crop origin
    int Wl, Hl, rho;
    float* ref;
    float2* stats;
    int n_ref_items;  // Q_REF items
    int prep_target;  // Q_QUAD + Q_STATS items
    int cam_s;        // matching images: block size (1 at the crop level)
    int cam_Wl[PS_MAX_CAMS], cam_Hl[PS_MAX_CAMS];
    void* quad[PS_MAX_CAMS];
};

// Static description of one sweep of the batch.
struct JobD {
    int n_cams, n_levels, image_half;
    int ref_w;                 // row pitch of the reference image
    int cam_w[PS_MAX_CAMS];    // row pitch of the matching images
    PrepD prep[PS_MAX_LEVELS];
    MergeP M;                  // merge rule (its box list is unused: boxes come with the run)
    int filter, cont_half;
    float gamma, delta;
    float* merged;             // merged map before the continuity filter
    int tiles_total;           // tiles over both levels
    int merge_items;           // Q_MERGE items (= Q_CONT items)
};

// Per-run inputs and outputs of one sweep (staged from pinned host memory).
struct JobIO {
    const uint8_t* img[1 + PS_MAX_CAMS];
    float* depth;
    int n_boxes, box0;  // boxes[box0 .. box0 + n_boxes) of the run's box list
};

struct BatchArgs {
    const JobD* jobs;
    const LevelD* levels;  // [sweep][PS_MAX_LEVELS]
    const JobIO* io;
    const ps_box* boxes;
    const int4* queue;
    int n_queue;
    int* head;             // next queue entry
    int* abort;            // set when a wait gave up
    unsigned* status;      // DEV_* bits
    int* ctr;              // [sweep][C_N]
    unsigned long long* t;  // [0] kernel start (min over CTAs), [1 + i] sweep i complete (global timer, ns)
    unsigned long long limit_ns;  // time limit of one dependency wait
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int load_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait until *ctr >= target.  False when the batch was aborted or
// the wait gave up (which aborts it).
__device__ inline bool wait_for(const BatchArgs& A, const int* ctr, int target) {
    if (load_acquire(ctr) >= target) return true;
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    for (int it = 0; it < SPIN_LIMIT_ITERS; ++it) {
        if (load_acquire(ctr) >= target) return true;
        if (load_acquire(A.abort)) return false;
        if (global_ns() - t0 > A.limit_ns) break;
        __nanosleep(ns);
        ns = ns < 1024 ? 2 * ns : 1024;
    }
    atomicOr(A.status, DEV_TIMEOUT);
    atomicExch(A.abort, 1);
    return false;
}

// Thread 0: the item's inputs are complete (waiting if needed).
__device__ inline bool item_ready(const BatchArgs& A, int4 q) {
    if (load_acquire(A.abort)) return false;
    const int kind = q.x & 15, lvl = (q.x >> 4) & 1, job = q.y;
    const JobD& J = A.jobs[job];
    const int* c = A.ctr + job * C_N;
    switch (kind) {
        case Q_STATS: return wait_for(A, c + C_REF0 + lvl, J.prep[lvl].n_ref_items);
        case Q_SWEEP: return wait_for(A, c + C_PREP0 + lvl, J.prep[lvl].prep_target);
        case Q_MERGE: return wait_for(A, c + C_TILES, J.tiles_total);
        case Q_CONT: return wait_for(A, c + C_MERGE, J.merge_items);
        default: return true;
    }
}

// All threads: publish the item's writes, then count it.
__device__ __forceinline__ void item_done(int* ctr) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(ctr, 1);
}

template <int TH, int KP>
__global__ void __launch_bounds__(NT, 1) batch_kernel(const __grid_constant__ BatchArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ CamS cams[PS_MAX_CAMS];
    __shared__ __align__(16) LevelD sL;
    __shared__ int4 s_q;
    __shared__ int s_go, s_flag;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x;
    if (tid == 0) atomicMin(A.t, global_ns());
    const uint32_t tmem = tm_alloc(&s_tmem);
    for (;;) {
        if (tid == 0) {
            const int t = atomicAdd(A.head, 1);
            int go = -1;
            if (t < A.n_queue) {
                s_q = A.queue[t];
                go = item_ready(A, s_q) ? 1 : 0;
                __threadfence();  // the inputs' writes are visible to the whole CTA after the barrier
            }
            s_go = go;
        }
        __syncthreads();
        const int go = s_go;
        const int4 q = s_q;
        if (go < 0) break;
        if (go == 0) {  // aborted: skip
            __syncthreads();
            continue;
        }
        const int kind = q.x & 15, lvl = (q.x >> 4) & 1, cam = q.x >> 8, job = q.y, idx = q.z;
        const JobD& J = A.jobs[job];
        const JobIO& io = A.io[job];
        int* c = A.ctr + job * C_N;
        if (kind == Q_SWEEP) {
            // the level record goes to shared memory (read all through the item)
            const int* src = reinterpret_cast<const int*>(A.levels + job * PS_MAX_LEVELS + lvl);
            int* dst = reinterpret_cast<int*>(&sL);
            for (int i = tid; i < (int)(sizeof(LevelD) / sizeof(int)); i += NT) dst[i] = src[i];
            __syncthreads();
            sweep_item<TH, KP>(sL, J.image_half, idx, cams, smem, &s_flag, tmem);
        } else if (kind == Q_REF || kind == Q_STATS) {
            const PrepD& P = J.prep[lvl];
            const int y0 = idx * PREP_ROWS, n = min(PREP_ROWS, P.Hl - y0) * P.Wl;
            (void)PS_DCHECK(y0 >= 0 && y0 < P.Hl, CHK_ITEM);
            for (int i = tid; i < n; i += NT) {
                const int y = y0 + i / P.Wl, x = i % P.Wl;
                if (kind == Q_REF)
                    P.ref[(size_t)y * P.Wl + x] = ref_px(io.img[0], J.ref_w, P.s, P.x0, P.y0, P.Wl, P.Hl, x, y);
                else
                    P.stats[(size_t)y * P.Wl + x] = stats_px(P.ref, P.Wl, P.Hl, P.rho, x, y);
            }
            item_done(c + (kind == Q_REF ? C_REF0 : C_PREP0) + lvl);
        } else if (kind == Q_QUAD) {
            const PrepD& P = J.prep[lvl];
            const int Wl = P.cam_Wl[cam], Hl = P.cam_Hl[cam];
            const int y0 = idx * PREP_ROWS, n = min(PREP_ROWS, Hl - y0) * Wl;
            (void)PS_DCHECK(y0 >= 0 && y0 < Hl && cam < J.n_cams, CHK_ITEM);
            for (int i = tid; i < n; i += NT)
                quad_px(io.img[1 + cam], J.cam_w[cam], P.cam_s, Wl, Hl, P.quad[cam], J.image_half, i % Wl,
                        y0 + i / Wl);
            item_done(c + C_PREP0 + lvl);
        } else {  // Q_MERGE or Q_CONT
            const int W = J.M.W, H = J.M.H;
            const int y0 = idx * MERGE_ROWS, n = min(MERGE_ROWS, H - y0) * W;
            (void)PS_DCHECK(y0 >= 0 && y0 < H, CHK_ITEM);
            const ps_box* bx = A.boxes + io.box0;
            const bool last = kind == Q_CONT || !J.filter;  // this pass writes the output
            for (int i = tid; i < n; i += NT) {
                const int v = y0 + i / W, u = i % W;
                float val = kind == Q_MERGE ? merge_px(J.M, u, v)
                                            : continuity_px(J.merged, W, H, J.cont_half, J.gamma, J.delta, u, v);
                if (last) {
                    if (in_boxes(bx, io.n_boxes, u, v)) val = 0.f;
                    io.depth[(size_t)v * W + u] = val;
                } else {
                    J.merged[(size_t)v * W + u] = val;
                }
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                if (kind == Q_MERGE) atomicAdd(c + C_MERGE, 1);
                // the sweep's last output rows stamp its completion time
                if (last && atomicAdd(c + C_OUT, 1) == J.merge_items - 1) A.t[1 + job] = global_ns();
            }
        }
        __syncthreads();
    }
    tm_free(tmem);
}

}  // namespace ps

// Fisheye plane-sweep stereo at multiple scales (Sec. III-A) on sm_103a.
//
// Kernels:
//   ray_table_kernel   Eq. 1 back-projection of every reference pixel of a
//                      level, in double precision, stored as float4 (once
//                      per rig, at psweep_create).
//   prep_kernel        per frame, in one launch for every level: the
//                      reference image of the level (s x s box mean, or the
//                      centred crop), centred intensities I/255 - 1/2, with
//                      its window mean and sum of squared deviations; the
//                      matching images in "quad" layout: entry (x, y) holds
//                      the 2 x 2 neighbourhood used by one bilinear sample,
//                      so a sample is one 16-byte gather; and the zeroing of
//                      the sweep's work counters.
//   sweep_kernel       the hot loop.  One CTA owns a 64 x 24 tile of output
//                      pixels of one level and walks every plane and every
//                      matching camera: warp the tile + window halo through
//                      the plane into shared memory, box-sum w, w^2, r w and
//                      the invalid count with separable sums, ZNCC -> cost,
//                      minimum over cameras, and a streaming winner-take-all
//                      that keeps the best, second best and the winner's two
//                      neighbours in tensor memory between plane pairs.  The
//                      cost volume never leaves the SM.  Both levels' tiles
//                      share one launch.
//   merge_kernel       full-resolution merge of the levels and box masks.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sweep_dev.cuh"

namespace ps {

namespace {

// ------------------------------------------------------------- ray table

__device__ void distort_d(const ps_camera& c, double x, double y, double* xd, double* yd) {
    double r2 = x * x + y * y;
    double rad = 1.0 + c.k1 * r2 + c.k2 * r2 * r2;
    *xd = x * rad + 2.0 * c.p1 * x * y + c.p2 * (r2 + 2.0 * x * x);
    *yd = y * rad + c.p1 * (r2 + 2.0 * y * y) + 2.0 * c.p2 * x * y;
}

// Unit ray of pixel (u, v) by Eq. 1, undistorting first by Newton
// iteration (residual < 1e-13 within 100 steps, else no ray).  Returns false
// where the pixel has no ray.
__device__ bool ray_of(const ps_camera& c, double u, double v, double r[3]) {
    double xd = (u - c.cx) / c.fx, yd = (v - c.cy) / c.fy;
    double X = xd, Y = yd;
    bool ok = false;
    for (int it = 0; it < 100; ++it) {
        double fx, fy;
        distort_d(c, X, Y, &fx, &fy);
        double ex = fx - xd, ey = fy - yd;
        if (fabs(ex) < 1e-13 && fabs(ey) < 1e-13) {
            ok = true;
            break;
        }
        double r2 = X * X + Y * Y;
        double rad = 1.0 + c.k1 * r2 + c.k2 * r2 * r2;
        double dr = c.k1 + 2.0 * c.k2 * r2;
        double a = rad + 2.0 * X * X * dr + 2.0 * c.p1 * Y + 6.0 * c.p2 * X;
        double b = 2.0 * X * Y * dr + 2.0 * c.p1 * X + 2.0 * c.p2 * Y;
        double d = rad + 2.0 * Y * Y * dr + 6.0 * c.p1 * Y + 2.0 * c.p2 * X;
        double det = a * d - b * b;
        if (det == 0.0) break;
        X -= (d * ex - b * ey) / det;
        Y -= (a * ey - b * ex) / det;
    }
    if (!ok) return false;
    double s = X * X + Y * Y;
    double disc = 1.0 + (1.0 - c.xi * c.xi) * s;
    if (s > c.r2_max || disc < 0.0) return false;
    double f = (c.xi + sqrt(disc)) / (s + 1.0);
    r[0] = f * X;
    r[1] = f * Y;
    r[2] = f - c.xi;
    return true;
}

// Per-pixel rays of a camera, float4 (x, y, z, 0) with NaN where there is none.
__global__ void ray_table_kernel(ps_camera c, int W, int H, float4* rays) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= W || y >= H) return;
    const float nan = __int_as_float(0x7fc00000);
    double r[3];
    float4 out = make_float4(nan, nan, nan, 0.f);
    if (ray_of(c, x, y, r)) out = make_float4((float)r[0], (float)r[1], (float)r[2], 0.f);
    rays[(size_t)y * W + x] = out;
}

// Widest polar angle of a ray through the image, taken on the border of the
// image grown by one pixel (the polar angle grows with the distance from the
// principal point under a one-to-one distortion); a border point without a
// ray counts as pi.  Result: float bits in *out (atomicMax on positive floats).
__global__ void view_angle_kernel(ps_camera c, int W, int H, unsigned* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int per_row = W + 2, per_col = H;
    int n = 2 * per_row + 2 * per_col;
    if (i >= n) return;
    double u, v;
    if (i < per_row) {
        u = i - 1;
        v = -1;
    } else if (i < 2 * per_row) {
        u = i - per_row - 1;
        v = H;
    } else if (i < 2 * per_row + per_col) {
        u = -1;
        v = i - 2 * per_row;
    } else {
        u = W;
        v = i - 2 * per_row - per_col;
    }
    double r[3];
    float ang = 3.14159266f;
    if (ray_of(c, u, v, r)) ang = (float)acos(fmin(1.0, fmax(-1.0, r[2])));
    atomicMax(out, __float_as_uint(ang));
}

// Reference level image and its window statistics in one pass: a 32 x 8
// tile of level pixels plus a window halo is formed in shared memory, the
// tile is written out and each pixel's statistics come from shared memory.
constexpr int RS_TX = 32, RS_TY = 8, RS_MAXH = 4;
constexpr int PREP_T = RS_TX * RS_TY;  // threads of a prep block
__device__ __forceinline__ void ref_stats_tile(const uint8_t* img, int W, int s, int x0, int y0, int Wl, int Hl,
                                               int rho, float* ref, float2* stats, int tbx, int tby, float* tile) {
    const int hw = RS_TX + 2 * rho, hh = RS_TY + 2 * rho;
    const int bx = tbx * RS_TX - rho, by = tby * RS_TY - rho;
    const int tid = threadIdx.x, tx = tid % RS_TX, ty = tid / RS_TX;
    for (int p = tid; p < hw * hh; p += PREP_T) {
        int x = bx + p % hw, y = by + p / hw;
        tile[p] = (x >= 0 && y >= 0 && x < Wl && y < Hl) ? ref_px(img, W, s, x0, y0, Wl, Hl, x, y) : 0.0f;
    }
    __syncthreads();
    const int x = tbx * RS_TX + tx, y = tby * RS_TY + ty;
    if (x >= Wl || y >= Hl) return;
    const float* c = tile + (ty + rho) * hw + tx + rho;
    ref[(size_t)y * Wl + x] = *c;
    stats[(size_t)y * Wl + x] = (x >= rho && y >= rho && x < Wl - rho && y < Hl - rho) ? window_stats(c, hw, rho)
                                                                                      : make_float2(0.f, -1.f);
}

// Quad images of the matching cameras of a level.  A block covers PREP_T
// columns of QROWS rows; each thread walks down its column forming level
// pixel (x, y + 1) once per row (row y's value comes from the previous row)
// and takes the (x + 1) column from its lane neighbour, so every level pixel
// is computed about once per quad that needs it instead of four times.
constexpr int QROWS = 8;
struct QuadJobs {
    const uint8_t* img[PS_MAX_CAMS];
    void* out[PS_MAX_CAMS];
    int W[PS_MAX_CAMS], Wl[PS_MAX_CAMS], Hl[PS_MAX_CAMS];
    int s, half;
};

__device__ __forceinline__ void quad_rows(const QuadJobs& Q, int j, int xb, int yb) {
    const int Wl = Q.Wl[j], Hl = Q.Hl[j];
    const int y0 = yb * QROWS;
    if (xb * PREP_T >= Wl || y0 >= Hl) return;  // whole block outside this camera
    const int x = xb * PREP_T + threadIdx.x;
    const uint8_t* img = Q.img[j];
    const int W = Q.W[j], s = Q.s;
    const bool edge = (threadIdx.x & 31) == 31;
    float a = level_px(img, W, Wl, Hl, s, x, y0);
    float a1 = __shfl_down_sync(0xffffffffu, a, 1);
    if (edge) a1 = level_px(img, W, Wl, Hl, s, x + 1, y0);
    const int y1 = min(Hl, y0 + QROWS);
    for (int y = y0; y < y1; ++y) {
        const float b = level_px(img, W, Wl, Hl, s, x, y + 1);
        float b1 = __shfl_down_sync(0xffffffffu, b, 1);
        if (edge) b1 = level_px(img, W, Wl, Hl, s, x + 1, y + 1);
        if (x < Wl) {
            const size_t o = (size_t)y * Wl + x;
            if (Q.half) {  // FP16 storage: four halves in 8 bytes
                __half2 p = __floats2half2_rn(a, a1), q = __floats2half2_rn(b, b1);
                static_cast<uint2*>(Q.out[j])[o] =
                    make_uint2(*reinterpret_cast<unsigned*>(&p), *reinterpret_cast<unsigned*>(&q));
            } else {
                static_cast<float4*>(Q.out[j])[o] = make_float4(a, a1 - a, b, b1 - b);  // layout: quad_px
            }
        }
        a = b;
        a1 = b1;
    }
}

// Everything a frame's sweep reads, in one launch: per level the reference
// tiles and the quad rows of every matching camera, and the zeroing of the
// sweep's work counters.  Block b takes the role of the range it falls in;
// roles are uniform over a block.
struct PrepLevel {
    int W, s, x0, y0, Wl, Hl, rho;  // reference image and level
    float* ref;
    float2* stats;
    int rs_tiles_x, rs_blocks;      // reference tiles
    QuadJobs Q;
    int n_cams, q_xblocks, q_rows, q_blocks;  // quad blocks: PREP_T columns x QROWS-row bands x cameras
    int* done;                      // per-tile chunk counters to zero
    int n_done;
};

struct PrepP {
    const uint8_t* ref_img;
    int n_levels;
    PrepLevel L[PS_MAX_LEVELS];
    int* tile_counter;
};

__global__ void __launch_bounds__(PREP_T) prep_kernel(const __grid_constant__ PrepP P) {
    __shared__ float tile[(RS_TY + 2 * RS_MAXH) * (RS_TX + 2 * RS_MAXH)];
    int b = blockIdx.x;
    if (b == 0) {
        if (threadIdx.x == 0) *P.tile_counter = 0;
        for (int l = 0; l < P.n_levels; ++l)
            for (int i = threadIdx.x; i < P.L[l].n_done; i += PREP_T) P.L[l].done[i] = 0;
    }
    for (int l = 0; l < P.n_levels; ++l) {
        const PrepLevel& L = P.L[l];
        if (b < L.rs_blocks) {
            ref_stats_tile(P.ref_img, L.W, L.s, L.x0, L.y0, L.Wl, L.Hl, L.rho, L.ref, L.stats, b % L.rs_tiles_x,
                           b / L.rs_tiles_x, tile);
            return;
        }
        b -= L.rs_blocks;
        if (b < L.q_blocks) {
            const int per_cam = L.q_xblocks * L.q_rows, j = b / per_cam, r = b - j * per_cam;
            quad_rows(L.Q, j, r % L.q_xblocks, r / L.q_xblocks);
            return;
        }
        b -= L.q_blocks;
    }
}

// Persistent CTAs take work items (a tile and a chunk of its planes) from a
// counter; levels are ordered so the heavier items start first.
__global__ void __launch_bounds__(NT, 1) sweep_kernel(const __grid_constant__ SweepParams P, int* tile_counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ CamS cams[PS_MAX_CAMS];
    __shared__ int s_tile, s_flag;
    __shared__ uint32_t s_tmem;
    const int total = P.lv[0].n_items + (P.n_levels > 1 ? P.lv[1].n_items : 0);
    const uint32_t tmem = tm_alloc(&s_tmem);
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= total) break;
        if (t < P.lv[0].n_items)
            sweep_item<TH_SINGLE, KP_SINGLE>(P.lv[0], P.image_half, t, cams, smem, &s_flag, tmem);
        else
            sweep_item<TH_SINGLE, KP_SINGLE>(P.lv[1], P.image_half, t - P.lv[0].n_items, cams, smem, &s_flag, tmem);
    }
    tm_free(tmem);
}

// ------------------------------------------------------------- merge

__global__ void merge_kernel(const __grid_constant__ MergeP P, const ps_box* boxes, float* out) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y;
    if (u >= P.W || v >= P.H) return;
    float val = merge_px(P, u, v);
    if (in_boxes(P.boxes, min(P.n_boxes, 16), u, v) || (P.n_boxes > 16 && in_boxes(boxes + 16, P.n_boxes - 16, u, v)))
        val = 0.f;
    out[(size_t)v * P.W + u] = val;
}

// Local depth continuity on the merged map, then the boxes.
__global__ void continuity_kernel(const float* in, int W, int H, int half, float gamma, float delta,
                                  const __grid_constant__ MergeP P, const ps_box* boxes, float* out) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y;
    if (u >= W || v >= H) return;
    float res = continuity_px(in, W, H, half, gamma, delta, u, v);
    if (in_boxes(P.boxes, min(P.n_boxes, 16), u, v) || (P.n_boxes > 16 && in_boxes(boxes + 16, P.n_boxes - 16, u, v)))
        res = 0.f;
    out[(size_t)v * W + u] = res;
}

}  // namespace

// ===================================================================== host

int build_rays(const ps_camera& cam, float4* rays, double* max_angle) {
    const int W = cam.width, H = cam.height;
    ray_table_kernel<<<dim3((W + 127) / 128, H), 128>>>(cam, W, H, rays);
    PS_CUDA(cudaGetLastError());
    if (max_angle) {
        unsigned* bits = nullptr;
        PS_CUDA(cudaMalloc(&bits, sizeof(unsigned)));
        cudaMemset(bits, 0, sizeof(unsigned));
        int n = 2 * (W + 2) + 2 * H;
        view_angle_kernel<<<(n + 255) / 256, 256>>>(cam, W, H, bits);
        unsigned hb = 0;
        cudaError_t e = cudaMemcpy(&hb, bits, sizeof(unsigned), cudaMemcpyDeviceToHost);
        cudaFree(bits);
        if (e != cudaSuccess) return cuda_fail(e, "view angle");
        float a;
        std::memcpy(&a, &hb, sizeof(a));
        *max_angle = a;
    }
    return PS_OK;
}

CamF to_camf(const ps_camera& c) {
    CamF f;
    f.xi = (float)c.xi;
    f.fx = (float)c.fx;
    f.fy = (float)c.fy;
    f.cx = (float)c.cx;
    f.cy = (float)c.cy;
    f.k1 = (float)c.k1;
    f.k2 = (float)c.k2;
    f.p1 = (float)c.p1;
    f.p2 = (float)c.p2;
    f.r2_max = c.r2_max > 3.0e38 ? 3.0e38f : (float)c.r2_max;
    double lim = c.xi > 0 ? std::min(c.xi, 1.0 / c.xi) : 0.0;
    f.lim = (float)(-lim);
    f.width = c.width;
    f.height = c.height;
    return f;
}

}  // namespace ps

using namespace ps;

namespace {

void free_sweep(psweep_t* h) {
    if (!h) return;
    h->prof.release();
    for (int l = 0; l < PS_MAX_LEVELS; ++l) {
        cudaFree(h->rays[l]);
        cudaFree(h->planes[l]);
        cudaFree(h->ref_img[l]);
        cudaFree(h->stats[l]);
        cudaFree(h->partial[l]);
        cudaFree(h->done[l]);
        for (int j = 0; j < PS_MAX_CAMS; ++j) cudaFree(h->quad[l][j]);
        cudaFree(h->out_depth[l]);
        cudaFree(h->out_c1[l]);
        cudaFree(h->out_c2[l]);
        cudaFree(h->out_k[l]);
    }
    cudaFree(h->boxes_dev);
    cudaFree(h->tile_counter);
    cudaFree(h->status);
    for (int i = 0; i <= PS_MAX_CAMS; ++i) cudaFree(h->stage_img[i]);
    cudaFree(h->stage_depth);
    cudaFree(h->merged);
    delete h;
}

int check_camera(const ps_camera& c, const char* what) {
    PS_ARG(c.width > 0 && c.height > 0 && c.width <= 16384 && c.height <= 16384, "%s: bad image size %dx%d", what,
           c.width, c.height);
    PS_ARG(std::isfinite(c.fx) && std::isfinite(c.fy) && c.fx > 0 && c.fy > 0, "%s: focal lengths must be > 0",
           what);
    PS_ARG(std::isfinite(c.xi) && c.xi >= 0, "%s: xi must be >= 0", what);
    PS_ARG(std::isfinite(c.cx) && std::isfinite(c.cy), "%s: principal point not finite", what);
    PS_ARG(c.r2_max > 0, "%s: r2_max must be > 0", what);
    return PS_OK;
}

ps_camera scaled_camera(const ps_camera& c, int s) {
    ps_camera o = c;
    o.fx = c.fx / s;
    o.fy = c.fy / s;
    o.cx = (c.cx - (s - 1) / 2.0) / s;
    o.cy = (c.cy - (s - 1) / 2.0) / s;
    o.width = c.width / s;
    o.height = c.height / s;
    return o;
}

}  // namespace

namespace ps {

void fill_level(const psweep_t* h, int l, int th, int chunk, LevelD& D) {
    std::memset(&D, 0, sizeof(D));
    const ps_level& L = h->levels[l];
    D.W = h->lW[l];
    D.H = h->lH[l];
    D.rho = L.window / 2;
    D.n_planes = h->n_planes[l];
    D.n_sets = L.n_sets;
    for (int k = 0; k < L.n_sets; ++k) D.sets[k] = h->sets[l][k];
    D.planes = h->planes[l];
    D.rays = h->rays[l];
    D.ref = h->ref_img[l];
    D.stats = h->stats[l];
    D.n_cams = h->n_cams;
    for (int j = 0; j < h->n_cams; ++j) {
        for (int i = 0; i < 9; ++i) D.cams[j].R[i] = (float)h->poses[j].R[i];
        for (int i = 0; i < 3; ++i) D.cams[j].t[i] = (float)h->poses[j].t[i];
        D.cams[j].cam = to_camf(h->lcam[l][j]);
        D.cams[j].quad = h->quad[l][j];
    }
    D.tiles_x = (D.W + TW - 1) / TW;
    D.tiles_y = (D.H + th - 1) / th;
    D.n_tiles = D.tiles_x * D.tiles_y;
    D.k_begin = 0;
    D.k_end = D.n_planes;
    D.chunk = chunk;
    D.n_chunks = (D.n_planes + D.chunk - 1) / D.chunk;
    D.n_items = D.n_tiles * D.n_chunks;
    D.depth = h->out_depth[l];
    D.c1 = h->out_c1[l];
    D.c2 = h->out_c2[l];
    D.kstar = h->out_k[l];
    D.status = h->status;
}

int sweep_sync_status(psweep_t* h, cudaStream_t s) {
    unsigned st = 0;
    PS_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    if (!st) return PS_OK;
    PS_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), s));
    PS_CUDA(cudaStreamSynchronize(s));
    set_error("psweep: a tile's plane chunks were counted more often than it has chunks "
              "(overlapping calls on one sweep handle?)");
    return PS_ERR_STATE;
}

int balanced_chunk(int n_planes, int most) {
    const int n_chunks = (n_planes + most - 1) / most;
    return (n_planes + n_chunks - 1) / n_chunks;
}

void fill_merge(const psweep_t* h, const LevelD* lv, MergeP& M) {
    std::memset(&M, 0, sizeof(M));
    M.W = h->ref.width;
    M.H = h->ref.height;
    M.s = 1;
    M.Wl = M.Hl = 1;
    for (int l = 0; l < h->n_levels; ++l) {
        const ps_level& L = h->levels[l];
        if (L.kind == PS_LEVEL_DOWNSAMPLE) {
            M.low = lv[l].depth;
            M.low_c1 = lv[l].c1;
            M.low_c2 = lv[l].c2;
            M.s = L.factor;
            M.Wl = h->lW[l];
            M.Hl = h->lH[l];
        } else {
            M.crop = lv[l].depth;
            M.crop_c1 = lv[l].c1;
            M.crop_c2 = lv[l].c2;
            M.cx0 = h->cx0[l];
            M.cy0 = h->cy0[l];
            M.cw = L.crop_w;
            M.ch = L.crop_h;
        }
    }
    const ps_filter& F = h->filter;
    if (F.enable) {
        M.filter = 1;
        M.alpha_upper = (float)F.alpha_upper;
        M.alpha_lower = (float)F.alpha_lower;
        M.split_row = (float)(F.split_row >= 0 ? F.split_row : h->ref.height / 2.0);
        M.ratio_min = (float)F.ratio_min;
    }
}

}  // namespace ps

extern "C" int psweep_create(const ps_sweep_desc* d, psweep_t** out) {
    clear_error();
    PS_ARG(out != nullptr, "psweep_create: out is NULL");
    *out = nullptr;
    PS_ARG(d != nullptr, "psweep_create: desc is NULL");
    int st = check_camera(d->ref, "reference camera");
    if (st) return st;
    PS_ARG(d->n_cams >= 1 && d->n_cams <= PS_MAX_CAMS, "n_cams must be in 1..%d", PS_MAX_CAMS);
    PS_ARG(d->cams && d->ref_to_cam, "cams / ref_to_cam are NULL");
    PS_ARG(d->n_levels >= 1 && d->n_levels <= PS_MAX_LEVELS, "n_levels must be in 1..%d", PS_MAX_LEVELS);
    PS_ARG(d->levels != nullptr, "levels is NULL");
    int n_down = 0, n_crop = 0;
    for (int l = 0; l < d->n_levels; ++l) {
        const ps_level& L = d->levels[l];
        PS_ARG(L.window == 5 || L.window == 7 || L.window == 9, "level %d: window must be 5, 7 or 9", l);
        PS_ARG(L.n_sets >= 1 && L.n_sets <= PS_MAX_SETS, "level %d: n_sets must be in 1..%d", l, PS_MAX_SETS);
        for (int s = 0; s < L.n_sets; ++s) {
            const ps_plane_set& P = L.sets[s];
            PS_ARG(P.count >= 1 && P.count <= 4096, "level %d set %d: count must be in 1..4096", l, s);
            PS_ARG(P.family == PS_PLANES_FRONTO || P.family == PS_PLANES_GROUND, "level %d set %d: bad family", l,
                   s);
            if (P.family == PS_PLANES_FRONTO)
                PS_ARG(P.a > 0 && P.b >= P.a, "level %d set %d: need 0 < near <= far", l, s);
            else {
                double nn = std::sqrt(P.n[0] * P.n[0] + P.n[1] * P.n[1] + P.n[2] * P.n[2]);
                PS_ARG(nn > 0 && P.a > 0 && P.b >= P.a, "level %d set %d: need a normal and 0 < a <= b", l, s);
            }
        }
        if (L.kind == PS_LEVEL_DOWNSAMPLE) {
            ++n_down;
            PS_ARG(L.factor == 1 || L.factor == 2 || L.factor == 4, "level %d: factor must be 1, 2 or 4", l);
            PS_ARG(d->ref.width % L.factor == 0 && d->ref.height % L.factor == 0,
                   "level %d: factor must divide the reference size", l);
            for (int j = 0; j < d->n_cams; ++j)
                PS_ARG(d->cams[j].width % L.factor == 0 && d->cams[j].height % L.factor == 0,
                       "level %d: factor must divide camera %d's size", l, j);
        } else if (L.kind == PS_LEVEL_CROP) {
            ++n_crop;
            PS_ARG(L.crop_w > 0 && L.crop_h > 0 && L.crop_w <= d->ref.width && L.crop_h <= d->ref.height,
                   "level %d: bad crop size", l);
        } else {
            PS_ARG(false, "level %d: unknown kind %d", l, L.kind);
        }
    }
    PS_ARG(n_down <= 1 && n_crop <= 1, "at most one downsample level and one crop level");
    if (d->filter.enable) {
        const ps_filter& f = d->filter;
        PS_ARG(f.window >= 1 && f.window <= 15 && f.window % 2 == 1, "filter: window must be odd, 1 .. 15");
        PS_ARG(f.delta >= 0 && f.delta <= 1 && f.gamma > 0 && f.ratio_min >= 0,
               "filter: need 0 <= delta <= 1, gamma > 0, ratio_min >= 0");
        PS_ARG(std::isfinite(f.alpha_upper) && std::isfinite(f.alpha_lower), "filter: alpha not finite");
    }
    for (int j = 0; j < d->n_cams; ++j) {
        st = check_camera(d->cams[j], "matching camera");
        if (st) return st;
    }

    psweep_t* h = new psweep_t();
    h->ref = d->ref;
    h->n_cams = d->n_cams;
    h->n_levels = d->n_levels;
    h->filter = d->filter;
    h->image_half = d->image_half ? 1 : 0;
    for (int j = 0; j < d->n_cams; ++j) {
        h->cams[j] = d->cams[j];
        h->poses[j] = d->ref_to_cam[j];
    }
#define PS_TRY(call)                                 \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) {                     \
            free_sweep(h);                           \
            set_error("%s: %s", #call, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA; \
        }                                            \
    } while (0)
    for (int l = 0; l < d->n_levels; ++l) {
        const ps_level& L = d->levels[l];
        h->levels[l] = L;
        if (L.kind == PS_LEVEL_DOWNSAMPLE) {
            h->lref[l] = scaled_camera(d->ref, L.factor);
            for (int j = 0; j < d->n_cams; ++j) h->lcam[l][j] = scaled_camera(d->cams[j], L.factor);
            h->cx0[l] = h->cy0[l] = 0;
        } else {
            int x0 = (d->ref.width - L.crop_w) / 2, y0 = (d->ref.height - L.crop_h) / 2;
            h->lref[l] = d->ref;
            h->lref[l].cx -= x0;
            h->lref[l].cy -= y0;
            h->lref[l].width = L.crop_w;
            h->lref[l].height = L.crop_h;
            for (int j = 0; j < d->n_cams; ++j) h->lcam[l][j] = d->cams[j];
            h->cx0[l] = x0;
            h->cy0[l] = y0;
        }
        const int W = h->lref[l].width, H = h->lref[l].height;
        h->lW[l] = W;
        h->lH[l] = H;
        // plane table (double on the host, stored as float)
        std::vector<PlaneD> planes;
        for (int s = 0; s < L.n_sets; ++s) {
            const ps_plane_set& P = L.sets[s];
            SetD S;
            S.family = P.family;
            S.start = (int)planes.size();
            S.count = P.count;
            S.a = (float)P.a;
            S.b = (float)P.b;
            double n[3] = {0, 0, 1};
            if (P.family == PS_PLANES_GROUND) {
                double nn = std::sqrt(P.n[0] * P.n[0] + P.n[1] * P.n[1] + P.n[2] * P.n[2]);
                for (int i = 0; i < 3; ++i) n[i] = P.n[i] / nn;
            }
            S.nx = (float)n[0];
            S.ny = (float)n[1];
            S.nz = (float)n[2];
            h->sets[l][s] = S;
            for (int i = 0; i < P.count; ++i) {
                double t = P.count > 1 ? (double)i / (P.count - 1) : 0.0;
                double dd = P.family == PS_PLANES_FRONTO ? 1.0 / (1.0 / P.b + t * (1.0 / P.a - 1.0 / P.b))
                                                         : P.a + t * (P.b - P.a);
                planes.push_back({(float)n[0], (float)n[1], (float)n[2], (float)dd});
            }
        }
        h->n_planes[l] = (int)planes.size();
        PS_TRY(cudaMalloc(&h->planes[l], sizeof(PlaneD) * planes.size()));
        PS_TRY(cudaMemcpy(h->planes[l], planes.data(), sizeof(PlaneD) * planes.size(), cudaMemcpyHostToDevice));
        PS_TRY(cudaMalloc(&h->rays[l], sizeof(float4) * (size_t)W * H));
        if (build_rays(h->lref[l], h->rays[l], nullptr)) {
            free_sweep(h);
            return PS_ERR_CUDA;
        }
        PS_TRY(cudaMalloc(&h->ref_img[l], sizeof(float) * (size_t)W * H));
        PS_TRY(cudaMalloc(&h->stats[l], sizeof(float2) * (size_t)W * H));
        {
            // work items: tiles x chunks of at most PLANE_CHUNK planes, so that
            // items of both levels cost about the same and balance across SMs;
            // a level with at least 16 waves of items even at twice that takes
            // chunks of up to 2 PLANE_CHUNK (half the per-item work: direction
            // tables, reference tile, chunk records; the tail stays short)
            const int n_tiles = ((W + TW - 1) / TW) * ((H + TH_SINGLE - 1) / TH_SINGLE);
            int dev = 0, sms = 0;
            PS_TRY(cudaGetDevice(&dev));
            PS_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            const int c2 = balanced_chunk(h->n_planes[l], 2 * PLANE_CHUNK);
            const long long items2 = (long long)n_tiles * ((h->n_planes[l] + c2 - 1) / c2);
            h->chunk[l] = items2 >= 16LL * sms ? c2 : balanced_chunk(h->n_planes[l], PLANE_CHUNK);
            const int n_chunks = (h->n_planes[l] + h->chunk[l] - 1) / h->chunk[l];
            if (n_chunks > 1)
                PS_TRY(cudaMalloc(&h->partial[l], sizeof(float) * 7 * TH_SINGLE * TW * (size_t)n_tiles * n_chunks));
            PS_TRY(cudaMalloc(&h->done[l], sizeof(int) * (size_t)n_tiles));
        }
        for (int j = 0; j < d->n_cams; ++j) {
            const ps_camera& cj = h->lcam[l][j];
            PS_TRY(cudaMalloc(&h->quad[l][j], (d->image_half ? sizeof(uint2) : sizeof(float4)) * (size_t)cj.width * cj.height));
        }
        PS_TRY(cudaMalloc(&h->out_depth[l], sizeof(float) * (size_t)W * H));
        PS_TRY(cudaMalloc(&h->out_c1[l], sizeof(float) * (size_t)W * H));
        PS_TRY(cudaMalloc(&h->out_c2[l], sizeof(float) * (size_t)W * H));
        PS_TRY(cudaMalloc(&h->out_k[l], sizeof(int32_t) * (size_t)W * H));
    }
    PS_TRY(cudaMalloc(&h->boxes_dev, sizeof(ps_box) * 256));
    h->boxes_cap = 256;
    PS_TRY(cudaMalloc(&h->stage_img[0], (size_t)d->ref.width * d->ref.height));
    for (int j = 0; j < d->n_cams; ++j)
        PS_TRY(cudaMalloc(&h->stage_img[1 + j], (size_t)d->cams[j].width * d->cams[j].height));
    PS_TRY(cudaMalloc(&h->stage_depth, sizeof(float) * (size_t)d->ref.width * d->ref.height));
    if (d->filter.enable) PS_TRY(cudaMalloc(&h->merged, sizeof(float) * (size_t)d->ref.width * d->ref.height));
    PS_TRY(cudaMalloc(&h->tile_counter, sizeof(int)));
    PS_TRY(cudaMalloc(&h->status, sizeof(unsigned)));
    PS_TRY(cudaMemset(h->status, 0, sizeof(unsigned)));
    {
        int dev = 0, optin = 0;
        PS_TRY(cudaGetDevice(&dev));
        PS_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        h->smem_optin = optin;
        PS_TRY(cudaFuncSetAttribute(sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024));
    }
    {
        int dev = 0, sms = 0, per_sm = 0;
        PS_TRY(cudaGetDevice(&dev));
        PS_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        PS_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel, NT, sweep_smem<TH_SINGLE, KP_SINGLE>(4, d->n_cams)));
        if (per_sm < 1) {
            free_sweep(h);
            PS_ARG(false, "psweep_create: the sweep kernel does not fit one SM");
        }
        h->grid = sms;  // one CTA per SM: each CTA allocates all of its SM's tensor memory
    }
    PS_TRY(cudaDeviceSynchronize());
#undef PS_TRY
    *out = h;
    return PS_OK;
}

extern "C" void psweep_destroy(psweep_t* h) { free_sweep(h); }

namespace {

// The launches of one sweep up to the level outputs: one prep launch (level
// images, reference statistics, quads, counters) and the persistent sweep
// kernel.  With ranges (plane_lo/plane_hi per level, NULL = every plane)
// and records (per level, NULL = the level outputs) the sweep covers only
// those planes and writes per-pixel records.  by_level receives each
// level's record in the handle's level order.
int launch_sweep(psweep_t* h, const uint8_t* const* images, const int32_t* plane_lo, const int32_t* plane_hi,
                 float* const* records, const ps_level_out* level_out, cudaStream_t s, LevelD* by_level) {
    SweepParams P;
    std::memset(&P, 0, sizeof(P));
    P.n_levels = h->n_levels;
    P.image_half = h->image_half;
    h->prof.mark(0, s);
    // heavier level first in the tile order (planes x halo samples per tile)
    int order[PS_MAX_LEVELS] = {0, 1};
    if (h->n_levels == 2) {
        auto cost = [&](int l) {  // one work item: planes x halo samples
            int r = h->levels[l].window / 2;
            return (double)h->chunk[l] * (TW + 2 * r) * (TH_SINGLE + 2 * r);
        };
        if (cost(1) > cost(0)) std::swap(order[0], order[1]);
    }
    PrepP prep;
    std::memset(&prep, 0, sizeof(prep));
    prep.ref_img = images[0];
    prep.n_levels = h->n_levels;
    int prep_blocks = 0;
    for (int oi = 0; oi < h->n_levels; ++oi) {
        const int l = order[oi];
        const ps_level& L = h->levels[l];
        const int W = h->lW[l], H = h->lH[l];
        const bool down = L.kind == PS_LEVEL_DOWNSAMPLE;
        PrepLevel& R = prep.L[oi];
        R.W = h->ref.width;
        R.s = down ? L.factor : 0;
        R.x0 = down ? 0 : h->cx0[l];
        R.y0 = down ? 0 : h->cy0[l];
        R.Wl = W;
        R.Hl = H;
        R.rho = L.window / 2;
        R.ref = h->ref_img[l];
        R.stats = h->stats[l];
        R.rs_tiles_x = (W + RS_TX - 1) / RS_TX;
        R.rs_blocks = R.rs_tiles_x * ((H + RS_TY - 1) / RS_TY);
        {
            QuadJobs& Q = R.Q;
            int wmax = 0, hmax = 0;
            for (int j = 0; j < h->n_cams; ++j) {
                const ps_camera& cj = h->lcam[l][j];
                Q.img[j] = images[1 + j];
                Q.out[j] = h->quad[l][j];
                Q.W[j] = h->cams[j].width;
                Q.Wl[j] = cj.width;
                Q.Hl[j] = cj.height;
                wmax = std::max(wmax, cj.width);
                hmax = std::max(hmax, cj.height);
            }
            Q.s = down ? L.factor : 1;
            Q.half = h->image_half;
            R.n_cams = h->n_cams;
            R.q_xblocks = (wmax + PREP_T - 1) / PREP_T;
            R.q_rows = (hmax + QROWS - 1) / QROWS;
            R.q_blocks = R.q_xblocks * R.q_rows * h->n_cams;
        }
        prep_blocks += R.rs_blocks + R.q_blocks;
        LevelD& D = P.lv[oi];
        fill_level(h, l, TH_SINGLE, h->chunk[l], D);
        if (plane_lo) {
            // planes [lo, hi) only, in chunks of at most the handle's chunk (so the
            // chunk scratch sized for the whole level holds them)
            D.k_begin = plane_lo[l];
            D.k_end = plane_hi[l];
            D.chunk = balanced_chunk(std::max(1, D.k_end - D.k_begin), h->chunk[l]);
            D.n_chunks = std::max(1, (D.k_end - D.k_begin + D.chunk - 1) / D.chunk);
            D.n_items = D.n_tiles * D.n_chunks;
        }
        if (records) D.records = records[l];
        D.partial = h->partial[l];
        D.done = h->done[l];
        R.done = D.done;  // zeroed by the prep launch
        R.n_done = D.n_tiles;
        const ps_level_out* lo = level_out ? &level_out[l] : nullptr;
        if (lo && lo->depth) D.depth = lo->depth;
        if (lo && lo->best_cost) D.c1 = lo->best_cost;
        if (lo && lo->second_cost) D.c2 = lo->second_cost;
        if (lo && lo->plane_idx) D.kstar = lo->plane_idx;
    }
    PS_CUDA(cudaGetLastError());
    size_t smem = 0;
    int tiles = 0;
    for (int l = 0; l < h->n_levels; ++l) {
        int r = P.lv[l].rho;
        const int nc = h->n_cams;
        smem = std::max(smem, sweep_smem<TH_SINGLE, KP_SINGLE>(r, nc));
        tiles += P.lv[l].n_items;
    }
    prep.tile_counter = h->tile_counter;
    prep_kernel<<<prep_blocks, PREP_T, 0, s>>>(prep);
    PS_CUDA(cudaGetLastError());
    h->prof.mark(1, s);
    sweep_kernel<<<std::min(tiles, h->grid), NT, smem, s>>>(P, h->tile_counter);
    PS_CUDA(cudaGetLastError());
    h->prof.mark(2, s);
    for (int oi = 0; oi < h->n_levels; ++oi) by_level[order[oi]] = P.lv[oi];
    return PS_OK;
}

// The level merge, the filters and the boxes into depth_out (level records
// in the handle's level order).
int merge_levels(psweep_t* h, const LevelD* by_level, const ps_box* boxes, int32_t n_boxes, float* depth_out,
                 cudaStream_t s) {
    MergeP M;
    fill_merge(h, by_level, M);
    const ps_filter& F = h->filter;
    M.n_boxes = n_boxes;
    for (int b = 0; b < n_boxes && b < 16; ++b) M.boxes[b] = boxes[b];
    if (n_boxes > 16)
        PS_CUDA(cudaMemcpyAsync(h->boxes_dev, boxes, sizeof(ps_box) * n_boxes, cudaMemcpyHostToDevice, s));
    if (F.enable) {
        // cost filters and merge into the scratch map; continuity and boxes into the output
        MergeP M0 = M;
        M0.n_boxes = 0;
        merge_kernel<<<dim3((M.W + 127) / 128, M.H), 128, 0, s>>>(M0, h->boxes_dev, h->merged);
        PS_CUDA(cudaGetLastError());
        continuity_kernel<<<dim3((M.W + 127) / 128, M.H), 128, 0, s>>>(h->merged, M.W, M.H, F.window / 2,
                                                                       (float)F.gamma, (float)F.delta, M,
                                                                       h->boxes_dev, depth_out);
    } else {
        merge_kernel<<<dim3((M.W + 127) / 128, M.H), 128, 0, s>>>(M, h->boxes_dev, depth_out);
    }
    PS_CUDA(cudaGetLastError());
    return PS_OK;
}

int check_frame_args(psweep_t* h, const uint8_t* const* images, const char* fn) {
    PS_ARG(h != nullptr, "%s: handle is NULL", fn);
    PS_ARG(images != nullptr, "%s: images is NULL", fn);
    for (int i = 0; i <= h->n_cams; ++i) PS_ARG(images[i] != nullptr, "%s: images[%d] is NULL", fn, i);
    return PS_OK;
}

}  // namespace

extern "C" int psweep_depth(psweep_t* h, const uint8_t* const* images, const ps_box* boxes, int32_t n_boxes,
                            float* depth_out, const ps_level_out* level_out, void* stream) {
    clear_error();
    int st = check_frame_args(h, images, "psweep_depth");
    if (st) return st;
    PS_ARG(depth_out != nullptr, "psweep_depth: depth_out is NULL");
    PS_ARG(n_boxes >= 0 && n_boxes <= h->boxes_cap, "psweep_depth: n_boxes must be in 0..%d", h->boxes_cap);
    PS_ARG(n_boxes == 0 || boxes != nullptr, "psweep_depth: boxes is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    LevelD by_level[PS_MAX_LEVELS];
    st = launch_sweep(h, images, nullptr, nullptr, nullptr, level_out, s, by_level);
    if (st) return st;
    st = merge_levels(h, by_level, boxes, n_boxes, depth_out, s);
    if (st) return st;
    h->prof.mark(3, s);
    h->prof.end_call();
    return PS_OK;
}

extern "C" int psweep_level_outputs(psweep_t* h, const ps_level_out* level_out, void* stream) {
    clear_error();
    PS_ARG(h != nullptr && level_out != nullptr, "psweep_level_outputs: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (int l = 0; l < h->n_levels; ++l) {
        const size_t n = (size_t)h->lW[l] * h->lH[l];
        const ps_level_out& o = level_out[l];
        if (o.depth) PS_CUDA(cudaMemcpyAsync(o.depth, h->out_depth[l], 4 * n, cudaMemcpyDeviceToDevice, s));
        if (o.best_cost) PS_CUDA(cudaMemcpyAsync(o.best_cost, h->out_c1[l], 4 * n, cudaMemcpyDeviceToDevice, s));
        if (o.second_cost) PS_CUDA(cudaMemcpyAsync(o.second_cost, h->out_c2[l], 4 * n, cudaMemcpyDeviceToDevice, s));
        if (o.plane_idx) PS_CUDA(cudaMemcpyAsync(o.plane_idx, h->out_k[l], 4 * n, cudaMemcpyDeviceToDevice, s));
    }
    return PS_OK;
}

extern "C" int psweep_depth_planes(psweep_t* h, const uint8_t* const* images, const int32_t* plane_lo,
                                   const int32_t* plane_hi, float* const* records, void* stream) {
    clear_error();
    int st = check_frame_args(h, images, "psweep_depth_planes");
    if (st) return st;
    PS_ARG(plane_lo && plane_hi && records, "psweep_depth_planes: NULL argument");
    for (int l = 0; l < h->n_levels; ++l) {
        PS_ARG(0 <= plane_lo[l] && plane_lo[l] <= plane_hi[l] && plane_hi[l] <= h->n_planes[l],
               "psweep_depth_planes: level %d: need 0 <= plane_lo <= plane_hi <= %d", l, h->n_planes[l]);
        PS_ARG(records[l] != nullptr, "psweep_depth_planes: records[%d] is NULL", l);
    }
    cudaStream_t s = (cudaStream_t)stream;
    LevelD by_level[PS_MAX_LEVELS];
    st = launch_sweep(h, images, plane_lo, plane_hi, records, nullptr, s, by_level);
    if (st) return st;
    h->prof.mark(3, s);
    h->prof.end_call();
    return PS_OK;
}

namespace ps {
namespace {

struct RecordMergeP {
    LevelD L;
    int n_parts;
    const float* rec[PS_MAX_PARTS];
    int lo[PS_MAX_PARTS];
};

__global__ void merge_records_kernel(const __grid_constant__ RecordMergeP P) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= P.L.W || y >= P.L.H) return;
    merge_record_px(P.L, P.rec, P.lo, P.n_parts, x, y);
}

}  // namespace
}  // namespace ps

extern "C" int psweep_merge_records(psweep_t* h, int32_t n_parts, const int32_t* part_lo,
                                    const float* const* records, const ps_box* boxes, int32_t n_boxes,
                                    float* depth_out, const ps_level_out* level_out, void* stream) {
    clear_error();
    PS_ARG(h != nullptr, "psweep_merge_records: handle is NULL");
    PS_ARG(n_parts >= 1 && n_parts <= PS_MAX_PARTS, "psweep_merge_records: n_parts must be in 1..%d", PS_MAX_PARTS);
    PS_ARG(part_lo && records && depth_out, "psweep_merge_records: NULL argument");
    PS_ARG(n_boxes >= 0 && n_boxes <= h->boxes_cap, "psweep_merge_records: n_boxes must be in 0..%d", h->boxes_cap);
    PS_ARG(n_boxes == 0 || boxes != nullptr, "psweep_merge_records: boxes is NULL");
    const int NL = h->n_levels;
    for (int l = 0; l < NL; ++l) {
        PS_ARG(part_lo[l] == 0, "psweep_merge_records: level %d: the first part must start at plane 0", l);
        for (int p = 0; p < n_parts; ++p) {
            const int lo = part_lo[p * NL + l], hi = p + 1 < n_parts ? part_lo[(p + 1) * NL + l] : h->n_planes[l];
            PS_ARG(lo <= hi && hi <= h->n_planes[l], "psweep_merge_records: level %d: part starts must rise to at most %d",
                   l, h->n_planes[l]);
            PS_ARG(hi == lo || records[p * NL + l] != nullptr, "psweep_merge_records: records of part %d level %d is NULL",
                   p, l);
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    h->prof.mark(0, s);
    h->prof.mark(1, s);
    LevelD by_level[PS_MAX_LEVELS];
    for (int l = 0; l < NL; ++l) {
        RecordMergeP P;
        std::memset(&P, 0, sizeof(P));
        fill_level(h, l, TH_SINGLE, h->chunk[l], P.L);
        const ps_level_out* lo = level_out ? &level_out[l] : nullptr;
        if (lo && lo->depth) P.L.depth = lo->depth;
        if (lo && lo->best_cost) P.L.c1 = lo->best_cost;
        if (lo && lo->second_cost) P.L.c2 = lo->second_cost;
        if (lo && lo->plane_idx) P.L.kstar = lo->plane_idx;
        P.n_parts = n_parts;
        for (int p = 0; p < n_parts; ++p) {
            P.rec[p] = records[p * NL + l];
            P.lo[p] = part_lo[p * NL + l];
        }
        merge_records_kernel<<<dim3((P.L.W + 127) / 128, P.L.H), 128, 0, s>>>(P);
        PS_CUDA(cudaGetLastError());
        by_level[l] = P.L;
    }
    h->prof.mark(2, s);
    int st = merge_levels(h, by_level, boxes, n_boxes, depth_out, s);
    if (st) return st;
    h->prof.mark(3, s);
    h->prof.end_call();
    return PS_OK;
}

extern "C" int psweep_profile(psweep_t* h, int32_t capacity) {
    clear_error();
    PS_ARG(h != nullptr && capacity >= 0 && capacity <= (1 << 20), "psweep_profile: bad arguments");
    return h->prof.enable(3, capacity);
}

extern "C" int psweep_profile_read(psweep_t* h, double* stage_ms, int32_t* n_calls) {
    clear_error();
    PS_ARG(h != nullptr && stage_ms != nullptr, "psweep_profile_read: NULL argument");
    PS_ARG(h->prof.cap > 0, "psweep_profile_read: profiling is off");
    return h->prof.read(stage_ms, n_calls);
}

extern "C" int psweep_frame_host(psweep_t* h, tsdf_t* t, const uint8_t* const* host_images, const ps_box* boxes,
                                 int32_t n_boxes, const ps_pose* world_to_ref, const double* local_center,
                                 float* host_depth_out, void* stream) {
    clear_error();
    PS_ARG(h != nullptr && host_images != nullptr, "psweep_frame_host: handle or images NULL");
    PS_ARG(t == nullptr || world_to_ref != nullptr, "psweep_frame_host: world_to_ref is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const uint8_t* dev[1 + PS_MAX_CAMS];
    for (int i = 0; i <= h->n_cams; ++i) {
        PS_ARG(host_images[i] != nullptr, "psweep_frame_host: host_images[%d] is NULL", i);
        const ps_camera& c = i == 0 ? h->ref : h->cams[i - 1];
        PS_CUDA(cudaMemcpyAsync(h->stage_img[i], host_images[i], (size_t)c.width * c.height,
                                cudaMemcpyHostToDevice, s));
        dev[i] = h->stage_img[i];
    }
    int st = psweep_depth(h, dev, boxes, n_boxes, h->stage_depth, nullptr, stream);
    if (st) return st;
    if (t) {
        st = tsdf_integrate(t, h->stage_depth, world_to_ref, local_center, stream);
        if (st) return st;
    }
    if (host_depth_out)
        PS_CUDA(cudaMemcpyAsync(host_depth_out, h->stage_depth, sizeof(float) * (size_t)h->ref.width * h->ref.height,
                                cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    return PS_OK;
}

namespace ps {
PS_DEFINE_CHECK_READER(check_bits_sweep)
}  // namespace ps

// Device-side pieces of the fisheye plane sweep (Sec. III-A) shared by the
// single-frame launch (sweep.cu) and the batched persistent launch
// (batch.cu): level and camera records, the per-pixel rules for level
// images, reference statistics and the merge, the tile routine of the hot
// loop, and the sweep handle.
#pragma once

#include <cuda_fp16.h>

#include "internal.cuh"

namespace ps {

constexpr int TW = 64;   // output tile width (pixels)
constexpr int NT = 768;  // threads per CTA (one CTA per SM); all of them warp (phase A)
constexpr int NTV = 512; // threads that own output pixels: phase V, winner-take-all, outputs
constexpr int RUN = 4;   // outputs per horizontal run (phase H)
constexpr int PLANE_CHUNK = 32;  // most planes one work item sweeps (default)
static_assert(NT / 32 >= TW / RUN, "phase H: one warp per run, one lane per halo row");
// Tile height TH (output rows; 16 or 24) and KP (planes warped per camera
// before the window sums, 1 or 2) are template parameters of the tile
// routine; the single-frame launch uses these, the batched launch picks
// any of the four combinations.
constexpr int TH_SINGLE = 24;
constexpr int KP_SINGLE = 2;

struct PlaneD {
    float nx, ny, nz, d;  // plane n . X = d (reference frame)
};

struct SetD {
    int family, start, count;
    float a, b;
    float nx, ny, nz;
};

struct CamJ {
    float R[9], t[3];  // reference -> matching camera
    CamF cam;          // intrinsics at this level
    const void* quad;  // float4 quads, or four halves per quad with FP16 storage
};

struct LevelD {
    int W, H, rho;
    int n_planes, n_sets;
    SetD sets[PS_MAX_SETS];
    const PlaneD* planes;
    const float4* rays;   // (rx, ry, rz, 0), NaN where the pixel has no ray
    const float* ref;     // centred intensities
    const float2* stats;  // reference window mean and sum of squared deviations
    int n_cams;
    CamJ cams[PS_MAX_CAMS];
    int tiles_x, tiles_y, n_tiles;
    int k_begin, k_end;            // planes [k_begin, k_end) are swept (the whole level, or one part of it)
    int chunk, n_chunks, n_items;  // planes per work item, items per tile, tiles x items
    float* partial;                // [n_items][7][TH x TW] chunk results (when n_chunks > 1)
    int* done;                     // [n_tiles] finished chunks per tile (zeroed per launch)
    int* tiles_done;               // bumped once per finished tile (batched launch), or NULL
    unsigned* status;              // latched DEV_* bits of the owning handle, or NULL
    float* depth;
    float* c1;
    float* c2;
    int32_t* kstar;
    float* records;  // non-NULL: write each pixel's record of planes [k_begin, k_end) instead of its outputs
};

// Per-pixel record of a range of planes, as planes of H x W floats: the
// range's best cost, its second best, the costs of the best plane's
// neighbours inside the range (+inf at the range's ends), the costs of the
// range's first and last plane, and the best plane's index (int bits; -1 =
// none).  Records of consecutive ranges merge into the whole level's
// winner-take-all (merge_record_px).
enum { REC_C1, REC_C2, REC_CM, REC_CP, REC_FIRST, REC_LAST, REC_K, REC_N };

// Matching camera as the sweep reads it (staged in shared memory per work
// item).  The projection constants are kept twice: as scalars, and as
// (value, value) pairs for the two-plane form of the warp on packed FP32
// operations.
struct CamS {
    float R[9], t[3];
    float xi, fx, fy, cx, cy, k1, k2, p1, p2, r2_max, lim, wm1, hm1;
    int width;
    const void* quad;
    float2 xi2, fx2, fy2, cx2, cy2, k12, k22, p12, p1x2, p22, p2x2, lim2;  // pairs; p1x2 = 2 p1, p2x2 = 2 p2
};

// CamS of a matching camera.
__device__ __forceinline__ void cam_consts(const CamJ& J, CamS& c) {
    for (int i = 0; i < 9; ++i) c.R[i] = J.R[i];
    for (int i = 0; i < 3; ++i) c.t[i] = J.t[i];
    c.xi = J.cam.xi; c.fx = J.cam.fx; c.fy = J.cam.fy; c.cx = J.cam.cx; c.cy = J.cam.cy;
    c.k1 = J.cam.k1; c.k2 = J.cam.k2; c.p1 = J.cam.p1; c.p2 = J.cam.p2; c.r2_max = J.cam.r2_max;
    c.lim = J.cam.lim;
    c.wm1 = (float)(J.cam.width - 1);
    c.hm1 = (float)(J.cam.height - 1);
    c.width = J.cam.width;
    c.quad = J.quad;
    c.xi2 = make_float2(c.xi, c.xi); c.fx2 = make_float2(c.fx, c.fx); c.fy2 = make_float2(c.fy, c.fy);
    c.cx2 = make_float2(c.cx, c.cx); c.cy2 = make_float2(c.cy, c.cy); c.k12 = make_float2(c.k1, c.k1);
    c.k22 = make_float2(c.k2, c.k2); c.p12 = make_float2(c.p1, c.p1);
    c.p1x2 = make_float2(2.0f * c.p1, 2.0f * c.p1); c.p22 = make_float2(c.p2, c.p2);
    c.p2x2 = make_float2(2.0f * c.p2, 2.0f * c.p2); c.lim2 = make_float2(c.lim, c.lim);
}

struct SweepParams {
    int n_levels;
    int image_half;  // matching quads stored as FP16
    LevelD lv[PS_MAX_LEVELS];
};

// ------------------------------------------------------------- level images

// ------------------------------------------------------------- level images

// Centred intensity of the s x s block at level pixel (x, y), clamped to the
// image.  Blocks of 2 or 4 bytes per row are read as one 2- or 4-byte word
// when the image base allows it (the integer sum is the same either way).
__device__ __forceinline__ float level_px(const uint8_t* img, int W, int Wl, int Hl, int s, int x, int y) {
    x = min(x, Wl - 1);
    y = min(y, Hl - 1);
    int acc = 0;
    const bool words = ((reinterpret_cast<uintptr_t>(img) | (uintptr_t)W) & (uintptr_t)(s - 1)) == 0;
    if (s == 4 && words) {
        for (int dy = 0; dy < 4; ++dy) {
            unsigned v = *reinterpret_cast<const unsigned*>(img + (size_t)(4 * y + dy) * W + 4 * x);
            acc += (int)((v & 0xffu) + ((v >> 8) & 0xffu) + ((v >> 16) & 0xffu) + (v >> 24));
        }
    } else if (s == 2 && words) {
        for (int dy = 0; dy < 2; ++dy) {
            unsigned short v = *reinterpret_cast<const unsigned short*>(img + (size_t)(2 * y + dy) * W + 2 * x);
            acc += (int)((v & 0xffu) + (v >> 8));
        }
    } else {
        for (int dy = 0; dy < s; ++dy)
            for (int dx = 0; dx < s; ++dx) acc += img[(size_t)(s * y + dy) * W + (s * x + dx)];
    }
    // one explicit rounding, whatever the calling kernel lets the compiler contract
    return __fmaf_rn((float)acc, 1.0f / (255.0f * (float)(s * s)), -0.5f);
}

// Reference intensity at level pixel (x, y): the s x s block mean (s > 0), or
// pixel (x0 + x, y0 + y) of the full image (s == 0, the centred crop).
__device__ __forceinline__ float ref_px(const uint8_t* img, int W, int s, int x0, int y0, int Wl, int Hl, int x,
                                        int y) {
    if (s > 0) return level_px(img, W, Wl, Hl, s, x, y);
    return __fmaf_rn((float)img[(size_t)(y0 + y) * W + (x0 + x)], 1.0f / 255.0f, -0.5f);
}

// Matching image of a level in "quad" layout: one bilinear sample is one
// 16-byte gather (8 bytes with FP16 storage).  FP32 entry (x, y) holds
// I(x, y), I(x+1, y) - I(x, y), I(x, y+1), I(x+1, y+1) - I(x, y+1) (centred
// intensities), so the sample needs no horizontal differences; the FP16
// entry holds the four intensities themselves (a difference of two halves
// is not always a half), and the sample forms the differences in FP32.
__device__ __forceinline__ void quad_px(const uint8_t* img, int W, int s, int Wl, int Hl, void* out, int half, int x,
                                        int y) {
    float4 q;
    q.x = level_px(img, W, Wl, Hl, s, x, y);
    q.y = level_px(img, W, Wl, Hl, s, x + 1, y);
    q.z = level_px(img, W, Wl, Hl, s, x, y + 1);
    q.w = level_px(img, W, Wl, Hl, s, x + 1, y + 1);
    if (half) {  // FP16 storage: four halves in 8 bytes
        __half2 a = __floats2half2_rn(q.x, q.y), b = __floats2half2_rn(q.z, q.w);
        static_cast<uint2*>(out)[(size_t)y * Wl + x] =
            make_uint2(*reinterpret_cast<unsigned*>(&a), *reinterpret_cast<unsigned*>(&b));
    } else {
        static_cast<float4*>(out)[(size_t)y * Wl + x] = make_float4(q.x, q.y - q.x, q.z, q.w - q.z);
    }
}

// Mean and sum of squared deviations of the window of radius rho centred on
// base[0] (row stride `stride`), by the two-pass direct sums.  (Unrolling
// the loops per radius took the prep launch from 32 to 95 registers and
// from 82% to 23% occupancy: 57.8 against 32.6 us per frame.)
__device__ __forceinline__ float2 window_stats(const float* base, int stride, int rho) {
    float s = 0.f;
    for (int dy = -rho; dy <= rho; ++dy)
        for (int dx = -rho; dx <= rho; ++dx) s += base[dy * stride + dx];
    float m = s / (float)((2 * rho + 1) * (2 * rho + 1));
    float v = 0.f;
    for (int dy = -rho; dy <= rho; ++dy)
        for (int dx = -rho; dx <= rho; ++dx) {
            float e = base[dy * stride + dx] - m;
            v = fmaf(e, e, v);
        }
    return make_float2(m, v);
}

// Mean and sum of squared deviations of the reference window around level
// pixel (x, y); var = -1 where the window leaves the image.  Computed once
// per frame, read by the sweep for every plane.
__device__ __forceinline__ float2 stats_px(const float* ref, int W, int H, int rho, int x, int y) {
    if (x >= rho && y >= rho && x < W - rho && y < H - rho) return window_stats(ref + (size_t)y * W + x, W, rho);
    return make_float2(0.f, -1.f);
}

// ------------------------------------------------------------- sweep

// Reciprocal and reciprocal square root as the single approximate PTX
// instructions with subnormals flushed (rcp.approx.ftz, rsqrt.approx.ftz).
// Their operands here (squared norms of points in metres, the unified
// model's denominator, window variances above N 1e-8) are never subnormal,
// where the non-flushing forms would add a rescaling sequence per call.
__device__ __forceinline__ float rcp_ftz(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Bilinear sample of a matching camera at pixel (u, v), as a centred
// intensity; NaN when `ok` is false (the point does not project) or (u, v)
// lies outside [0, W-1] x [0, H-1].  The gather is clamped into the image and
// always issued, so the warp does not diverge; a clamp that moved the point
// marks it outside (NaN compares unequal, so a NaN position is rejected
// too).  An invalid sample also sets `bad` (the caller's flag for the tile's
// invalid-sample path), from the same predicate: testing the returned value
// for NaN instead cost 3 % of the sweep kernel's time.  HALF: quads stored
// as FP16.
template <bool HALF>
__device__ __forceinline__ float sample_at(const CamS& c, float u, float v, bool ok, int& bad) {
    float uc = fminf(fmaxf(u, 0.0f), c.wm1), vc = fminf(fmaxf(v, 0.0f), c.hm1);
    ok = ok && (uc == u) && (vc == v);
    int x0 = (int)uc, y0 = (int)vc;
    if (!PS_DCHECK(x0 >= 0 && x0 < c.width && y0 >= 0 && (float)y0 <= c.hm1, CHK_GATHER)) {
        x0 = 0;
        y0 = 0;
        ok = false;
    }
    float ax = uc - (float)x0, ay = vc - (float)y0;
    float4 q;
    if (HALF) {
        uint2 h = __ldg(static_cast<const uint2*>(c.quad) + y0 * c.width + x0);
        float2 a = __half22float2(*reinterpret_cast<const __half2*>(&h.x));
        float2 b = __half22float2(*reinterpret_cast<const __half2*>(&h.y));
        q = make_float4(a.x, a.y - a.x, b.x, b.y - b.x);
    } else {
        q = __ldg(static_cast<const float4*>(c.quad) + y0 * c.width + x0);  // differences stored
    }
    float top = fmaf(ax, q.y, q.x);
    float bot = fmaf(ax, q.w, q.z);
    float w = fmaf(ay, bot - top, top);
    bad |= ok ? 0 : 1;
    return ok ? w : __int_as_float(0x7fc00000);
}

// The sample of a matching camera at the projection of X_j (camera frame):
// unified model, then radial-tangential distortion; NaN (and `bad` set) when
// the point does not project (sphere side, distortion range) or lands
// outside the image.
template <bool HALF>
__device__ __forceinline__ float warp_sample(const CamS& c, float X, float Y, float Z, int& bad) {
    float n2 = fmaf(X, X, fmaf(Y, Y, Z * Z));
    float n = n2 * rsqrt_ftz(n2);
    float inv = rcp_ftz(fmaf(c.xi, n, Z));
    float mx = X * inv, my = Y * inv;
    float r2 = fmaf(mx, mx, my * my);
    float rad = fmaf(r2, fmaf(c.k2, r2, c.k1), 1.0f);
    float mxy = mx * my;
    float xd = fmaf(mx, rad, fmaf(2.0f * c.p1, mxy, c.p2 * fmaf(2.0f * mx, mx, r2)));
    float yd = fmaf(my, rad, fmaf(c.p1, fmaf(2.0f * my, my, r2), 2.0f * c.p2 * mxy));
    float u = fmaf(c.fx, xd, c.cx);
    float v = fmaf(c.fy, yd, c.cy);
    return sample_at<HALF>(c, u, v, (Z > c.lim * n) && (r2 <= c.r2_max), bad);
}

// warp_sample for two points at once (lane x: the first plane, lane y: the
// second).  The projection runs on packed FP32 pairs; per lane every
// operation and its rounding are those of warp_sample (2 m = m + m exactly),
// so each result is bit-identical to a warp_sample call.
template <bool HALF>
__device__ __forceinline__ float2 warp_sample2(const CamS& c, float2 X, float2 Y, float2 Z, int& bad) {
    float2 n2 = fma2(X, X, fma2(Y, Y, mul2(Z, Z)));
    float2 n = mul2(n2, make_float2(rsqrt_ftz(n2.x), rsqrt_ftz(n2.y)));
    float2 den = fma2(c.xi2, n, Z);
    float2 inv = make_float2(rcp_ftz(den.x), rcp_ftz(den.y));
    float2 mx = mul2(X, inv), my = mul2(Y, inv);
    float2 r2 = fma2(mx, mx, mul2(my, my));
    float2 rad = fma2(r2, fma2(c.k22, r2, c.k12), dup2(1.0f));
    float2 mxy = mul2(mx, my);
    float2 xd = fma2(mx, rad, fma2(c.p1x2, mxy, mul2(c.p22, fma2(add2(mx, mx), mx, r2))));
    float2 yd = fma2(my, rad, fma2(c.p12, fma2(add2(my, my), my, r2), mul2(c.p2x2, mxy)));
    float2 u = fma2(c.fx2, xd, c.cx2), v = fma2(c.fy2, yd, c.cy2);
    float2 ln = mul2(c.lim2, n);
    return make_float2(sample_at<HALF>(c, u.x, v.x, (Z.x > ln.x) && (r2.x <= c.r2_max), bad),
                       sample_at<HALF>(c, u.y, v.y, (Z.y > ln.y) && (r2.y <= c.r2_max), bad));
}

// Winner-take-all state in tensor memory.  Each output-owning thread keeps
// the state of its SEG pixels (best and second-best cost, the costs of the
// previous, first and winner's neighbouring planes, the winner and whether
// the next plane's cost is owed) in 8 SEG words of TMEM between plane pairs,
// not in registers: the registers go to the warp instead.  A warp reaches
// the TMEM lanes of its quadrant (warp id mod 4); the warps of a quadrant
// take 32 columns each (warps that own no pixels hold an unused copy).  The CTA allocates TMEM_COLS
// columns once (tm_alloc) and frees them before it exits (tm_free).
// The same lanes also hold each thread's direction tables (see sweep_tile):
// TM_TAB + 9 j holds, for matching camera j, the three coordinates of the
// direction of each of the thread's (at most 3) halo positions.
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t TM_WARP_COLS = 80;  // columns of one warp: state, then tables
constexpr uint32_t TM_TAB = 32;        // first table column of a warp
static_assert((NT / 32 + 3) / 4 * TM_WARP_COLS <= TMEM_COLS, "TMEM columns of every warp");
static_assert(TM_TAB + 9 * PS_MAX_CAMS <= TM_WARP_COLS, "state and tables of every camera fit a warp's columns");

__device__ __forceinline__ uint32_t tm_addr(uint32_t base) {
    const uint32_t w = threadIdx.x >> 5;
    return base + (((w & 3u) * 32u) << 16) + (w >> 2) * TM_WARP_COLS;
}

// 9 words at TMEM address a (warp-collective; waits for the thread's earlier
// stores first and for the load's completion).
__device__ __forceinline__ void tm_ld9(uint32_t a, float (&v)[9]) {
    uint32_t r[9];
    asm volatile(
        "tcgen05.wait::st.sync.aligned;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%9];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%8}, [%10];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8])
        : "r"(a), "r"(a + 8u)
        : "memory");
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tm_st9(uint32_t a, const float (&v)[9]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x1.b32 [%1], {%10};" ::"r"(a),
        "r"(a + 8u), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])),
        "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8]))
        : "memory");
}

// Warp 0 allocates the CTA's columns and writes their address to *slot;
// every thread reads it after the barrier.
__device__ __forceinline__ uint32_t tm_alloc(uint32_t* slot) {
    if (threadIdx.x < 32)
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n\t"
            "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::"r"((uint32_t)__cvta_generic_to_shared(slot)),
            "n"(TMEM_COLS)
            : "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return *slot;
}

// Every thread's TMEM stores have completed; warp 0 frees the columns.
__device__ __forceinline__ void tm_free(uint32_t base) {
    asm volatile("tcgen05.wait::st.sync.aligned;\n\ttcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "n"(TMEM_COLS) : "memory");
}

// 32 words of this thread's TMEM lane (warp-collective).  The load waits for
// the thread's earlier stores and for its own completion.
__device__ __forceinline__ void tm_ld32(uint32_t a, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.wait::st.sync.aligned;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                 "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                 "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(a)
        : "memory");
}
__device__ __forceinline__ void tm_st32(uint32_t a, const uint32_t (&r)[32]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(a),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                 "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
                 "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
                 "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
                 : "memory");
}

// The state arrays of SEG pixels, packed 8 words per pixel.
#define PS_WTA_ARGS(Q) Q float (&c1)[SEG], Q float (&c2)[SEG], Q float (&cprev)[SEG], Q float (&cminus)[SEG], \
    Q float (&cplus)[SEG], Q float (&cfirst)[SEG], Q int (&kb)[SEG], Q bool (&needp)[SEG]
// 24 words (x16 + x8) of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tm_ld24(uint32_t a, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.wait::st.sync.aligned;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%25];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(a), "r"(a + 16u)
        : "memory");
}
__device__ __forceinline__ void tm_st24(uint32_t a, const uint32_t (&r)[32]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17};\n\t"
                 "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%18, %19, %20, %21, %22, %23, %24, %25};" ::"r"(a), "r"(a + 16u),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                 "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
                 "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23])
                 : "memory");
}

template <int SEG>
__device__ __forceinline__ void wta_load(uint32_t a, PS_WTA_ARGS()) {
    static_assert(8 * SEG <= 32, "the state of SEG pixels fits 32 words");
    uint32_t r[32];
    if constexpr (SEG == 3) tm_ld24(a, r); else tm_ld32(a, r);
#pragma unroll
    for (int i = 0; i < SEG; ++i) {
        c1[i] = __uint_as_float(r[8 * i]);
        c2[i] = __uint_as_float(r[8 * i + 1]);
        cprev[i] = __uint_as_float(r[8 * i + 2]);
        cminus[i] = __uint_as_float(r[8 * i + 3]);
        cplus[i] = __uint_as_float(r[8 * i + 4]);
        cfirst[i] = __uint_as_float(r[8 * i + 5]);
        kb[i] = (int)r[8 * i + 6];
        needp[i] = r[8 * i + 7] != 0u;
    }
}
template <int SEG>
__device__ __forceinline__ void wta_store(uint32_t a, PS_WTA_ARGS(const)) {
    uint32_t r[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) r[i] = 0u;
#pragma unroll
    for (int i = 0; i < SEG; ++i) {
        r[8 * i] = __float_as_uint(c1[i]);
        r[8 * i + 1] = __float_as_uint(c2[i]);
        r[8 * i + 2] = __float_as_uint(cprev[i]);
        r[8 * i + 3] = __float_as_uint(cminus[i]);
        r[8 * i + 4] = __float_as_uint(cplus[i]);
        r[8 * i + 5] = __float_as_uint(cfirst[i]);
        r[8 * i + 6] = (uint32_t)kb[i];
        r[8 * i + 7] = needp[i] ? 1u : 0u;
    }
    if constexpr (SEG == 3) tm_st24(a, r); else tm_st32(a, r);
}
#undef PS_WTA_ARGS

// Tile geometry.  A CTA owns TW x TH output pixels of one level plus a halo of
// RHO on every side (HH rows x HWL columns of warped samples per plane and
// camera).  Per plane set, every halo position keeps, per matching camera,
// a = R_j r / (n . r), so that the plane at offset d maps it to d a + t_j
// (in the TMEM lane of the thread that warps the position).
// Phase A: every thread warps PPT halo positions into W.  Phase H: thread
// (row, run) slides a 2 RHO + 1 window along RUN outputs of one halo row and
// stores (sum w, sum w^2, sum r w, invalid count) in H.  Phase V: thread
// (column, segment) slides down SEG output rows, forms ZNCC and keeps the
// minimum over cameras.  Strides make every phase's shared-memory accesses
// free of bank conflicts.  KP planes are warped per camera before the
// window sums, so consecutive gathers hit overlapping footprints of the same
// image; with KP = 2 the three phases handle both planes at once on packed
// FP32 pairs (pair_pass) and H holds both planes' sums.
template <int RHO, int TH, int KP>
struct Geo {
    static constexpr int SEG = TH / 8;                // output rows per vertical segment (phase V)
    static constexpr int HH = TH + 2 * RHO;           // halo rows (<= 32)
    static constexpr int HWL = TW + 2 * RHO;          // halo columns
    static constexpr int WS = 76;                     // W / R row stride (floats): 76 = 12 mod 32
    static constexpr int HS = TW + 1;                 // H row stride (float4): odd
    static constexpr int NPOS = HH * HWL;
    static constexpr int PPT = (NPOS + NT - 1) / NT;
    static constexpr int NRUNPOS = RUN + 2 * RHO;     // positions one horizontal run reads
    static constexpr int NV = (NRUNPOS + 3) / 4;      // float4 loads per run
    static constexpr int N = (2 * RHO + 1) * (2 * RHO + 1);
    // two planes per pass: W holds (plane 0, plane 1) pairs with a row stride
    // of 74 pairs (148 = 20 mod 32 words, so the 16-byte loads of the lanes
    // of phase H, one halo row each, hit distinct bank groups)
    static constexpr int WS2 = 74;
    static constexpr int NV2 = (NRUNPOS + 1) / 2;     // 16-byte loads (two pairs) per run
    // With two planes per pass, two matching cameras go through each step
    // (CG = 2): W and H hold both cameras' samples and sums.
    static constexpr int CG = KP == 2 ? 2 : 1;
    static constexpr int WSZ = KP == 2 ? 2 * HH * WS2 : HH * WS;  // floats of one camera's W
    // KP = 2: one camera's H is [HH][HS] float4 (sw0, sw1, sww0, sww1) and
    // [HH][HS] float2 (srw0, srw1): HCAM4 float4s; the invalid-sample flags
    // of a step with invalid samples are bytes F [CG][HH][TW] (bit q: some
    // sample of plane q's horizontal window is invalid).  KP = 1: KP x
    // [HH][HS] float4 (sw, sww, srw, invalid count).
    static constexpr int HCAM4 = HH * HS * 3 / 2;
    static constexpr int HREG4 = KP == 2 ? CG * HCAM4 : KP * HH * HS;
    static constexpr int FSZ = KP == 2 ? CG * HH * TW : 0;
    // H, CG W buffers, R and the flags (the direction tables are in TMEM)
    static constexpr int DTAB = 64;  // plane offsets of a work item staged in shared memory
    static constexpr size_t smem(int) {
        return sizeof(float4) * HREG4 + sizeof(float) * (CG * WSZ + HH * WS) + FSZ + sizeof(float) * DTAB;
    }
    static_assert(HH % 2 == 0, "a camera's H blocks stay 16-byte aligned");
    static_assert(PPT <= 3, "three directions per thread and camera in TMEM");
    static_assert(NTV == TW * (TH / SEG) && TH % 8 == 0 && NTV <= NT, "phase V: one thread per column and row segment");
    static_assert(KP == 1 || KP == 2, "one or two planes per pass");
    static_assert(HH <= 32, "phase H maps one warp lane per halo row");
    static_assert(HWL <= WS && 4 * NV + TW - RUN <= WS, "row stride covers the runs' loads");
    static_assert(HWL <= WS2 && 2 * NV2 + TW - RUN <= WS2, "pair row stride covers the runs' loads");
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Phases A, H and V of one matching camera for two planes at once (planes
// at offsets d0 and d1 of the current set), on packed FP32 pairs: lane x is
// the first plane, lane y the second.  Per lane every sum and every rounding
// is that of the one-plane path, so the costs are bit-identical to it.
// W2 holds (plane 0, plane 1) sample pairs; H holds, per halo row and output
// column, (sw0, sw1, sww0, sww1) in the first buffer and (srw0, srw1, m0, m1)
// in the second (m: invalid samples in the run).  cmin0 / cmin1 hold the
// running minimum over cameras of the two planes' costs.  Each phase is a
// function of its task (halo position, halo row run, output column segment)
// alone, so any thread-to-task mapping gives the same results.

// Phase A: warped sample pairs at halo positions p = t0 + i STRIDE, whose
// directions are av[3 i .. 3 i + 2]; returns whether any of this thread's
// samples is invalid.
template <int RHO, bool HALF, int TH, int STRIDE>
__device__ __forceinline__ int pair_phase_a(const CamS& C, const float (&av)[9], float d0, float d1, float2* W2, int t0) {
    using G = Geo<RHO, TH, 2>;
    constexpr int HWL = G::HWL, WS2 = G::WS2, NPOS = G::NPOS;
    constexpr int NP = (NPOS + STRIDE - 1) / STRIDE;
    static_assert(NP <= 3, "three directions per thread and camera");
    int bad = 0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        int p = t0 + i * STRIDE;
        if (p < NPOS) {
            const float4 a = make_float4(av[3 * i], av[3 * i + 1], av[3 * i + 2], 0.f);
            float2 w = warp_sample2<HALF>(C, make_float2(fmaf(d0, a.x, C.t[0]), fmaf(d1, a.x, C.t[0])),
                                          make_float2(fmaf(d0, a.y, C.t[1]), fmaf(d1, a.y, C.t[1])),
                                          make_float2(fmaf(d0, a.z, C.t[2]), fmaf(d1, a.z, C.t[2])), bad);
            int hy = p / HWL, hx = p - hy * HWL;
            W2[hy * WS2 + hx] = w;
        }
    }
    return bad;
}

// Phase H: sliding horizontal sums of both planes along run `hrun` of halo
// row `hrow` (bad: some sample of the tile is invalid), for NC cameras
// (camera c's samples at W2 + c WSZ / 2, its sums at Hs + c HCAM4 and, when
// bad, its flags at Fs + c HH TW); the reference samples of the run are
// loaded once.
template <int RHO, int TH, int NC = 1>
__device__ __forceinline__ void pair_phase_h(const float2* W2, const float* Rs, float4* Hs, unsigned char* Fs,
                                             int hrow, int hrun, int bad) {
    using G = Geo<RHO, TH, 2>;
    constexpr int HH = G::HH, WS = G::WS, WS2 = G::WS2, HS = G::HS;
    // phase H: sliding horizontal sums of both planes along a run of one halo row
    if (hrow < HH && hrun < TW / RUN) {
        const float* rr = Rs + hrow * WS + RUN * hrun;
        float r[4 * G::NV];
#pragma unroll
        for (int qq = 0; qq < G::NV; ++qq) {
            float4 b = *reinterpret_cast<const float4*>(rr + 4 * qq);
            r[4 * qq] = b.x; r[4 * qq + 1] = b.y; r[4 * qq + 2] = b.z; r[4 * qq + 3] = b.w;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const float2* wr = W2 + c * (G::WSZ / 2) + hrow * WS2 + RUN * hrun;
            float2 w[2 * G::NV2];
#pragma unroll
            for (int qq = 0; qq < G::NV2; ++qq) {
                float4 a = *reinterpret_cast<const float4*>(wr + 2 * qq);
                w[2 * qq] = make_float2(a.x, a.y);
                w[2 * qq + 1] = make_float2(a.z, a.w);
            }
            float4* ha = Hs + c * G::HCAM4 + hrow * HS + RUN * hrun;
            float2* hb = reinterpret_cast<float2*>(Hs + c * G::HCAM4 + HH * HS) + hrow * HS + RUN * hrun;
            unsigned char* fl = Fs + c * HH * TW + hrow * TW + RUN * hrun;
            float2 sw = dup2(0.f), sww = dup2(0.f), srw = dup2(0.f), sm = dup2(0.f);
            if (!bad) {  // every sample of the tile is valid (the common case)
#pragma unroll
                for (int t = 0; t <= 2 * RHO; ++t) {
                    sw = add2(sw, w[t]);
                    sww = fma2(w[t], w[t], sww);
                    srw = fma2(dup2(r[t]), w[t], srw);
                }
                ha[0] = make_float4(sw.x, sw.y, sww.x, sww.y);
                hb[0] = srw;
#pragma unroll
                for (int o = 1; o < RUN; ++o) {
                    const int a = o + 2 * RHO, b = o - 1;
                    sw = add2(sw, add2(w[a], neg2(w[b])));
                    sww = add2(sww, fma2(w[a], w[a], mul2(neg2(w[b]), w[b])));
                    srw = add2(srw, fma2(dup2(r[a]), w[a], mul2(dup2(-r[b]), w[b])));
                    ha[o] = make_float4(sw.x, sw.y, sww.x, sww.y);
                    hb[o] = srw;
                }
            } else {  // invalid samples: excluded from the sums and counted
#pragma unroll
                for (int t = 0; t <= 2 * RHO; ++t) {
                    const bool bx = isnan(w[t].x), by = isnan(w[t].y);
                    const float2 wt = make_float2(bx ? 0.0f : w[t].x, by ? 0.0f : w[t].y);
                    sw = add2(sw, wt);
                    sww = fma2(wt, wt, sww);
                    srw = fma2(dup2(r[t]), wt, srw);
                    sm = add2(sm, make_float2(bx ? 1.0f : 0.0f, by ? 1.0f : 0.0f));
                }
                ha[0] = make_float4(sw.x, sw.y, sww.x, sww.y);
                hb[0] = srw;
                fl[0] = (unsigned char)((sm.x != 0.0f ? 1 : 0) | (sm.y != 0.0f ? 2 : 0));
#pragma unroll
                for (int o = 1; o < RUN; ++o) {
                    const int a = o + 2 * RHO, b = o - 1;
                    const bool ax = isnan(w[a].x), ay = isnan(w[a].y), bx = isnan(w[b].x), by = isnan(w[b].y);
                    const float2 wa = make_float2(ax ? 0.0f : w[a].x, ay ? 0.0f : w[a].y);
                    const float2 wb = make_float2(bx ? 0.0f : w[b].x, by ? 0.0f : w[b].y);
                    sw = add2(sw, add2(wa, neg2(wb)));
                    sww = add2(sww, fma2(wa, wa, mul2(neg2(wb), wb)));
                    srw = add2(srw, fma2(dup2(r[a]), wa, mul2(dup2(-r[b]), wb)));
                    sm = add2(sm, add2(make_float2(ax ? 1.0f : 0.0f, ay ? 1.0f : 0.0f),
                                       neg2(make_float2(bx ? 1.0f : 0.0f, by ? 1.0f : 0.0f))));
                    ha[o] = make_float4(sw.x, sw.y, sww.x, sww.y);
                    hb[o] = srw;
                    fl[o] = (unsigned char)((sm.x != 0.0f ? 1 : 0) | (sm.y != 0.0f ? 2 : 0));
                }
            }
        }
    }
}

// Phase V: sliding vertical sums of both planes down the SEG rows of one
// output column segment (base_v: its first H entry), ZNCC against the
// reference statistics st, and the minimum over cameras.
template <int RHO, int TH, bool BAD>
__device__ __forceinline__ void pair_phase_v_(const float4* Hs, const unsigned char* Fs,
                                              const float2 (&st)[TH / 8], int base_v, int base_f,
                                              float (&cmin0)[TH / 8], float (&cmin1)[TH / 8]) {
    constexpr bool bad = BAD;
    using G = Geo<RHO, TH, 2>;
    constexpr int SEG = G::SEG, HH = G::HH, HS = G::HS, N = G::N;
    const float4* Ha = Hs;
    const float2* Hb = reinterpret_cast<const float2*>(Hs + HH * HS);
    // phase V: sliding vertical sums of both planes down SEG rows, ZNCC, minimum over cameras;
    // when some sample of the tile is invalid, f0 / f1 count the flagged rows of the window
    float2 vs = dup2(0.f), vss = dup2(0.f), vrs = dup2(0.f);
    int f0 = 0, f1 = 0;
#pragma unroll
    for (int dy = 0; dy <= 2 * RHO; ++dy) {
        const float4 a = Ha[base_v + dy * HS];
        const float2 b = Hb[base_v + dy * HS];
        vs = add2(vs, make_float2(a.x, a.y));
        vss = add2(vss, make_float2(a.z, a.w));
        vrs = add2(vrs, b);
        if (bad) {
            const int f = Fs[base_f + dy * TW];
            f0 += f & 1;
            f1 += f >> 1;
        }
    }
#pragma unroll
    for (int i = 0; i < SEG; ++i) {
        if (i > 0) {
            const float4 a = Ha[base_v + (i + 2 * RHO) * HS], c = Ha[base_v + (i - 1) * HS];
            const float2 b = Hb[base_v + (i + 2 * RHO) * HS], d = Hb[base_v + (i - 1) * HS];
            vs = add2(vs, add2(make_float2(a.x, a.y), make_float2(-c.x, -c.y)));
            vss = add2(vss, add2(make_float2(a.z, a.w), make_float2(-c.z, -c.w)));
            vrs = add2(vrs, add2(b, neg2(d)));
            if (bad) {
                const int fa = Fs[base_f + (i + 2 * RHO) * TW], fc = Fs[base_f + (i - 1) * TW];
                f0 += (fa & 1) - (fc & 1);
                f1 += (fa >> 1) - (fc >> 1);
            }
        }
        const float2 var_w = fma2(mul2(neg2(vs), dup2(1.0f / (float)N)), vs, vss);
        const float2 cov = fma2(dup2(-st[i].x), vs, vrs);
        const float2 zr = mul2(mul2(cov, dup2(st[i].y)), make_float2(rsqrt_ftz(var_w.x), rsqrt_ftz(var_w.y)));
        // cost = (1 - z) / 2 with |ZNCC| <= 1: saturating the FMA to [0, 1] gives
        // exactly the values of clamping z to [-1, 1] first (the ends map to
        // 0.5 -+ 0.5 exactly), in one instruction per plane
        const float2 cost = make_float2(__saturatef(__fmaf_rn(-0.5f, zr.x, 0.5f)),
                                        __saturatef(__fmaf_rn(-0.5f, zr.y, 0.5f)));
        const bool ref_ok = !isnan(st[i].y);
        const bool ok0 = (!BAD || f0 == 0) && var_w.x >= (float)N * 1e-8f && ref_ok;
        const bool ok1 = (!BAD || f1 == 0) && var_w.y >= (float)N * 1e-8f && ref_ok;
        cmin0[i] = ok0 ? fminf(cmin0[i], cost.x) : cmin0[i];
        cmin1[i] = ok1 ? fminf(cmin1[i], cost.y) : cmin1[i];
    }
}
// (the tile's invalid-sample flag is uniform: two code paths, the common one
// without the flag counts)
template <int RHO, int TH>
__device__ __forceinline__ void pair_phase_v(const float4* Hs, const unsigned char* Fs, int bad,
                                             const float2 (&st)[TH / 8], int base_v, int base_f,
                                             float (&cmin0)[TH / 8], float (&cmin1)[TH / 8]) {
    if (bad)
        pair_phase_v_<RHO, TH, true>(Hs, Fs, st, base_v, base_f, cmin0, cmin1);
    else
        pair_phase_v_<RHO, TH, false>(Hs, Fs, st, base_v, base_f, cmin0, cmin1);
}

template <int RHO, bool HALF, int TH>
__device__ __forceinline__ void pair_pass(const CamS& C, const float (&av)[9], float d0, float d1, float2* W2,
                                          const float* Rs, float4* Hs, unsigned char* Fs, const float2 (&st)[TH / 8],
                                          int base_v, int base_f, float (&cmin0)[TH / 8], float (&cmin1)[TH / 8]) {
    const int tid = threadIdx.x;
    int bad = pair_phase_a<RHO, HALF, TH, NT>(C, av, d0, d1, W2, tid);
    bad = __syncthreads_or(bad);
    using G = Geo<RHO, TH, 2>;
    const int hrow = tid & 31, hrun = tid >> 5;
    if (hrow < G::HH && hrun < TW / RUN) pair_phase_h<RHO, TH>(W2, Rs, Hs, Fs, hrow, hrun, bad);
    __syncthreads();
    if (tid < NTV) pair_phase_v<RHO, TH>(Hs, Fs, bad, st, base_v, base_f, cmin0, cmin1);
}

// Two matching cameras in one step (the second camera's samples and sums in
// the second W and H buffers): one pair of barriers for both.  Each phase
// computes what it computes for one camera, and the invalid-sample flag is
// shared (the flagged path gives valid samples the same sums), so the costs
// are those of two one-camera steps.
// Phase A of a two-camera step: the first camera's sample pairs at the
// thread's halo positions, then the second's, into W2 and W2b (measured
// faster than interleaving the cameras per position since the compiler
// issues flush-to-zero reciprocals: street 0.766 against 0.770 ms).  The
// second camera's directions (TMEM address tab1) are loaded only when its
// warp starts, so they hold no registers during the first camera's
// (0.759 against 0.766 ms).
template <int RHO, bool HALF, int TH>
__device__ __forceinline__ int pair_phase_a2(const CamS& C0, const CamS& C1, const float (&av0)[9], uint32_t tab1,
                                             float d0, float d1, float2* W2, float2* W2b, int t0) {
    using G = Geo<RHO, TH, 2>;
    constexpr int HWL = G::HWL, WS2 = G::WS2, NPOS = G::NPOS;
    constexpr int NP = (NPOS + NT - 1) / NT;
    int bad = 0;
    float av1[9];  // the second camera's directions, loaded once the first camera's warp is done
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (c == 1) tm_ld9(tab1, av1);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            int p = t0 + i * NT;
            if (p >= NPOS) continue;
            int hy = p / HWL, hx = p - hy * HWL;
            {
                const CamS& C = c ? C1 : C0;
                const float* av = c ? static_cast<const float*>(av1) : static_cast<const float*>(av0);
                const float4 a = make_float4(av[3 * i], av[3 * i + 1], av[3 * i + 2], 0.f);
                float2 w = warp_sample2<HALF>(C, make_float2(fmaf(d0, a.x, C.t[0]), fmaf(d1, a.x, C.t[0])),
                                              make_float2(fmaf(d0, a.y, C.t[1]), fmaf(d1, a.y, C.t[1])),
                                              make_float2(fmaf(d0, a.z, C.t[2]), fmaf(d1, a.z, C.t[2])), bad);
                (c ? W2b : W2)[hy * WS2 + hx] = w;
            }
        }
    }
    return bad;
}

template <int RHO, bool HALF, int TH>
__device__ __forceinline__ void pair_pass2(const CamS& C0, const CamS& C1, const float (&av0)[9], uint32_t tab1,
                                           float d0, float d1, float2* W2, const float* Rs, float4* Hs,
                                           unsigned char* Fs, const float2 (&st)[TH / 8], int base_v, int base_f,
                                           float (&cmin0)[TH / 8], float (&cmin1)[TH / 8]) {
    using G = Geo<RHO, TH, 2>;
    const int tid = threadIdx.x;
    float2* W2b = W2 + G::WSZ / 2;
    float4* Hsb = Hs + G::HCAM4;
    int bad = pair_phase_a2<RHO, HALF, TH>(C0, C1, av0, tab1, d0, d1, W2, W2b, tid);
    bad = __syncthreads_or(bad);
    const int hrow = tid & 31, hrun = tid >> 5;
    pair_phase_h<RHO, TH, 2>(W2, Rs, Hs, Fs, hrow, hrun, bad);
    __syncthreads();
    if (tid < NTV) {
        pair_phase_v<RHO, TH>(Hs, Fs, bad, st, base_v, base_f, cmin0, cmin1);
        pair_phase_v<RHO, TH>(Hsb, Fs + G::HH * TW, bad, st, base_v, base_f, cmin0, cmin1);
    }
}

// Parabola through the winner and its neighbours in the same plane set, and
// the range along the pixel's ray; writes the level outputs of one pixel.
__device__ inline void finish_pixel(const LevelD& L, int gx, int gy, float c1, float c2, int kb, float cminus, float cplus) {
    const float inf = __int_as_float(0x7f800000);
    size_t o = (size_t)gy * L.W + gx;
    float depth = 0.f;
    if (kb >= 0) {
        int s = 0;
        while (s + 1 < L.n_sets && L.sets[s + 1].start <= kb) ++s;
        const SetD S = L.sets[s];
        int li = kb - S.start;
        float delta = 0.f;
        if (li > 0 && li < S.count - 1 && cminus < inf && cplus < inf) {
            float den = cminus - 2.0f * c1 + cplus;
            if (den > 0.f) delta = fminf(0.5f, fmaxf(-0.5f, (cminus - cplus) / (2.0f * den)));
        }
        float t = S.count > 1 ? ((float)li + delta) / (float)(S.count - 1) : 0.f;
        float param = S.family == PS_PLANES_FRONTO ? 1.0f / fmaf(t, 1.0f / S.a - 1.0f / S.b, 1.0f / S.b)
                                                   : fmaf(t, S.b - S.a, S.a);
        float4 r = L.rays[o];
        float nr = S.nx * r.x + S.ny * r.y + S.nz * r.z;
        depth = param / nr;
    }
    if (L.depth) L.depth[o] = depth;
    if (L.c1) L.c1[o] = c1;
    if (L.c2) L.c2[o] = c2;
    if (L.kstar) L.kstar[o] = kb;
}

// Record of pixel (gx, gy) over the planes [k_begin, k_end) of this launch.
__device__ __forceinline__ void write_record(const LevelD& L, int gx, int gy, float c1, float c2, float cm, float cp,
                                             float first, float last, int kb) {
    const size_t n = (size_t)L.W * L.H, o = (size_t)gy * L.W + gx;
    L.records[REC_C1 * n + o] = c1;
    L.records[REC_C2 * n + o] = c2;
    L.records[REC_CM * n + o] = cm;
    L.records[REC_CP * n + o] = cp;
    L.records[REC_FIRST * n + o] = first;
    L.records[REC_LAST * n + o] = last;
    L.records[REC_K * n + o] = __int_as_float(kb);
}

// Winner-take-all of one pixel from the records of n_parts consecutive
// plane ranges (part p covers [lo[p], lo[p + 1]), the last one up to
// n_planes), then its outputs as finish_pixel writes them.  The same rule as
// the tile's merge of its plane chunks: the first part holding the lowest
// cost wins (ties keep the lowest plane), the second best is the minimum of
// the winner's second best and every other part's best, and a neighbour
// cost outside the winner's range comes from the adjacent part's first or
// last plane.
__device__ inline void merge_record_px(const LevelD& L, const float* const* rec, const int* lo, int n_parts, int gx,
                                       int gy) {
    const float inf = __int_as_float(0x7f800000);
    const size_t n = (size_t)L.W * L.H, o = (size_t)gy * L.W + gx;
    int wc = -1;
    float b1 = inf;
    for (int p = 0; p < n_parts; ++p) {
        const int hi = p + 1 < n_parts ? lo[p + 1] : L.n_planes;
        if (hi <= lo[p]) continue;  // empty part
        const float v = rec[p][REC_C1 * n + o];
        if (v < b1) {
            b1 = v;
            wc = p;
        }
    }
    float b2 = inf, cm = inf, cp = inf;
    int k = -1;
    if (wc >= 0) {
        b2 = rec[wc][REC_C2 * n + o];
        for (int p = 0; p < n_parts; ++p) {
            const int hi = p + 1 < n_parts ? lo[p + 1] : L.n_planes;
            if (p != wc && hi > lo[p]) b2 = fminf(b2, rec[p][REC_C1 * n + o]);
        }
        k = __float_as_int(rec[wc][REC_K * n + o]);
        const int whi = wc + 1 < n_parts ? lo[wc + 1] : L.n_planes;
        int prev = wc - 1, next = wc + 1;
        while (prev >= 0 && (prev + 1 < n_parts ? lo[prev + 1] : L.n_planes) <= lo[prev]) --prev;
        while (next < n_parts && (next + 1 < n_parts ? lo[next + 1] : L.n_planes) <= lo[next]) ++next;
        cm = k > lo[wc] ? rec[wc][REC_CM * n + o] : (prev >= 0 ? rec[prev][REC_LAST * n + o] : inf);
        cp = k < whi - 1 ? rec[wc][REC_CP * n + o] : (next < n_parts ? rec[next][REC_FIRST * n + o] : inf);
    }
    finish_pixel(L, gx, gy, b1, b2, k, cm, cp);
}

// End of a work item.  When the item completed its tile and the level counts
// finished tiles (batched launch), the tile's outputs are made visible to the
// whole GPU before the count moves.  `finished` is uniform over the CTA.
__device__ __forceinline__ void tile_finished(const LevelD& L, bool finished) {
    if (L.tiles_done != nullptr && finished) {
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(L.tiles_done, 1);
    } else {
        __syncthreads();
    }
}

// End of a work item whose tile has several plane chunks (its chunk record
// is written): count it, and when it completes the tile, merge the chunks'
// records in plane order into the tile's outputs (or records).
template <int TH>
__device__ inline void merge_chunks(const LevelD& L, int tile, int* s_flag) {
    constexpr int SEG = TH / 8;
    const int tid = threadIdx.x;
    const int tx = tile % L.tiles_x, ty = tile / L.tiles_x;
    const int ox = tid % TW, oy0 = (tid / TW) * SEG;
    const float inf = __int_as_float(0x7f800000);
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const int prev = atomicAdd(&L.done[tile], 1);
        *s_flag = prev == L.n_chunks - 1;
        // more completions than chunks: the counters were not this call's alone
        if (prev >= L.n_chunks && L.status) atomicOr(L.status, DEV_STATE);
    }
    __syncthreads();
    if (*s_flag && tid < NTV) {
        __threadfence();
        const float* base = L.partial + (size_t)tile * L.n_chunks * 7 * (TH * TW);
#pragma unroll 1
        for (int i = 0; i < SEG; ++i) {
            const int gx = tx * TW + ox, gy = ty * TH + oy0 + i;
            const int px = (oy0 + i) * TW + ox;
            // global winner (first chunk holding the lowest cost: ties keep the lowest plane)
            int wc = -1;
            float b1 = inf;
            for (int c = 0; c < L.n_chunks; ++c) {
                float v = __ldcg(base + ((size_t)c * 7 + 0) * (TH * TW) + px);
                if (v < b1) {
                    b1 = v;
                    wc = c;
                }
            }
            float b2 = inf, cm = inf, cp = inf;
            int k = -1;
            if (wc >= 0) {
                const float* P = base + (size_t)wc * 7 * (TH * TW) + px;
                b2 = __ldcg(P + 1 * (TH * TW));
                for (int c = 0; c < L.n_chunks; ++c)
                    if (c != wc) b2 = fminf(b2, __ldcg(base + ((size_t)c * 7 + 0) * (TH * TW) + px));
                k = __float_as_int(__ldcg(P + 6 * (TH * TW)));
                const int lo = L.k_begin + wc * L.chunk, hi = min(L.k_end, lo + L.chunk);
                cm = k > lo ? __ldcg(P + 2 * (TH * TW))
                            : (wc > 0 ? __ldcg(base + ((size_t)(wc - 1) * 7 + 5) * (TH * TW) + px) : inf);
                cp = k < hi - 1 ? __ldcg(P + 3 * (TH * TW))
                                : (wc + 1 < L.n_chunks ? __ldcg(base + ((size_t)(wc + 1) * 7 + 4) * (TH * TW) + px)
                                                       : inf);
            }
            if (gx < L.W && gy < L.H) {
                if (L.records) {
                    const float first = __ldcg(base + 4 * (TH * TW) + px);
                    const float last = __ldcg(base + ((size_t)(L.n_chunks - 1) * 7 + 5) * (TH * TW) + px);
                    write_record(L, gx, gy, b1, b2, cm, cp, first, last, k);
                } else {
                    finish_pixel(L, gx, gy, b1, b2, k, cm, cp);
                }
            }
        }
    }
    tile_finished(L, *s_flag != 0);
}

template <int RHO, bool HALF, int TH, int KP>
__device__ inline void sweep_tile(const LevelD& L, const CamS* cams, int item, unsigned char* smem_raw, int* s_flag,
                                  uint32_t tmem) {
    using G = Geo<RHO, TH, KP>;
    constexpr int SEG = G::SEG;
    if (!PS_DCHECK(item >= 0 && item < L.n_items, CHK_ITEM)) return;  // uniform over the CTA
    const int tile = item / L.n_chunks, chunk = item - tile * L.n_chunks;
    const int k_lo = L.k_begin + chunk * L.chunk, k_hi = min(L.k_end, k_lo + L.chunk);
    constexpr int HH = G::HH, HWL = G::HWL, WS = G::WS, HS = G::HS, NPOS = G::NPOS, N = G::N;
    float4* Hs = reinterpret_cast<float4*>(smem_raw);            // window sums (layout: Geo)
    float* Ws = reinterpret_cast<float*>(Hs + G::HREG4);          // [CG] warped samples (NaN = invalid): KP = 1
    float2* W2 = reinterpret_cast<float2*>(Ws);                   //   [HH][WS], KP = 2 [HH][WS2] pairs (k0, k0 + 1)
    float* Rs = Ws + G::CG * G::WSZ;                              // [HH][WS] reference intensities
    unsigned char* Fs = reinterpret_cast<unsigned char*>(Rs + HH * WS);  // KP = 2: invalid-sample flags
    float* Ds = reinterpret_cast<float*>(Fs + G::FSZ);                   // plane offsets d of the item's planes
    const int tid = threadIdx.x;
    const int tx = tile % L.tiles_x, ty = tile / L.tiles_x;
    const int gx0 = tx * TW - RHO, gy0 = ty * TH - RHO;
    const float nan = __int_as_float(0x7fc00000);
    const float inf = __int_as_float(0x7f800000);

    for (int p = tid; p < NPOS; p += NT) {
        int hy = p / HWL, hx = p - hy * HWL;
        int gx = gx0 + hx, gy = gy0 + hy;
        bool in = gx >= 0 && gy >= 0 && gx < L.W && gy < L.H;
        Rs[hy * WS + hx] = in ? L.ref[(size_t)gy * L.W + gx] : 0.0f;
    }
    // the item's plane offsets, read by every step from shared memory rather
    // than from the plane table in global memory
    const bool dtab = k_hi - k_lo <= G::DTAB;  // uniform
    if (dtab)
        for (int k = tid; k < k_hi - k_lo; k += NT) Ds[k] = L.planes[k_lo + k].d;
    // outputs of this thread (tid < NTV): column ox, rows oy0 .. oy0 + SEG - 1;
    // their reference window mean and 1/sqrt(sum of squared deviations), NaN = unusable
    const bool owner = tid < NTV;  // uniform over each warp
    const int ox = tid % TW, oy0 = (tid / TW) * SEG;
    const uint32_t tm = tm_addr(tmem);
    float2 st[SEG];
#pragma unroll
    for (int i = 0; i < SEG; ++i) {
        int gx = tx * TW + ox, gy = ty * TH + oy0 + i;
        float2 v = make_float2(0.f, -1.f);
        if (owner && gx < L.W && gy < L.H) v = L.stats[(size_t)gy * L.W + gx];
        st[i] = v.y >= (float)N * 1e-8f ? make_float2(v.x, rsqrtf(v.y)) : make_float2(nan, nan);
    }
    {
        float c1[SEG], c2[SEG], cprev[SEG], cminus[SEG], cplus[SEG], cfirst[SEG];
        int kb[SEG];
        bool needp[SEG];
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            c1[i] = c2[i] = cprev[i] = cminus[i] = cplus[i] = cfirst[i] = inf;
            kb[i] = -1;
            needp[i] = false;
        }
        wta_store<SEG>(tm, c1, c2, cprev, cminus, cplus, cfirst, kb, needp);
    }
    const int hrow = tid & 31, hrun = tid >> 5;  // phase H item
    const int base_v = oy0 * HS + ox;            // phase V first H entry
    const int base_f = oy0 * TW + ox;            // phase V first flag (KP = 2)

    for (int s = 0; s < L.n_sets; ++s) {
        const int s_lo = max(L.sets[s].start, k_lo), k_end = min(L.sets[s].start + L.sets[s].count, k_hi);
        if (s_lo >= k_end) continue;  // the set lies outside this work item's planes
        const float snx = L.sets[s].nx, sny = L.sets[s].ny, snz = L.sets[s].nz;
        // this thread's halo positions p = tid + i NT: per matching camera the
        // directions R_j r / (n . r) (NaN = none), into this thread's TMEM lane
        float rx[G::PPT], ry[G::PPT], rz[G::PPT], rinv[G::PPT];
#pragma unroll
        for (int i = 0; i < G::PPT; ++i) {
            const int p = tid + i * NT;
            const int hy = p / HWL, hx = p - hy * HWL;
            const int gx = gx0 + hx, gy = gy0 + hy;
            float4 r = make_float4(nan, nan, nan, 0.f);
            if (p < NPOS && gx >= 0 && gy >= 0 && gx < L.W && gy < L.H) r = L.rays[(size_t)gy * L.W + gx];
            float nr = snx * r.x + sny * r.y + snz * r.z;
            rinv[i] = nr > 0.0f ? 1.0f / nr : nan;
            rx[i] = r.x;
            ry[i] = r.y;
            rz[i] = r.z;
        }
#pragma unroll
        for (int j = 0; j < PS_MAX_CAMS; ++j) {  // unrolled: camera j's constants at fixed offsets in shared memory
            if (j >= L.n_cams) break;
            const CamS& C = cams[j];
            float av[9];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (i < G::PPT) {
                    av[3 * i] = rinv[i] * fmaf(C.R[0], rx[i], fmaf(C.R[1], ry[i], C.R[2] * rz[i]));
                    av[3 * i + 1] = rinv[i] * fmaf(C.R[3], rx[i], fmaf(C.R[4], ry[i], C.R[5] * rz[i]));
                    av[3 * i + 2] = rinv[i] * fmaf(C.R[6], rx[i], fmaf(C.R[7], ry[i], C.R[8] * rz[i]));
                } else {
                    av[3 * i] = av[3 * i + 1] = av[3 * i + 2] = nan;
                }
            }
            tm_st9(tm + TM_TAB + 9 * j, av);
        }
        __syncthreads();
        // planes go in groups of KP: the planes of a group are swept with one camera
        // before the next camera, so consecutive gathers hit overlapping
        // footprints of the same image
        for (int k0 = s_lo; k0 < k_end; k0 += KP) {
            const int np = min(KP, k_end - k0);
            float cmin[KP][SEG];
#pragma unroll
            for (int q = 0; q < KP; ++q)
#pragma unroll
                for (int i = 0; i < SEG; ++i) cmin[q][i] = inf;
#pragma unroll
            for (int j = 0; j < PS_MAX_CAMS; j += (KP == 2 ? 2 : 1)) {  // unrolled, as above
                if (j >= L.n_cams) break;
                const CamS& C = cams[j];
                float av[9];
                tm_ld9(tm + TM_TAB + 9 * j, av);
                const float d0 = dtab ? Ds[k0 - k_lo] : __ldg(&L.planes[k0].d);
                const float d1 = dtab ? Ds[k0 + np - 1 - k_lo] : __ldg(&L.planes[k0 + np - 1].d);
                if constexpr (KP == 2) {
                    if (j + 1 < L.n_cams) {  // two cameras in one step
                        pair_pass2<RHO, HALF, TH>(C, cams[j + 1], av, tm + TM_TAB + 9 * (j + 1), d0, d1, W2, Rs, Hs, Fs, st, base_v,
                                                  base_f, cmin[0], cmin[1]);
                    } else {
                        pair_pass<RHO, HALF, TH>(C, av, d0, d1, W2, Rs, Hs, Fs, st, base_v, base_f, cmin[0], cmin[1]);
                    }
                } else {
                    // phase A: warped samples of the tile + halo for the plane
                    int bad = 0;
#pragma unroll 3
                    for (int i = 0; i < G::PPT; ++i) {
                        int p = tid + i * NT;
                        if (p < NPOS) {
                            const float4 a = make_float4(av[3 * i], av[3 * i + 1], av[3 * i + 2], 0.f);
                            float w0 = warp_sample<HALF>(C, fmaf(d0, a.x, C.t[0]), fmaf(d0, a.y, C.t[1]), fmaf(d0, a.z, C.t[2]),
                                                         bad);
                            int hy = p / HWL, hx = p - hy * HWL;
                            Ws[hy * WS + hx] = w0;
                        }
                    }
                    bad = __syncthreads_or(bad);
                    // phase H: sliding horizontal sums along a run of one halo row
                    if (hrow < HH && hrun < TW / RUN) {
                        const float* wr = Ws + hrow * WS + RUN * hrun;
                        const float* rr = Rs + hrow * WS + RUN * hrun;
                        float w[4 * G::NV], r[4 * G::NV];
#pragma unroll
                        for (int qq = 0; qq < G::NV; ++qq) {
                            float4 a = *reinterpret_cast<const float4*>(wr + 4 * qq);
                            float4 b = *reinterpret_cast<const float4*>(rr + 4 * qq);
                            w[4 * qq] = a.x; w[4 * qq + 1] = a.y; w[4 * qq + 2] = a.z; w[4 * qq + 3] = a.w;
                            r[4 * qq] = b.x; r[4 * qq + 1] = b.y; r[4 * qq + 2] = b.z; r[4 * qq + 3] = b.w;
                        }
                        float4* hrow_out = Hs + hrow * HS + RUN * hrun;
                        float sw = 0.f, sww = 0.f, srw = 0.f, sm = 0.f;
                        if (!bad) {  // every sample of the tile is valid (the common case)
#pragma unroll
                            for (int t = 0; t <= 2 * RHO; ++t) {
                                sw += w[t];
                                sww = fmaf(w[t], w[t], sww);
                                srw = fmaf(r[t], w[t], srw);
                            }
                            hrow_out[0] = make_float4(sw, sww, srw, 0.f);
#pragma unroll
                            for (int o = 1; o < RUN; ++o) {
                                const int a = o + 2 * RHO, b = o - 1;
                                sw += w[a] - w[b];
                                sww += fmaf(w[a], w[a], -w[b] * w[b]);
                                srw += fmaf(r[a], w[a], -r[b] * w[b]);
                                hrow_out[o] = make_float4(sw, sww, srw, 0.f);
                            }
                        } else {  // invalid samples: excluded from the sums and counted
#pragma unroll
                            for (int t = 0; t <= 2 * RHO; ++t) {
                                bool bt = isnan(w[t]);
                                float wt = bt ? 0.0f : w[t];
                                sw += wt;
                                sww = fmaf(wt, wt, sww);
                                srw = fmaf(r[t], wt, srw);
                                sm += bt ? 1.0f : 0.0f;
                            }
                            hrow_out[0] = make_float4(sw, sww, srw, sm);
#pragma unroll
                            for (int o = 1; o < RUN; ++o) {
                                const int a = o + 2 * RHO, b = o - 1;
                                bool ba = isnan(w[a]), bb = isnan(w[b]);
                                float wa = ba ? 0.0f : w[a], wb = bb ? 0.0f : w[b];
                                sw += wa - wb;
                                sww += fmaf(wa, wa, -wb * wb);
                                srw += fmaf(r[a], wa, -r[b] * wb);
                                sm += (ba ? 1.0f : 0.0f) - (bb ? 1.0f : 0.0f);
                                hrow_out[o] = make_float4(sw, sww, srw, sm);
                            }
                        }
                    }
                    __syncthreads();
                    if (!owner) continue;
                    // phase V: sliding vertical sums down SEG rows, ZNCC, minimum over cameras
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int dy = 0; dy <= 2 * RHO; ++dy) {
                        float4 h = Hs[base_v + dy * HS];
                        v.x += h.x; v.y += h.y; v.z += h.z; v.w += h.w;
                    }
#pragma unroll
                    for (int i = 0; i < SEG; ++i) {
                        if (i > 0) {
                            float4 a = Hs[base_v + (i + 2 * RHO) * HS], b = Hs[base_v + (i - 1) * HS];
                            v.x += a.x - b.x; v.y += a.y - b.y; v.z += a.z - b.z; v.w += a.w - b.w;
                        }
                        float var_w = fmaf(-v.x * (1.0f / (float)N), v.x, v.y);
                        float cov = fmaf(-st[i].x, v.x, v.z);
                        bool ok = v.w == 0.0f && var_w >= (float)N * 1e-8f && !isnan(st[i].y);
                        // (1 - z) / 2 saturated to [0, 1], as in pair_phase_v_
                        float cost = __saturatef(__fmaf_rn(-0.5f, cov * st[i].y * rsqrt_ftz(var_w), 0.5f));
                        cmin[0][i] = ok ? fminf(cmin[0][i], cost) : cmin[0][i];
                    }
                }
            }
            // streaming winner-take-all with each plane's aggregated cost, in plane order
            if (!owner) continue;
            float c1[SEG], c2[SEG], cprev[SEG], cminus[SEG], cplus[SEG], cfirst[SEG];
            int kb[SEG];
            bool needp[SEG];
            wta_load<SEG>(tm, c1, c2, cprev, cminus, cplus, cfirst, kb, needp);
            if (k0 == k_lo) {  // the item's first plane (uniform)
#pragma unroll
                for (int i = 0; i < SEG; ++i) cfirst[i] = cmin[0][i];
            }
#pragma unroll
            for (int q = 0; q < KP; ++q) {
                if (q >= np) break;
                const int k = k0 + q;
#pragma unroll
                for (int i = 0; i < SEG; ++i) {
                    float cc = cmin[q][i];
                    const bool lt = cc < c1[i];  // a new winner (ties keep the earlier plane)
                    cplus[i] = lt ? inf : (needp[i] ? cc : cplus[i]);
                    needp[i] = lt;
                    c2[i] = fminf(c2[i], fmaxf(c1[i], cc));  // second smallest of c1, c2, cc
                    c1[i] = fminf(c1[i], cc);
                    kb[i] = lt ? k : kb[i];
                    cminus[i] = lt ? cprev[i] : cminus[i];
                    cprev[i] = cc;
                }
            }
            wta_store<SEG>(tm, c1, c2, cprev, cminus, cplus, cfirst, kb, needp);
        }
    }

    float c1[SEG], c2[SEG], cprev[SEG], cminus[SEG], cplus[SEG], cfirst[SEG];
    int kb[SEG];
    bool needp[SEG];
    wta_load<SEG>(tm, c1, c2, cprev, cminus, cplus, cfirst, kb, needp);
    if (L.n_chunks == 1) {
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            if (!owner) break;
            int gx = tx * TW + ox, gy = ty * TH + oy0 + i;
            if (gx < L.W && gy < L.H) {
                if (L.records)
                    write_record(L, gx, gy, c1[i], c2[i], cminus[i], cplus[i], cfirst[i], cprev[i], kb[i]);
                else
                    finish_pixel(L, gx, gy, c1[i], c2[i], kb[i], cminus[i], cplus[i]);
            }
        }
        tile_finished(L, true);
        return;
    }
    // several work items share this tile: publish this item's result; the
    // item that completes the tile merges all of them in plane order
    float* part = L.partial + (size_t)item * 7 * (TH * TW);
#pragma unroll
    for (int i = 0; i < SEG; ++i) {
        if (!owner) break;
        const int px = (oy0 + i) * TW + ox;
        part[0 * TH * TW + px] = c1[i];
        part[1 * TH * TW + px] = c2[i];
        part[2 * TH * TW + px] = cminus[i];
        part[3 * TH * TW + px] = cplus[i];
        part[4 * TH * TW + px] = cfirst[i];
        part[5 * TH * TW + px] = cprev[i];  // cost of the item's last plane
        part[6 * TH * TW + px] = __int_as_float(kb[i]);
    }
    merge_chunks<TH>(L, tile, s_flag);
}

// Stage the matching cameras of a level in shared memory (one thread each).
__device__ __forceinline__ void stage_cams(const LevelD& L, CamS* cams) {
    if (threadIdx.x < L.n_cams) cam_consts(L.cams[threadIdx.x], cams[threadIdx.x]);
}

// One work item of a level: stage the matching cameras in shared memory and
// run the tile routine for the level's window radius and image storage.
template <int TH, int KP>
__device__ __forceinline__ void sweep_item(const LevelD& L, int half, int item, CamS* cams, unsigned char* smem,
                                           int* s_flag, uint32_t tmem) {
    stage_cams(L, cams);
    __syncthreads();
    if (half) {
        switch (L.rho) {
            case 2: sweep_tile<2, true, TH, KP>(L, cams, item, smem, s_flag, tmem); break;
            case 3: sweep_tile<3, true, TH, KP>(L, cams, item, smem, s_flag, tmem); break;
            default: sweep_tile<4, true, TH, KP>(L, cams, item, smem, s_flag, tmem); break;
        }
    } else {
        switch (L.rho) {
            case 2: sweep_tile<2, false, TH, KP>(L, cams, item, smem, s_flag, tmem); break;
            case 3: sweep_tile<3, false, TH, KP>(L, cams, item, smem, s_flag, tmem); break;
            default: sweep_tile<4, false, TH, KP>(L, cams, item, smem, s_flag, tmem); break;
        }
    }
}

// Dynamic shared memory of a work item with window radius rho.
template <int TH, int KP>
inline size_t sweep_smem(int rho, int n_cams) {
    return rho == 2 ? Geo<2, TH, KP>::smem(n_cams) : rho == 3 ? Geo<3, TH, KP>::smem(n_cams)
                                                  : Geo<4, TH, KP>::smem(n_cams);
}

// ------------------------------------------------------------- merge

// ------------------------------------------------------------- merge

struct MergeP {
    int W, H;
    const float* low;
    const float *low_c1, *low_c2;
    int s, Wl, Hl;
    const float* crop;
    const float *crop_c1, *crop_c2;
    int cx0, cy0, cw, ch;
    int filter;                     // apply the per-level cost filters
    float alpha_upper, alpha_lower, split_row, ratio_min;
    int n_boxes;
    ps_box boxes[16];
};

// A level pixel survives the cost filters: best cost at most alpha of its
// image part, second best at least ratio_min times the best.
__device__ __forceinline__ bool keep_level(const MergeP& P, float c1, float c2, float row) {
    float alpha = row < P.split_row ? P.alpha_upper : P.alpha_lower;
    return c1 <= alpha && c2 >= P.ratio_min * c1;
}

// Merged depth at full-resolution pixel (u, v) before the boxes: the
// low-resolution level's pixel under it, replaced by the crop level's pixel
// where the crop covers (u, v) and has a depth; with the cost filters on, a
// level pixel that fails them contributes nothing.
__device__ __forceinline__ float merge_px(const MergeP& P, int u, int v) {
    float val = 0.f;
    if (P.low) {
        int lu = min(u / P.s, P.Wl - 1), lv = min(v / P.s, P.Hl - 1);
        size_t i = (size_t)lv * P.Wl + lu;
        val = P.low[i];
        if (P.filter && val > 0.f &&
            !keep_level(P, P.low_c1[i], P.low_c2[i], (float)(P.s * lv) + 0.5f * (float)(P.s - 1)))
            val = 0.f;
    }
    if (P.crop && u >= P.cx0 && u < P.cx0 + P.cw && v >= P.cy0 && v < P.cy0 + P.ch) {
        size_t i = (size_t)(v - P.cy0) * P.cw + (u - P.cx0);
        float c = P.crop[i];
        if (c > 0.f && (!P.filter || keep_level(P, P.crop_c1[i], P.crop_c2[i], (float)v))) val = c;
    }
    return val;
}

// Local depth continuity at (u, v) of the merged map: the pixel keeps its
// depth when at least a fraction delta of the other in-image pixels of its
// window have a depth within gamma of it.
__device__ __forceinline__ float continuity_px(const float* in, int W, int H, int half, float gamma, float delta,
                                               int u, int v) {
    float d = in[(size_t)v * W + u];
    float res = 0.f;
    if (d > 0.f) {
        int cons = 0, tot = 0;
        for (int dy = -half; dy <= half; ++dy) {
            int vv = v + dy;
            if (vv < 0 || vv >= H) continue;
            for (int dx = -half; dx <= half; ++dx) {
                int uu = u + dx;
                if (uu < 0 || uu >= W || (dx == 0 && dy == 0)) continue;
                ++tot;
                float dn = in[(size_t)vv * W + uu];
                cons += (dn > 0.f && fabsf(dn - d) < gamma) ? 1 : 0;
            }
        }
        if (tot > 0 && (float)cons >= delta * (float)tot) res = d;
    }
    return res;
}

// (u, v) lies inside one of n boxes (half-open pixel ranges).
__device__ __forceinline__ bool in_boxes(const ps_box* b, int n, int u, int v) {
    bool in = false;
    for (int i = 0; i < n; ++i) in |= u >= b[i].x0 && u < b[i].x1 && v >= b[i].y0 && v < b[i].y1;
    return in;
}

}  // namespace ps

using namespace ps;

struct psweep_s {
    uint32_t magic = MAGIC_SWEEP;  // first word: handle type for ps_sync_status
    unsigned* status = nullptr;    // latched DEV_* bits (device word)
    ps_camera ref;
    int n_cams;
    ps_camera cams[PS_MAX_CAMS];
    ps_pose poses[PS_MAX_CAMS];
    int n_levels;
    ps_level levels[PS_MAX_LEVELS];
    // per level
    ps_camera lref[PS_MAX_LEVELS];              // reference camera at the level
    ps_camera lcam[PS_MAX_LEVELS][PS_MAX_CAMS];  // matching cameras at the level
    int lW[PS_MAX_LEVELS], lH[PS_MAX_LEVELS];
    int cx0[PS_MAX_LEVELS], cy0[PS_MAX_LEVELS];
    float4* rays[PS_MAX_LEVELS] = {};
    PlaneD* planes[PS_MAX_LEVELS] = {};
    float* ref_img[PS_MAX_LEVELS] = {};
    float2* stats[PS_MAX_LEVELS] = {};
    float* partial[PS_MAX_LEVELS] = {};
    int* done[PS_MAX_LEVELS] = {};
    int chunk[PS_MAX_LEVELS] = {};
    void* quad[PS_MAX_LEVELS][PS_MAX_CAMS] = {};
    int image_half = 0;
    int* tile_counter = nullptr;
    int grid = 0;
    int smem_optin = 0;
    float* out_depth[PS_MAX_LEVELS] = {};
    float* out_c1[PS_MAX_LEVELS] = {};
    float* out_c2[PS_MAX_LEVELS] = {};
    int32_t* out_k[PS_MAX_LEVELS] = {};
    ps_box* boxes_dev = nullptr;
    int boxes_cap = 0;
    SetD sets[PS_MAX_LEVELS][PS_MAX_SETS];
    int n_planes[PS_MAX_LEVELS];
    // host-frame staging (psweep_frame_host)
    uint8_t* stage_img[1 + PS_MAX_CAMS] = {};
    float* stage_depth = nullptr;
    ps_filter filter{};
    float* merged = nullptr;  // merged map before the continuity filter
    StageProfiler prof;
};

namespace ps {

// Level record of level l of a sweep for tiles of th rows and work items of
// `chunk` planes; outputs go to the handle's level buffers, and the chunk
// scratch, tile counters and finished-tile count are left NULL for the caller.
void fill_level(const psweep_t* h, int l, int th, int chunk, LevelD& D);

// Planes per work item: at most `most`, balanced over the items of a tile.
int balanced_chunk(int n_planes, int most);

// Merge rule of a sweep reading the level outputs of lv[l] (level order of
// the handle), with the handle's cost filters; no boxes.
void fill_merge(const psweep_t* h, const LevelD* lv, MergeP& M);

}  // namespace ps

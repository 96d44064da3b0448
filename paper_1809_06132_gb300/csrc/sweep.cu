// Fisheye plane-sweep stereo at multiple scales (Sec. III-A) on sm_103a.
//
// Kernels:
//   ray_table_kernel   Eq. 1 back-projection of every reference pixel of a
//                      level, in double precision, stored as float4 (once
//                      per rig, at psweep_create).
//   ref_level_kernel   reference image of a level (s x s box mean, or the
//                      centred crop), centred intensities I/255 - 1/2.
//   quad_level_kernel  matching image of a level in "quad" layout: entry
//                      (x, y) holds the 2 x 2 neighbourhood used by one
//                      bilinear sample, so a sample is one 16-byte gather.
//   sweep_kernel       the hot loop.  One CTA owns a TW x TH tile of output
//                      pixels of one level and walks every plane and every
//                      matching camera: warp the tile + window halo through
//                      the plane into shared memory, box-sum w, w^2, r w and
//                      the invalid count with separable sums, ZNCC -> cost,
//                      minimum over cameras, and a streaming winner-take-all
//                      that keeps the best, second best and the winner's two
//                      neighbours in registers.  The cost volume never
//                      leaves the SM.  Both levels' tiles share one launch.
//   merge_kernel       full-resolution merge of the levels and box masks.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "internal.cuh"

namespace ps {

namespace {

constexpr int TW = 64;   // output tile width (pixels)
constexpr int TH = 24;   // output tile height
constexpr int NT = 512;  // threads per CTA (one CTA per SM)
constexpr int RUN = 4;   // outputs per horizontal run (phase H)
constexpr int SEG = 3;   // output rows per vertical segment (phase V)
constexpr int KP = 2;    // planes swept per camera before moving to the next camera
constexpr int PLANE_CHUNK = 32;  // most planes one work item sweeps
static_assert(NT == TW * (TH / SEG), "phase V: one thread per column and row segment");
static_assert(NT / 32 >= TW / RUN, "phase H: one warp per run, one lane per halo row");

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
    int chunk, n_chunks, n_items;  // planes per work item, items per tile, tiles x items
    float* partial;                // [n_items][7][TH * TW] chunk results (when n_chunks > 1)
    int* done;                     // [n_tiles] finished chunks per tile (zeroed per launch)
    float* depth;
    float* c1;
    float* c2;
    int32_t* kstar;
};

struct SweepParams {
    int n_levels;
    int image_half;  // matching quads stored as FP16
    LevelD lv[PS_MAX_LEVELS];
};

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

// ------------------------------------------------------------- level images

// Centred intensity of the s x s block at level pixel (x, y), clamped to the image.
__device__ __forceinline__ float level_px(const uint8_t* img, int W, int Wl, int Hl, int s, int x, int y) {
    x = min(x, Wl - 1);
    y = min(y, Hl - 1);
    int acc = 0;
    for (int dy = 0; dy < s; ++dy)
        for (int dx = 0; dx < s; ++dx) acc += img[(size_t)(s * y + dy) * W + (s * x + dx)];
    return (float)acc * (1.0f / (255.0f * s * s)) - 0.5f;
}

__global__ void ref_level_kernel(const uint8_t* img, int W, int s, int x0, int y0, int Wl, int Hl, float* out) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= Wl || y >= Hl) return;
    float v;
    if (s > 0)
        v = level_px(img, W, Wl, Hl, s, x, y);
    else
        v = img[(size_t)(y0 + y) * W + (x0 + x)] * (1.0f / 255.0f) - 0.5f;
    out[(size_t)y * Wl + x] = v;
}

// Matching image of a level in "quad" layout: entry (x, y) holds the
// centred intensities at (x, y), (x+1, y), (x, y+1), (x+1, y+1), so one
// bilinear sample is one 16-byte gather.
__global__ void quad_level_kernel(const uint8_t* img, int W, int s, int Wl, int Hl, void* out, int half) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= Wl || y >= Hl) return;
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
        static_cast<float4*>(out)[(size_t)y * Wl + x] = q;
    }
}

// ------------------------------------------------------------- reference statistics

// Mean and sum of squared deviations of the reference window around every
// level pixel (two-pass, direct sums); var = -1 where the window leaves the
// image.  Computed once per frame, read by the sweep for every plane.
__global__ void ref_stats_kernel(const float* ref, int W, int H, int rho, float2* out) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= W || y >= H) return;
    float2 o = make_float2(0.f, -1.f);
    if (x >= rho && y >= rho && x < W - rho && y < H - rho) {
        float s = 0.f;
        for (int dy = -rho; dy <= rho; ++dy)
            for (int dx = -rho; dx <= rho; ++dx) s += ref[(size_t)(y + dy) * W + x + dx];
        float m = s / (float)((2 * rho + 1) * (2 * rho + 1));
        float v = 0.f;
        for (int dy = -rho; dy <= rho; ++dy)
            for (int dx = -rho; dx <= rho; ++dx) {
                float e = ref[(size_t)(y + dy) * W + x + dx] - m;
                v = fmaf(e, e, v);
            }
        o = make_float2(m, v);
    }
    out[(size_t)y * W + x] = o;
}

// ------------------------------------------------------------- sweep

// Matching camera as the sweep reads it (staged in shared memory per tile).
struct CamS {
    float R[9], t[3];
    float xi, fx, fy, cx, cy, k1, k2, p1, p2, r2_max, lim, wm1, hm1;
    int width;
    const void* quad;
};

// Bilinear sample of a matching camera at the projection of X_j (camera
// frame), as a centred intensity; NaN when the point does not project
// (sphere side, distortion range) or lands outside [0, W-1] x [0, H-1].
// The gather is clamped into the image and always issued, so the warp does
// not diverge; a clamp that moved the point marks it outside (NaN compares
// unequal, so a NaN position is rejected too).  HALF: quads stored as FP16.
template <bool HALF>
__device__ __forceinline__ float warp_sample(const CamS& c, float X, float Y, float Z) {
    float n2 = fmaf(X, X, fmaf(Y, Y, Z * Z));
    float n = n2 * rsqrtf(n2);
    float inv = __fdividef(1.0f, fmaf(c.xi, n, Z));
    float mx = X * inv, my = Y * inv;
    float r2 = fmaf(mx, mx, my * my);
    float rad = fmaf(r2, fmaf(c.k2, r2, c.k1), 1.0f);
    float mxy = mx * my;
    float xd = fmaf(mx, rad, fmaf(2.0f * c.p1, mxy, c.p2 * fmaf(2.0f * mx, mx, r2)));
    float yd = fmaf(my, rad, fmaf(c.p1, fmaf(2.0f * my, my, r2), 2.0f * c.p2 * mxy));
    float u = fmaf(c.fx, xd, c.cx);
    float v = fmaf(c.fy, yd, c.cy);
    float uc = fminf(fmaxf(u, 0.0f), c.wm1), vc = fminf(fmaxf(v, 0.0f), c.hm1);
    bool ok = (Z > c.lim * n) && (r2 <= c.r2_max) && (uc == u) && (vc == v);
    int x0 = (int)uc, y0 = (int)vc;
    float ax = uc - (float)x0, ay = vc - (float)y0;
    float4 q;
    if (HALF) {
        uint2 h = __ldg(static_cast<const uint2*>(c.quad) + y0 * c.width + x0);
        float2 a = __half22float2(*reinterpret_cast<const __half2*>(&h.x));
        float2 b = __half22float2(*reinterpret_cast<const __half2*>(&h.y));
        q = make_float4(a.x, a.y, b.x, b.y);
    } else {
        q = __ldg(static_cast<const float4*>(c.quad) + y0 * c.width + x0);
    }
    float top = fmaf(ax, q.y - q.x, q.x);
    float bot = fmaf(ax, q.w - q.z, q.z);
    float w = fmaf(ay, bot - top, top);
    return ok ? w : __int_as_float(0x7fc00000);
}

// Tile geometry.  A CTA owns TW x TH output pixels of one level plus a halo of
// RHO on every side (HH rows x HWL columns of warped samples per plane and
// camera).  Per plane set, every halo position keeps, per matching camera,
// a = R_j r / (n . r), so that the plane at offset d maps it to d a + t_j.
// Phase A: every thread warps PPT halo positions into W.  Phase H: thread
// (row, run) slides a 2 RHO + 1 window along RUN outputs of one halo row and
// stores (sum w, sum w^2, sum r w, invalid count) in H.  Phase V: thread
// (column, segment) slides down SEG output rows, forms ZNCC and keeps the
// minimum over cameras.  Strides make every phase's shared-memory accesses
// free of bank conflicts.
template <int RHO>
struct Geo {
    static constexpr int HH = TH + 2 * RHO;           // halo rows (<= 32)
    static constexpr int HWL = TW + 2 * RHO;          // halo columns
    static constexpr int WS = 76;                     // W / R row stride (floats): 76 = 12 mod 32
    static constexpr int HS = TW + 1;                 // H row stride (float4): odd
    static constexpr int NPOS = HH * HWL;
    static constexpr int PPT = (NPOS + NT - 1) / NT;
    static constexpr int NRUNPOS = RUN + 2 * RHO;     // positions one horizontal run reads
    static constexpr int NV = (NRUNPOS + 3) / 4;      // float4 loads per run
    static constexpr int N = (2 * RHO + 1) * (2 * RHO + 1);
    // n_cams direction tables, H, two W (one per plane of a pair) and R
    static constexpr size_t smem(int n_cams) {
        return sizeof(float4) * ((size_t)n_cams * NPOS + HH * HS) + sizeof(float) * 3 * HH * WS;
    }
    static_assert(HH <= 32, "phase H maps one warp lane per halo row");
    static_assert(HWL <= WS && 4 * NV + TW - RUN <= WS, "row stride covers the runs' loads");
};

// Parabola through the winner and its neighbours in the same plane set, and
// the range along the pixel's ray; writes the level outputs of one pixel.
__device__ void finish_pixel(const LevelD& L, int gx, int gy, float c1, float c2, int kb, float cminus, float cplus) {
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

template <int RHO, bool HALF>
__device__ void sweep_tile(const LevelD& L, const CamS* cams, int item, unsigned char* smem_raw, int* s_flag) {
    using G = Geo<RHO>;
    const int tile = item / L.n_chunks, chunk = item - tile * L.n_chunks;
    const int k_lo = chunk * L.chunk, k_hi = min(L.n_planes, k_lo + L.chunk);
    constexpr int HH = G::HH, HWL = G::HWL, WS = G::WS, HS = G::HS, NPOS = G::NPOS, N = G::N;
    float4* Hs = reinterpret_cast<float4*>(smem_raw);            // [HH][HS] window sums
    float4* A = Hs + HH * HS;                                     // [n_cams][NPOS] (R_j r / n.r); NaN = none
    float* Ws = reinterpret_cast<float*>(A + L.n_cams * NPOS);    // [2][HH][WS] warped samples of the pair (NaN = invalid)
    float* Rs = Ws + 2 * HH * WS;                                 // [HH][WS] reference intensities
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
    // outputs of this thread: column ox, rows oy0 .. oy0 + SEG - 1; their
    // reference window mean and 1/sqrt(sum of squared deviations), NaN = unusable
    const int ox = tid % TW, oy0 = (tid / TW) * SEG;
    float2 st[SEG];
#pragma unroll
    for (int i = 0; i < SEG; ++i) {
        int gx = tx * TW + ox, gy = ty * TH + oy0 + i;
        float2 v = make_float2(0.f, -1.f);
        if (gx < L.W && gy < L.H) v = L.stats[(size_t)gy * L.W + gx];
        st[i] = v.y >= (float)N * 1e-8f ? make_float2(v.x, rsqrtf(v.y)) : make_float2(nan, nan);
    }
    float c1[SEG], c2[SEG], cprev[SEG], cminus[SEG], cplus[SEG], cfirst[SEG];
    int kb[SEG];
    bool needp[SEG];
#pragma unroll
    for (int i = 0; i < SEG; ++i) {
        c1[i] = c2[i] = cprev[i] = cminus[i] = cplus[i] = cfirst[i] = inf;
        kb[i] = -1;
        needp[i] = false;
    }
    const int hrow = tid & 31, hrun = tid >> 5;  // phase H item
    const int base_v = oy0 * HS + ox;            // phase V first H entry

    for (int s = 0; s < L.n_sets; ++s) {
        const int s_lo = max(L.sets[s].start, k_lo), k_end = min(L.sets[s].start + L.sets[s].count, k_hi);
        if (s_lo >= k_end) continue;  // the set lies outside this work item's planes
        const float snx = L.sets[s].nx, sny = L.sets[s].ny, snz = L.sets[s].nz;
        __syncthreads();  // previous users of A are done
        for (int p = tid; p < NPOS; p += NT) {
            int hy = p / HWL, hx = p - hy * HWL;
            int gx = gx0 + hx, gy = gy0 + hy;
            float4 r = make_float4(nan, nan, nan, 0.f);
            if (gx >= 0 && gy >= 0 && gx < L.W && gy < L.H) r = L.rays[(size_t)gy * L.W + gx];
            float nr = snx * r.x + sny * r.y + snz * r.z;
            float inv = nr > 0.0f ? 1.0f / nr : nan;
            for (int j = 0; j < L.n_cams; ++j) {
                const CamS& C = cams[j];
                A[j * NPOS + p] = make_float4(inv * fmaf(C.R[0], r.x, fmaf(C.R[1], r.y, C.R[2] * r.z)),
                                              inv * fmaf(C.R[3], r.x, fmaf(C.R[4], r.y, C.R[5] * r.z)),
                                              inv * fmaf(C.R[6], r.x, fmaf(C.R[7], r.y, C.R[8] * r.z)), 0.f);
            }
        }
        __syncthreads();
        // planes go in pairs: both planes of a pair are swept with one camera
        // before the next camera, so consecutive gathers hit overlapping
        // footprints of the same image
        for (int k0 = s_lo; k0 < k_end; k0 += KP) {
            const int np = min(KP, k_end - k0);
            float cmin[KP][SEG];
#pragma unroll
            for (int q = 0; q < KP; ++q)
#pragma unroll
                for (int i = 0; i < SEG; ++i) cmin[q][i] = inf;
            for (int j = 0; j < L.n_cams; ++j) {
                const CamS& C = cams[j];
                const float4* Aj = A + j * NPOS;
                // phase A: warped samples of the tile + halo for both planes of the pair
                const float d0 = __ldg(&L.planes[k0].d);
                const float d1 = __ldg(&L.planes[k0 + np - 1].d);
                int bad = 0;
#pragma unroll 3
                for (int i = 0; i < G::PPT; ++i) {
                    int p = tid + i * NT;
                    if (p < NPOS) {
                        float4 a = Aj[p];
                        float w0 = warp_sample<HALF>(C, fmaf(d0, a.x, C.t[0]), fmaf(d0, a.y, C.t[1]), fmaf(d0, a.z, C.t[2]));
                        float w1 = warp_sample<HALF>(C, fmaf(d1, a.x, C.t[0]), fmaf(d1, a.y, C.t[1]), fmaf(d1, a.z, C.t[2]));
                        bad |= isnan(w0) | isnan(w1);
                        int hy = p / HWL, hx = p - hy * HWL;
                        Ws[hy * WS + hx] = w0;
                        Ws[HH * WS + hy * WS + hx] = w1;
                    }
                }
                bad = __syncthreads_or(bad);
#pragma unroll
                for (int q = 0; q < KP; ++q) {
                    if (q >= np) break;
                    if (q > 0) __syncthreads();  // the previous plane's vertical pass is done with H
                    // phase H: sliding horizontal sums along a run of one halo row
                    if (hrow < HH && hrun < TW / RUN) {
                        const float* wr = Ws + q * HH * WS + hrow * WS + RUN * hrun;
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
                        float z = fminf(1.0f, fmaxf(-1.0f, cov * st[i].y * rsqrtf(var_w)));  // |ZNCC| <= 1
                        float cost = fmaf(-0.5f, z, 0.5f);
                        cmin[q][i] = ok ? fminf(cmin[q][i], cost) : cmin[q][i];
                    }
                }
            }
            // streaming winner-take-all with each plane's aggregated cost, in plane order
#pragma unroll
            for (int q = 0; q < KP; ++q) {
                if (q >= np) break;
                const int k = k0 + q;
#pragma unroll
                for (int i = 0; i < SEG; ++i) {
                    float cc = cmin[q][i];
                    if (k == k_lo) cfirst[i] = cc;
                    if (needp[i]) {
                        cplus[i] = cc;
                        needp[i] = false;
                    }
                    if (cc < c1[i]) {
                        c2[i] = c1[i];
                        c1[i] = cc;
                        kb[i] = k;
                        cminus[i] = cprev[i];
                        cplus[i] = inf;
                        needp[i] = true;
                    } else if (cc < c2[i]) {
                        c2[i] = cc;
                    }
                    cprev[i] = cc;
                }
            }
        }
    }

    if (L.n_chunks == 1) {
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            int gx = tx * TW + ox, gy = ty * TH + oy0 + i;
            if (gx < L.W && gy < L.H) finish_pixel(L, gx, gy, c1[i], c2[i], kb[i], cminus[i], cplus[i]);
        }
        __syncthreads();
        return;
    }
    // several work items share this tile: publish this item's result; the
    // item that completes the tile merges all of them in plane order
    float* part = L.partial + (size_t)item * 7 * (TH * TW);
#pragma unroll
    for (int i = 0; i < SEG; ++i) {
        const int px = (oy0 + i) * TW + ox;
        part[0 * TH * TW + px] = c1[i];
        part[1 * TH * TW + px] = c2[i];
        part[2 * TH * TW + px] = cminus[i];
        part[3 * TH * TW + px] = cplus[i];
        part[4 * TH * TW + px] = cfirst[i];
        part[5 * TH * TW + px] = cprev[i];  // cost of the item's last plane
        part[6 * TH * TW + px] = __int_as_float(kb[i]);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) *s_flag = atomicAdd(&L.done[tile], 1) == L.n_chunks - 1;
    __syncthreads();
    if (*s_flag) {
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
                const int lo = wc * L.chunk, hi = min(L.n_planes, lo + L.chunk);
                cm = k > lo ? __ldcg(P + 2 * (TH * TW))
                            : (wc > 0 ? __ldcg(base + ((size_t)(wc - 1) * 7 + 5) * (TH * TW) + px) : inf);
                cp = k < hi - 1 ? __ldcg(P + 3 * (TH * TW))
                                : (wc + 1 < L.n_chunks ? __ldcg(base + ((size_t)(wc + 1) * 7 + 4) * (TH * TW) + px)
                                                       : inf);
            }
            if (gx < L.W && gy < L.H) finish_pixel(L, gx, gy, b1, b2, k, cm, cp);
        }
    }
    __syncthreads();
}

template <int LV>
__device__ __forceinline__ void run_level(const SweepParams& P, int item, CamS* cams, unsigned char* smem,
                                          int* s_flag) {
    const LevelD& L = P.lv[LV];
    if (threadIdx.x < L.n_cams) {
        const CamJ& J = L.cams[threadIdx.x];
        CamS& c = cams[threadIdx.x];
        for (int i = 0; i < 9; ++i) c.R[i] = J.R[i];
        for (int i = 0; i < 3; ++i) c.t[i] = J.t[i];
        c.xi = J.cam.xi; c.fx = J.cam.fx; c.fy = J.cam.fy; c.cx = J.cam.cx; c.cy = J.cam.cy;
        c.k1 = J.cam.k1; c.k2 = J.cam.k2; c.p1 = J.cam.p1; c.p2 = J.cam.p2; c.r2_max = J.cam.r2_max;
        c.lim = J.cam.lim;
        c.wm1 = (float)(J.cam.width - 1);
        c.hm1 = (float)(J.cam.height - 1);
        c.width = J.cam.width;
        c.quad = J.quad;
    }
    __syncthreads();
    if (P.image_half) {
        switch (L.rho) {
            case 2: sweep_tile<2, true>(L, cams, item, smem, s_flag); break;
            case 3: sweep_tile<3, true>(L, cams, item, smem, s_flag); break;
            default: sweep_tile<4, true>(L, cams, item, smem, s_flag); break;
        }
    } else {
        switch (L.rho) {
            case 2: sweep_tile<2, false>(L, cams, item, smem, s_flag); break;
            case 3: sweep_tile<3, false>(L, cams, item, smem, s_flag); break;
            default: sweep_tile<4, false>(L, cams, item, smem, s_flag); break;
        }
    }
}

// Persistent CTAs take work items (a tile and a chunk of its planes) from a
// counter; levels are ordered so the heavier items start first.
__global__ void __launch_bounds__(NT, 1) sweep_kernel(const __grid_constant__ SweepParams P, int* tile_counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ CamS cams[PS_MAX_CAMS];
    __shared__ int s_tile, s_flag;
    const int total = P.lv[0].n_items + (P.n_levels > 1 ? P.lv[1].n_items : 0);
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= total) break;
        if (t < P.lv[0].n_items)
            run_level<0>(P, t, cams, smem, &s_flag);
        else
            run_level<1>(P, t - P.lv[0].n_items, cams, smem, &s_flag);
    }
}

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

__global__ void merge_kernel(const __grid_constant__ MergeP P, const ps_box* boxes, float* out) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y;
    if (u >= P.W || v >= P.H) return;
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
    for (int b = 0; b < P.n_boxes; ++b) {
        ps_box bx = b < 16 ? P.boxes[b] : boxes[b];
        if (u >= bx.x0 && u < bx.x1 && v >= bx.y0 && v < bx.y1) val = 0.f;
    }
    out[(size_t)v * P.W + u] = val;
}

// Local depth continuity on the merged map, then the boxes: a pixel keeps its
// depth when at least a fraction delta of the other in-image pixels of its
// window have a depth within gamma of it.
__global__ void continuity_kernel(const float* in, int W, int H, int half, float gamma, float delta,
                                  const __grid_constant__ MergeP P, const ps_box* boxes, float* out) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y;
    if (u >= W || v >= H) return;
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
    for (int b = 0; b < P.n_boxes; ++b) {
        ps_box bx = b < 16 ? P.boxes[b] : boxes[b];
        if (u >= bx.x0 && u < bx.x1 && v >= bx.y0 && v < bx.y1) res = 0.f;
    }
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

struct psweep_s {
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
            // items of both levels cost about the same and balance across SMs
            const int n_tiles = ((W + TW - 1) / TW) * ((H + TH - 1) / TH);
            const int n_chunks = (h->n_planes[l] + PLANE_CHUNK - 1) / PLANE_CHUNK;
            h->chunk[l] = (h->n_planes[l] + n_chunks - 1) / n_chunks;
            if (n_chunks > 1)
                PS_TRY(cudaMalloc(&h->partial[l], sizeof(float) * 7 * TH * TW * (size_t)n_tiles * n_chunks));
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
        PS_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel, NT, Geo<4>::smem(d->n_cams)));
        h->grid = sms * std::max(1, per_sm);
    }
    PS_TRY(cudaDeviceSynchronize());
#undef PS_TRY
    *out = h;
    return PS_OK;
}

extern "C" void psweep_destroy(psweep_t* h) { free_sweep(h); }

extern "C" int psweep_depth(psweep_t* h, const uint8_t* const* images, const ps_box* boxes, int32_t n_boxes,
                            float* depth_out, const ps_level_out* level_out, void* stream) {
    clear_error();
    PS_ARG(h != nullptr, "psweep_depth: handle is NULL");
    PS_ARG(images != nullptr, "psweep_depth: images is NULL");
    for (int i = 0; i <= h->n_cams; ++i) PS_ARG(images[i] != nullptr, "psweep_depth: images[%d] is NULL", i);
    PS_ARG(depth_out != nullptr, "psweep_depth: depth_out is NULL");
    PS_ARG(n_boxes >= 0 && n_boxes <= h->boxes_cap, "psweep_depth: n_boxes must be in 0..%d", h->boxes_cap);
    PS_ARG(n_boxes == 0 || boxes != nullptr, "psweep_depth: boxes is NULL");
    cudaStream_t s = (cudaStream_t)stream;

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
            return (double)h->chunk[l] * (TW + 2 * r) * (TH + 2 * r);
        };
        if (cost(1) > cost(0)) std::swap(order[0], order[1]);
    }
    for (int oi = 0; oi < h->n_levels; ++oi) {
        const int l = order[oi];
        const ps_level& L = h->levels[l];
        const int W = h->lW[l], H = h->lH[l];
        if (L.kind == PS_LEVEL_DOWNSAMPLE) {
            int sf = L.factor;
            ref_level_kernel<<<dim3((W + 127) / 128, H), 128, 0, s>>>(images[0], h->ref.width, sf, 0, 0, W, H,
                                                                       h->ref_img[l]);
            for (int j = 0; j < h->n_cams; ++j) {
                const ps_camera& cj = h->lcam[l][j];
                quad_level_kernel<<<dim3((cj.width + 127) / 128, cj.height), 128, 0, s>>>(
                    images[1 + j], h->cams[j].width, sf, cj.width, cj.height, h->quad[l][j], h->image_half);
            }
        } else {
            ref_level_kernel<<<dim3((W + 127) / 128, H), 128, 0, s>>>(images[0], h->ref.width, 0, h->cx0[l],
                                                                       h->cy0[l], W, H, h->ref_img[l]);
            for (int j = 0; j < h->n_cams; ++j) {
                const ps_camera& cj = h->lcam[l][j];
                quad_level_kernel<<<dim3((cj.width + 127) / 128, cj.height), 128, 0, s>>>(
                    images[1 + j], h->cams[j].width, 1, cj.width, cj.height, h->quad[l][j], h->image_half);
            }
        }
        ref_stats_kernel<<<dim3((W + 127) / 128, H), 128, 0, s>>>(h->ref_img[l], W, H, L.window / 2, h->stats[l]);
        LevelD& D = P.lv[oi];
        D.W = W;
        D.H = H;
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
        D.tiles_x = (W + TW - 1) / TW;
        D.tiles_y = (H + TH - 1) / TH;
        D.n_tiles = D.tiles_x * D.tiles_y;
        D.chunk = h->chunk[l];
        D.n_chunks = (D.n_planes + D.chunk - 1) / D.chunk;
        D.n_items = D.n_tiles * D.n_chunks;
        D.partial = h->partial[l];
        D.done = h->done[l];
        PS_CUDA(cudaMemsetAsync(D.done, 0, sizeof(int) * D.n_tiles, s));
        const ps_level_out* lo = level_out ? &level_out[l] : nullptr;
        D.depth = lo && lo->depth ? lo->depth : h->out_depth[l];
        D.c1 = lo && lo->best_cost ? lo->best_cost : h->out_c1[l];
        D.c2 = lo && lo->second_cost ? lo->second_cost : h->out_c2[l];
        D.kstar = lo && lo->plane_idx ? lo->plane_idx : h->out_k[l];
    }
    PS_CUDA(cudaGetLastError());
    size_t smem = 0;
    int tiles = 0;
    for (int l = 0; l < h->n_levels; ++l) {
        int r = P.lv[l].rho;
        const int nc = h->n_cams;
        smem = std::max(smem, r == 2 ? Geo<2>::smem(nc) : r == 3 ? Geo<3>::smem(nc) : Geo<4>::smem(nc));
        tiles += P.lv[l].n_items;
    }
    PS_CUDA(cudaMemsetAsync(h->tile_counter, 0, sizeof(int), s));
    h->prof.mark(1, s);
    sweep_kernel<<<std::min(tiles, h->grid), NT, smem, s>>>(P, h->tile_counter);
    PS_CUDA(cudaGetLastError());
    h->prof.mark(2, s);

    MergeP M;
    std::memset(&M, 0, sizeof(M));
    M.W = h->ref.width;
    M.H = h->ref.height;
    M.s = 1;
    M.Wl = M.Hl = 1;
    for (int oi = 0; oi < h->n_levels; ++oi) {
        const int l = order[oi];
        const ps_level& L = h->levels[l];
        if (L.kind == PS_LEVEL_DOWNSAMPLE) {
            M.low = P.lv[oi].depth;
            M.low_c1 = P.lv[oi].c1;
            M.low_c2 = P.lv[oi].c2;
            M.s = L.factor;
            M.Wl = h->lW[l];
            M.Hl = h->lH[l];
        } else {
            M.crop = P.lv[oi].depth;
            M.crop_c1 = P.lv[oi].c1;
            M.crop_c2 = P.lv[oi].c2;
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

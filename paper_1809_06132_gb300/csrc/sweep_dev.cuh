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
constexpr int NT = 512;  // threads per CTA (one CTA per SM)
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
    int chunk, n_chunks, n_items;  // planes per work item, items per tile, tiles x items
    float* partial;                // [n_items][7][TH x TW] chunk results (when n_chunks > 1)
    int* done;                     // [n_tiles] finished chunks per tile (zeroed per launch)
    int* tiles_done;               // bumped once per finished tile (batched launch), or NULL
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

// Matching image of a level in "quad" layout: entry (x, y) holds the
// centred intensities at (x, y), (x+1, y), (x, y+1), (x+1, y+1), so one
// bilinear sample is one 16-byte gather (8 bytes with FP16 storage).
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
        static_cast<float4*>(out)[(size_t)y * Wl + x] = q;
    }
}

// Mean and sum of squared deviations of the window of radius rho centred on
// base[0] (row stride `stride`), by the two-pass direct sums.
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
// free of bank conflicts.  KP planes are warped per camera before the
// window sums of each run, so consecutive gathers hit overlapping
// footprints of the same image.
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
    // n_cams direction tables, H, KP W (one per plane of the group) and R
    static constexpr size_t smem(int n_cams) {
        return sizeof(float4) * ((size_t)n_cams * NPOS + HH * HS) + sizeof(float) * (KP + 1) * HH * WS;
    }
    static_assert(NT == TW * (TH / SEG) && TH % 8 == 0, "phase V: one thread per column and row segment");
    static_assert(KP == 1 || KP == 2, "one or two planes per pass");
    static_assert(HH <= 32, "phase H maps one warp lane per halo row");
    static_assert(HWL <= WS && 4 * NV + TW - RUN <= WS, "row stride covers the runs' loads");
};

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

template <int RHO, bool HALF, int TH, int KP>
__device__ inline void sweep_tile(const LevelD& L, const CamS* cams, int item, unsigned char* smem_raw, int* s_flag) {
    using G = Geo<RHO, TH, KP>;
    constexpr int SEG = G::SEG;
    if (!PS_DCHECK(item >= 0 && item < L.n_items, CHK_ITEM)) return;  // uniform over the CTA
    const int tile = item / L.n_chunks, chunk = item - tile * L.n_chunks;
    const int k_lo = chunk * L.chunk, k_hi = min(L.n_planes, k_lo + L.chunk);
    constexpr int HH = G::HH, HWL = G::HWL, WS = G::WS, HS = G::HS, NPOS = G::NPOS, N = G::N;
    float4* Hs = reinterpret_cast<float4*>(smem_raw);            // [HH][HS] window sums
    float4* A = Hs + HH * HS;                                     // [n_cams][NPOS] (R_j r / n.r); NaN = none
    float* Ws = reinterpret_cast<float*>(A + L.n_cams * NPOS);    // [KP][HH][WS] warped samples of the group (NaN = invalid)
    float* Rs = Ws + KP * HH * WS;                                // [HH][WS] reference intensities
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
            for (int j = 0; j < L.n_cams; ++j) {
                const CamS& C = cams[j];
                const float4* Aj = A + j * NPOS;
                // phase A: warped samples of the tile + halo for the group's planes
                const float d0 = __ldg(&L.planes[k0].d);
                const float d1 = __ldg(&L.planes[k0 + np - 1].d);
                int bad = 0;
#pragma unroll 3
                for (int i = 0; i < G::PPT; ++i) {
                    int p = tid + i * NT;
                    if (p < NPOS) {
                        float4 a = Aj[p];
                        float w0 = warp_sample<HALF>(C, fmaf(d0, a.x, C.t[0]), fmaf(d0, a.y, C.t[1]), fmaf(d0, a.z, C.t[2]));
                        if constexpr (KP == 2) {  // both gathers in flight before the stores
                            float w1 = warp_sample<HALF>(C, fmaf(d1, a.x, C.t[0]), fmaf(d1, a.y, C.t[1]),
                                                         fmaf(d1, a.z, C.t[2]));
                            bad |= isnan(w0) | isnan(w1);
                            int hy = p / HWL, hx = p - hy * HWL;
                            Ws[hy * WS + hx] = w0;
                            Ws[HH * WS + hy * WS + hx] = w1;
                        } else {
                            bad |= isnan(w0);
                            int hy = p / HWL, hx = p - hy * HWL;
                            Ws[hy * WS + hx] = w0;
                        }
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
        tile_finished(L, true);
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
    tile_finished(L, *s_flag != 0);
}

// One work item of a level: stage the matching cameras in shared memory and
// run the tile routine for the level's window radius and image storage.
template <int TH, int KP>
__device__ __forceinline__ void sweep_item(const LevelD& L, int half, int item, CamS* cams, unsigned char* smem,
                                           int* s_flag) {
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
    if (half) {
        switch (L.rho) {
            case 2: sweep_tile<2, true, TH, KP>(L, cams, item, smem, s_flag); break;
            case 3: sweep_tile<3, true, TH, KP>(L, cams, item, smem, s_flag); break;
            default: sweep_tile<4, true, TH, KP>(L, cams, item, smem, s_flag); break;
        }
    } else {
        switch (L.rho) {
            case 2: sweep_tile<2, false, TH, KP>(L, cams, item, smem, s_flag); break;
            case 3: sweep_tile<3, false, TH, KP>(L, cams, item, smem, s_flag); break;
            default: sweep_tile<4, false, TH, KP>(L, cams, item, smem, s_flag); break;
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

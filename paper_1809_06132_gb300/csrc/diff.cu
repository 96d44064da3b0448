// Differentiable plane sweep: soft-argmin depth over the plane hypotheses
// and its gradient with respect to the images and the matching cameras'
// poses.  Not in the paper: the winner-take-all depth (Sec. III-A) is
// piecewise constant, so for gradients the planes are averaged with softmax
// weights of their aggregated costs:
//   s_k = exp(-C_k / T) / sum over valid k' of exp(-C_k' / T)
//   range = 1 / sum_k s_k rho_k,   rho_k = (n_k . r) / d_k,
// and the soft minimum S = -T log sum_k exp(-C_k / T) is a second output.
// C_k = min over the matching cameras of (1 - ZNCC) / 2 (lowest camera index
// on a tie), exactly the sweep's cost but on real-valued images.
//
// Kernels (one CTA per 16 x 16 output tile, one thread per output pixel):
//   soft_fwd_kernel  per pair of planes and camera, warp the tile + window
//                    halo into shared memory; two-pass window ZNCC per pixel
//                    (both planes on packed FP32 pairs); minimum over
//                    cameras; online softmax over planes.
//   soft_bwd_kernel  recomputes the same costs (bit-identical) while keeping
//                    each warped sample's bilinear cell and pose derivative,
//                    forms dL/dC_k, spreads dL/dZNCC over both windows as
//                    separable box sums of per-pixel coefficients, then per
//                    warped halo sample scatters dL/dI to the 4 bilinear
//                    texels and adds dL/dw times the sample's pose
//                    derivative to a left perturbation (w, v) of each
//                    ref_to_cam pose (CTA reduction, FP64 atomics).
#include <cmath>
#include <cstring>
#include <vector>

#include "sweep_dev.cuh"

namespace ps {
int build_rays(const ps_camera& cam, float4* rays, double* max_angle);

namespace {

constexpr int DT = 16;                 // output tile edge
constexpr int DNT = DT * DT;           // threads per CTA

struct DiffCam {
    float R[9], t[3];
    CamF c;
    const float* img;
};

struct DiffP {
    int W, H, rho, K, n_cams;
    float T;
    const float4* rays;
    const PlaneD* planes;
    const float* ref;
    DiffCam cams[PS_MAX_CAMS];
};

// Projection of X_j (camera frame) with the unified model and distortion;
// false where the point does not project (the sweep's validity rules).
__device__ __forceinline__ bool project_f(const CamF& c, float X, float Y, float Z, float* u, float* v,
                                          float* n_out) {
    float n = sqrtf(fmaf(X, X, fmaf(Y, Y, Z * Z)));
    float inv = 1.0f / fmaf(c.xi, n, Z);
    float mx = X * inv, my = Y * inv;
    float r2 = fmaf(mx, mx, my * my);
    float rad = fmaf(r2, fmaf(c.k2, r2, c.k1), 1.0f);
    float mxy = mx * my;
    float xd = fmaf(mx, rad, fmaf(2.0f * c.p1, mxy, c.p2 * fmaf(2.0f * mx, mx, r2)));
    float yd = fmaf(my, rad, fmaf(c.p1, fmaf(2.0f * my, my, r2), 2.0f * c.p2 * mxy));
    *u = fmaf(c.fx, xd, c.cx);
    *v = fmaf(c.fy, yd, c.cy);
    *n_out = n;
    return (Z > c.lim * n) && (r2 <= c.r2_max);
}

// g = J^T (gu, gv) for the projection Jacobian J = d(u, v)/dX at X (camera
// frame), by reverse-mode differentiation of project_f instead of forming J:
// the adjoints of the distorted point, of the normalised point (mx, my),
// then of X through mx = X / den, my = Y / den, den = xi |X| + Z.
__device__ __forceinline__ void project_vjp_f(const CamF& c, float X, float Y, float Z, float gu, float gv,
                                              float g[3]) {
    const float n = sqrtf(fmaf(X, X, fmaf(Y, Y, Z * Z)));
    const float id = 1.0f / fmaf(c.xi, n, Z);
    const float mx = X * id, my = Y * id;
    const float r2 = fmaf(mx, mx, my * my);
    const float rad = fmaf(r2, fmaf(c.k2, r2, c.k1), 1.0f), drad = fmaf(2.0f * c.k2, r2, c.k1);
    // d(xd, yd)/d(mx, my) = [[a, b], [b, d]]
    const float a = rad + 2.0f * mx * mx * drad + 2.0f * c.p1 * my + 6.0f * c.p2 * mx;
    const float b = 2.0f * mx * my * drad + 2.0f * c.p1 * mx + 2.0f * c.p2 * my;
    const float d = rad + 2.0f * my * my * drad + 6.0f * c.p1 * my + 2.0f * c.p2 * mx;
    const float gxd = gu * c.fx, gyd = gv * c.fy;
    const float gmx = fmaf(gxd, a, gyd * b), gmy = fmaf(gxd, b, gyd * d);
    const float sden = fmaf(gmx, mx, gmy * my) * id;  // -dL/dden
    const float xn = c.xi / n;                        // d(xi n)/dX = xi X / n
    g[0] = fmaf(gmx, id, -sden * xn * X);
    g[1] = fmaf(gmy, id, -sden * xn * Y);
    g[2] = -sden * fmaf(xn, Z, 1.0f);
}

// The warp of halo position (gx, gy) through plane P into camera C: the
// point in the camera frame, the pixel and the bilinear sample (NaN when
// invalid: no ray, plane behind the ray, no projection, outside the image).
struct Warp {
    float X, Y, Z, u, v, w;
};

// n . r of a plane and a ray.  The plane's offset along the ray, and the
// bilinear blend below, are written with explicit roundings so that every
// kernel computes the same samples (the costs decide integers: a camera, a
// plane) whatever contractions the compiler would choose in each.
__device__ __forceinline__ float plane_dot(const PlaneD& pl, const float4& r) {
    return __fmaf_rn(pl.nz, r.z, __fmaf_rn(pl.ny, r.y, __fmul_rn(pl.nx, r.x)));
}

__device__ __forceinline__ float bilerp(float ax, float ay, float i00, float i10, float i01, float i11) {
    const float bx = __fsub_rn(1.0f, ax), by = __fsub_rn(1.0f, ay);
    const float top = __fmaf_rn(ax, i10, __fmul_rn(bx, i00));
    const float bot = __fmaf_rn(ax, i11, __fmul_rn(bx, i01));
    return __fmaf_rn(ay, bot, __fmul_rn(by, top));
}

// Bilinear sample of camera C at (u, v), NaN outside [0, W-1] x [0, H-1].
__device__ __forceinline__ float sample_uv(const DiffCam& C, float u, float v) {
    if (!(u >= 0.0f && u <= (float)(C.c.width - 1) && v >= 0.0f && v <= (float)(C.c.height - 1)))
        return __int_as_float(0x7fc00000);
    int x0 = (int)floorf(u), y0 = (int)floorf(v);
    int x1 = min(x0 + 1, C.c.width - 1), y1 = min(y0 + 1, C.c.height - 1);
    float ax = u - (float)x0, ay = v - (float)y0;
    const float* I = C.img;
    return bilerp(ax, ay, I[(size_t)y0 * C.c.width + x0], I[(size_t)y0 * C.c.width + x1],
                  I[(size_t)y1 * C.c.width + x0], I[(size_t)y1 * C.c.width + x1]);
}

__device__ __forceinline__ Warp warp_at(const DiffP& P, const DiffCam& C, const PlaneD& pl, int gx, int gy) {
    const float nan = __int_as_float(0x7fc00000);
    Warp o{0.f, 0.f, 0.f, 0.f, 0.f, nan};
    if (gx < 0 || gy < 0 || gx >= P.W || gy >= P.H) return o;
    float4 r = P.rays[(size_t)gy * P.W + gx];
    float nr = plane_dot(pl, r);
    if (!(nr > 0.0f)) return o;
    float lam = pl.d / nr;
    float x = lam * r.x, y = lam * r.y, z = lam * r.z;
    o.X = fmaf(C.R[0], x, fmaf(C.R[1], y, fmaf(C.R[2], z, C.t[0])));
    o.Y = fmaf(C.R[3], x, fmaf(C.R[4], y, fmaf(C.R[5], z, C.t[1])));
    o.Z = fmaf(C.R[6], x, fmaf(C.R[7], y, fmaf(C.R[8], z, C.t[2])));
    float n;
    if (!project_f(C.c, o.X, o.Y, o.Z, &o.u, &o.v, &n)) return o;
    o.w = sample_uv(C, o.u, o.v);
    return o;
}

// warp_at for two planes at once (lane x: p0, lane y: p1): the samples only,
// with the transform and the projection on packed FP32 pairs.  Per lane
// every operation and rounding is that of warp_at (2 m = m + m exactly), so
// each sample is bit-identical to warp_at's.
__device__ __forceinline__ float2 warp_pair(const DiffP& P, const DiffCam& C, const PlaneD& p0, const PlaneD& p1,
                                            int gx, int gy) {
    const float nan = __int_as_float(0x7fc00000);
    if (gx < 0 || gy < 0 || gx >= P.W || gy >= P.H) return make_float2(nan, nan);
    const float4 r = P.rays[(size_t)gy * P.W + gx];
    const float nr0 = plane_dot(p0, r), nr1 = plane_dot(p1, r);
    const bool f0 = nr0 > 0.0f, f1 = nr1 > 0.0f;
    if (!(f0 || f1)) return make_float2(nan, nan);
    const float2 lam = make_float2(p0.d / nr0, p1.d / nr1);
    const float2 x = mul2(lam, dup2(r.x)), y = mul2(lam, dup2(r.y)), z = mul2(lam, dup2(r.z));
    const float2 X = fma2(dup2(C.R[0]), x, fma2(dup2(C.R[1]), y, fma2(dup2(C.R[2]), z, dup2(C.t[0]))));
    const float2 Y = fma2(dup2(C.R[3]), x, fma2(dup2(C.R[4]), y, fma2(dup2(C.R[5]), z, dup2(C.t[1]))));
    const float2 Z = fma2(dup2(C.R[6]), x, fma2(dup2(C.R[7]), y, fma2(dup2(C.R[8]), z, dup2(C.t[2]))));
    const CamF& c = C.c;
    const float2 n2 = fma2(X, X, fma2(Y, Y, mul2(Z, Z)));
    const float2 n = make_float2(sqrtf(n2.x), sqrtf(n2.y));
    const float2 den = fma2(dup2(c.xi), n, Z);
    const float2 inv = make_float2(1.0f / den.x, 1.0f / den.y);
    const float2 mx = mul2(X, inv), my = mul2(Y, inv);
    const float2 r2 = fma2(mx, mx, mul2(my, my));
    const float2 rad = fma2(r2, fma2(dup2(c.k2), r2, dup2(c.k1)), dup2(1.0f));
    const float2 mxy = mul2(mx, my);
    const float2 xd = fma2(mx, rad, fma2(dup2(2.0f * c.p1), mxy, mul2(dup2(c.p2), fma2(add2(mx, mx), mx, r2))));
    const float2 yd = fma2(my, rad, fma2(dup2(c.p1), fma2(add2(my, my), my, r2), mul2(dup2(2.0f * c.p2), mxy)));
    const float2 u = fma2(dup2(c.fx), xd, dup2(c.cx)), v = fma2(dup2(c.fy), yd, dup2(c.cy));
    const float2 ln = mul2(dup2(c.lim), n);
    const bool g0 = f0 && (Z.x > ln.x) && (r2.x <= c.r2_max), g1 = f1 && (Z.y > ln.y) && (r2.y <= c.r2_max);
    return make_float2(g0 ? sample_uv(C, u.x, v.x) : nan, g1 ? sample_uv(C, u.y, v.y) : nan);
}

// Two-pass ZNCC of the pixel's window: reference samples R and warped
// samples Wv in the halo layout (row stride DS).  False when a sample is
// invalid or a window is flat.
struct Zn {
    float z, ma, mb, va, vb, sab;
};

// Shared-memory row stride of the halo buffers: 48 = 16 (mod 32), so the two
// output rows of a warp (16 pixels each) read disjoint banks.
constexpr int DS = 48;

template <int RHO>
__device__ __forceinline__ bool window_zncc(const float* R, const float* Wv, int lx, int ly, Zn* o) {
    constexpr int N = (2 * RHO + 1) * (2 * RHO + 1);
    float sa = 0.f, sb = 0.f;
    bool ok = true;
#pragma unroll
    for (int dy = 0; dy <= 2 * RHO; ++dy)
#pragma unroll
        for (int dx = 0; dx <= 2 * RHO; ++dx) {
            const int q = (ly + dy) * DS + lx + dx;
            float b = Wv[q];
            ok &= !isnan(b);
            sa += R[q];
            sb += b;
        }
    if (!ok) return false;
    float ma = sa / (float)N, mb = sb / (float)N;
    float cov = 0.f, va = 0.f, vb = 0.f;
#pragma unroll
    for (int dy = 0; dy <= 2 * RHO; ++dy)
#pragma unroll
        for (int dx = 0; dx <= 2 * RHO; ++dx) {
            const int q = (ly + dy) * DS + lx + dx;
            float ea = R[q] - ma, eb = Wv[q] - mb;
            cov = fmaf(ea, eb, cov);
            va = fmaf(ea, ea, va);
            vb = fmaf(eb, eb, vb);
        }
    if (va < (float)N * 1e-8f || vb < (float)N * 1e-8f) return false;
    o->sab = sqrtf(va * vb);
    o->z = cov / o->sab;
    o->ma = ma;
    o->mb = mb;
    o->va = va;
    o->vb = vb;
    return true;
}

// window_zncc for two planes at once: warped pairs Wv (lane x: the first
// plane, lane y: the second), one reference window.  The reference sums are
// shared; per lane every sum and rounding is window_zncc's, so z is
// bit-identical to it.  ok0 / ok1: the lanes' validity.
template <int RHO>
__device__ __forceinline__ float2 window_zncc2(const float* R, const float2* Wv, int lx, int ly, bool* ok0, bool* ok1) {
    constexpr int N = (2 * RHO + 1) * (2 * RHO + 1);
    float sa = 0.f;
    float2 sb = dup2(0.f);
    bool v0 = true, v1 = true;
#pragma unroll
    for (int dy = 0; dy <= 2 * RHO; ++dy)
#pragma unroll
        for (int dx = 0; dx <= 2 * RHO; ++dx) {
            const int q = (ly + dy) * DS + lx + dx;
            const float2 b = Wv[q];
            v0 &= !isnan(b.x);
            v1 &= !isnan(b.y);
            sa += R[q];
            sb = add2(sb, b);
        }
    *ok0 = *ok1 = false;
    if (!(v0 || v1)) return dup2(0.f);
    const float ma = sa / (float)N;
    const float2 nmb = make_float2(-(sb.x / (float)N), -(sb.y / (float)N));
    float va = 0.f;
    float2 cov = dup2(0.f), vb = dup2(0.f);
#pragma unroll
    for (int dy = 0; dy <= 2 * RHO; ++dy)
#pragma unroll
        for (int dx = 0; dx <= 2 * RHO; ++dx) {
            const int q = (ly + dy) * DS + lx + dx;
            const float ea = R[q] - ma;
            const float2 eb = add2(Wv[q], nmb);
            cov = fma2(dup2(ea), eb, cov);
            va = fmaf(ea, ea, va);
            vb = fma2(eb, eb, vb);
        }
    const float lim = (float)N * 1e-8f;
    *ok0 = v0 && !(va < lim || vb.x < lim);
    *ok1 = v1 && !(va < lim || vb.y < lim);
    return make_float2(cov.x / sqrtf(va * vb.x), cov.y / sqrtf(va * vb.y));
}

// Window 5: three CTAs per SM (80 registers, a small spill) measured faster
// than two without the limit.
template <int RHO>
__global__ void __launch_bounds__(DNT, RHO == 2 ? 3 : 1) soft_fwd_kernel(const __grid_constant__ DiffP P, float* range, float* cost,
                                                      float* aux) {
    constexpr int HW = DT + 2 * RHO, NPOS = HW * HW;
    __shared__ float Rs[HW * DS];
    __shared__ float2 W2[HW * DS];  // warped samples of a pair of planes
    const int tid = threadIdx.x, lx = tid % DT, ly = tid / DT;
    const int x0 = blockIdx.x * DT - RHO, y0 = blockIdx.y * DT - RHO;
    const int gx = blockIdx.x * DT + lx, gy = blockIdx.y * DT + ly;
    for (int p = tid; p < NPOS; p += DNT) {
        const int hx = p % HW, hy = p / HW, x = x0 + hx, y = y0 + hy;
        Rs[hy * DS + hx] = (x >= 0 && y >= 0 && x < P.W && y < P.H) ? P.ref[(size_t)y * P.W + x] : 0.0f;
    }
    const bool in = gx < P.W && gy < P.H;
    float4 ray = in ? P.rays[(size_t)gy * P.W + gx] : make_float4(0.f, 0.f, 0.f, 0.f);
    const bool use = in && gx >= RHO && gy >= RHO && gx < P.W - RHO && gy < P.H - RHO && !isnan(ray.x);
    const float inf = __int_as_float(0x7f800000);
    float cmin = inf, Z = 0.f, Nr = 0.f;
    // planes in pairs (k, k + 1), warped and matched together on packed FP32
    for (int k = 0; k < P.K; k += 2) {
        const int np = min(2, P.K - k);
        const PlaneD pl0 = P.planes[k], pl1 = P.planes[k + np - 1];
        float best[2] = {inf, inf};
        for (int j = 0; j < P.n_cams; ++j) {
            __syncthreads();
            for (int p = tid; p < NPOS; p += DNT) {
                const int hx = p % HW, hy = p / HW;
                W2[hy * DS + hx] = warp_pair(P, P.cams[j], pl0, pl1, x0 + hx, y0 + hy);
            }
            __syncthreads();
            if (use) {
                bool ok0, ok1;
                const float2 z = window_zncc2<RHO>(Rs, W2, lx, ly, &ok0, &ok1);
                const float c0 = 0.5f * (1.0f - z.x), c1 = 0.5f * (1.0f - z.y);
                if (ok0 && c0 < best[0]) best[0] = c0;
                if (ok1 && c1 < best[1]) best[1] = c1;
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (q >= np || !(best[q] < inf)) continue;
            const PlaneD& pl = q == 0 ? pl0 : pl1;
            const float bq = best[q];
            float rho_k = plane_dot(pl, ray) / pl.d;
            if (bq < cmin) {  // rescale the running sums to the new minimum
                float f = cmin < inf ? __expf(-(cmin - bq) / P.T) : 0.f;
                Z *= f;
                Nr *= f;
                cmin = bq;
            }
            float e = __expf(-(bq - cmin) / P.T);
            Z += e;
            Nr = fmaf(e, rho_k, Nr);
        }
    }
    if (!in) return;
    const size_t o = (size_t)gy * P.W + gx;
    const bool ok = cmin < inf;
    range[o] = ok ? Z / Nr : 0.f;
    if (cost) cost[o] = ok ? cmin - P.T * logf(Z) : 0.f;
    if (aux) {
        aux[3 * o] = ok ? cmin : inf;
        aux[3 * o + 1] = Z;
        aux[3 * o + 2] = ok ? Nr / Z : 0.f;
    }
}

struct GradOut {
    float* cam[PS_MAX_CAMS];
};

// Shared-memory layout of the backward kernel (floats), for window radius
// RHO and nc matching cameras.  nf = 4 nc + 3 coefficient fields.
template <int RHO>
struct BwdLayout {
    static constexpr int HW = DT + 2 * RHO, NPOS = HW * HW, BUF = HW * DS;
    static constexpr int FS = DT + 1;  // field row stride
    static constexpr int HS = HW + 1;  // horizontal-sum row stride (odd: the row-per-thread writes are conflict-free)
    __host__ __device__ static constexpr int nf(int nc) { return 4 * nc + 3; }
    // Rs, gR, nc x (Ws, gW), chain data (8 floats + 1 cell per sample and
    // camera), horizontal box sums [nf][DT][HS], fields / vertical box sums
    // [nf][NPOS] (the fields [nf][DT][FS] are dead once the horizontal sums exist)
    __host__ __device__ static constexpr size_t floats(int nc) {
        return (size_t)(2 + 2 * nc) * BUF + (size_t)nc * NPOS * 9 + (size_t)nf(nc) * DT * HS +
               (size_t)nf(nc) * NPOS;
    }
    static_assert(NPOS >= DT * FS, "the vertical sums reuse the field storage");
};

// The sample of halo position (gx, gy) through plane P in camera C, with
// what the chain rule needs later: the bilinear cell (y0 << 16 | x0, -1 when
// invalid), its weights (ax, ay) and m = (X x g, g), g = J^T (dw/du, dw/dv),
// J the 2 x 3 projection Jacobian at X (camera frame); gw m is then the
// sample's contribution to the gradient of a left perturbation (w, v) of
// ref_to_cam.  w is computed exactly as in the forward (warp_at).
struct WarpJ {
    float w;
    int cell;
    float ax, ay;
    float m[6];
};

__device__ __forceinline__ WarpJ warp_jac(const DiffP& P, const DiffCam& C, const PlaneD& pl, int gx, int gy) {
    WarpJ o;
    const Warp wp = warp_at(P, C, pl, gx, gy);
    o.w = wp.w;
    o.cell = -1;
    o.ax = o.ay = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) o.m[i] = 0.f;
    if (isnan(wp.w)) return o;
    const int Wc = C.c.width;
    const int xa = (int)floorf(wp.u), ya = (int)floorf(wp.v);
    const int xb = min(xa + 1, Wc - 1), yb = min(ya + 1, C.c.height - 1);
    const float ax = wp.u - (float)xa, ay = wp.v - (float)ya;
    const float* I = C.img;
    const float i00 = I[(size_t)ya * Wc + xa], i10 = I[(size_t)ya * Wc + xb];
    const float i01 = I[(size_t)yb * Wc + xa], i11 = I[(size_t)yb * Wc + xb];
    const float dwdu = (1.f - ay) * (i10 - i00) + ay * (i11 - i01);
    const float dwdv = (1.f - ax) * (i01 - i00) + ax * (i11 - i10);
    float g[3];
    project_vjp_f(C.c, wp.X, wp.Y, wp.Z, dwdu, dwdv, g);
    o.cell = (ya << 16) | xa;
    o.ax = ax;
    o.ay = ay;
    o.m[0] = wp.Y * g[2] - wp.Z * g[1];
    o.m[1] = wp.Z * g[0] - wp.X * g[2];
    o.m[2] = wp.X * g[1] - wp.Y * g[0];
    o.m[3] = g[0];
    o.m[4] = g[1];
    o.m[5] = g[2];
    return o;
}

// Backward of the soft sweep for one 16 x 16 tile.  Per plane:
//  1. warp the halo for every camera (samples + chain data, warp_jac);
//  2. per pixel, the plane's cost and winning camera jb as in the forward,
//     dL/dC, and the ZNCC gradient coefficients ka = gz / sqrt(va vb),
//     kz_a = gz z / va, kz_b = gz z / vb (gz = dL/dZNCC);
//  3. window gradients as box sums.  For a window sample q of pixel p,
//       dZNCC/da_q = (b_q - mb) / sqrt(va vb) - z (a_q - ma) / va   (a: ref)
//       dZNCC/db_q = (a_q - ma) / sqrt(va vb) - z (b_q - mb) / vb   (b: camera jb)
//     so, summed over the pixels whose window holds q,
//       gW_j(q) = a_q A1_j - A2_j - b_q A3_j + A4_j
//       gR(q)  += sum_j b_j(q) A1_j - B1 - a_q B2 + B3
//     with A1_j..A4_j the (2 RHO + 1)^2 box sums of ka, ka ma, kz_b, kz_b mb
//     over pixels with jb = j, and B1..B3 those of ka mb, kz_a, kz_a ma.
//     Intensities are taken relative to a per-tile centre (a) and a
//     per-plane, per-camera centre (b), which leaves every difference
//     unchanged and keeps the products small.  The box sums are separable
//     (rows, then columns) in shared memory: no atomics;
//  4. chain every sample with dL/dw != 0: dL/dI to its four texels (global
//     atomics) and gw m to the pose accumulators.
// After the planes: dL/dref of the halo (global atomics) and the CTA's pose
// gradient (FP64 atomics).
template <int RHO>
__global__ void __launch_bounds__(DNT) soft_bwd_kernel(const __grid_constant__ DiffP P, const float* aux,
                                                      const float* g_range, const float* g_cost, float* g_ref,
                                                      const __grid_constant__ GradOut G, double* g_pose) {
    using BL = BwdLayout<RHO>;
    constexpr int HW = BL::HW, NPOS = BL::NPOS, BUF = BL::BUF, FS = BL::FS, HS = BL::HS;
    const int nc = P.n_cams, nf = BL::nf(nc);
    extern __shared__ float sm[];
    float* Rs = sm;                                   // reference
    float* gR = Rs + BUF;                             // dL/dref, summed over planes
    float* Ws = gR + BUF;                             // [nc] warped samples of the current plane
    float* gW = Ws + nc * BUF;                        // [nc] dL/dw of the current plane
    float* Cm = gW + nc * BUF;                        // [nc][8][NPOS] m[0..5], ax, ay
    int* Cc = reinterpret_cast<int*>(Cm + nc * 8 * NPOS);  // [nc][NPOS] bilinear cell
    float* Hx = reinterpret_cast<float*>(Cc + nc * NPOS);  // [nf][DT][HS] horizontal box sums
    float* FV = Hx + nf * DT * HS;                    // [nf][DT][FS] fields, then [nf][NPOS] box sums
    __shared__ float red[DNT / 32][6 * PS_MAX_CAMS];
    const int tid = threadIdx.x, lx = tid % DT, ly = tid / DT;
    const int x0 = blockIdx.x * DT - RHO, y0 = blockIdx.y * DT - RHO;
    const int gx = blockIdx.x * DT + lx, gy = blockIdx.y * DT + ly;
    for (int p = tid; p < NPOS; p += DNT) {
        const int hx = p % HW, hy = p / HW, x = x0 + hx, y = y0 + hy;
        Rs[hy * DS + hx] = (x >= 0 && y >= 0 && x < P.W && y < P.H) ? P.ref[(size_t)y * P.W + x] : 0.0f;
        gR[hy * DS + hx] = 0.f;
    }
    const bool in = gx < P.W && gy < P.H;
    const size_t o = in ? (size_t)gy * P.W + gx : 0;
    float4 ray = in ? P.rays[o] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float inf = __int_as_float(0x7f800000);
    float cmin = inf, Z = 1.f, E = 0.f, gr = 0.f, gs = 0.f;
    if (in) {
        cmin = aux[3 * o];
        Z = aux[3 * o + 1];
        E = aux[3 * o + 2];
        gr = g_range ? g_range[o] : 0.f;
        gs = g_cost ? g_cost[o] : 0.f;
    }
    const bool use = in && gx >= RHO && gy >= RHO && gx < P.W - RHO && gy < P.H - RHO && !isnan(ray.x) &&
                     cmin < inf && (gr != 0.f || gs != 0.f);
    const float gE = use ? -gr / (E * E) : 0.f;
    float pose_acc[6 * PS_MAX_CAMS];
#pragma unroll
    for (int i = 0; i < 6 * PS_MAX_CAMS; ++i) pose_acc[i] = 0.f;
    __syncthreads();
    const int qc = (RHO + DT / 2) * DS + RHO + DT / 2;  // centre of the tile
    const float ca = Rs[qc];
    for (int k = 0; k < P.K; ++k) {
        const PlaneD pl = P.planes[k];
        __syncthreads();  // the previous plane's chain is done with gW and the chain data
        // 1. samples and chain data of the halo
        for (int p = tid; p < NPOS; p += DNT) {
            const int hx = p % HW, hy = p / HW;
            for (int j = 0; j < nc; ++j) {
                const WarpJ wj = warp_jac(P, P.cams[j], pl, x0 + hx, y0 + hy);
                Ws[j * BUF + hy * DS + hx] = wj.w;
                float* cm = Cm + j * 8 * NPOS + p;
#pragma unroll
                for (int i = 0; i < 6; ++i) cm[i * NPOS] = wj.m[i];
                cm[6 * NPOS] = wj.ax;
                cm[7 * NPOS] = wj.ay;
                Cc[j * NPOS + p] = wj.cell;
            }
        }
        __syncthreads();
        // the per-camera centre of this plane's warped samples (a broadcast read)
        auto centre = [&](int j) {
            const float c = Ws[j * BUF + qc];
            return isnan(c) ? 0.f : c;
        };
        // 2. the pixel's cost for this plane (as in the forward), its camera and coefficients
        float best = inf;
        int jb = -1;
        Zn zb;
        for (int j = 0; use && j < nc; ++j) {
            Zn zn;
            if (window_zncc<RHO>(Rs, Ws + j * BUF, lx, ly, &zn)) {
                float c = 0.5f * (1.0f - zn.z);
                if (c < best) {
                    best = c;
                    jb = j;
                    zb = zn;
                }
            }
        }
        float ka = 0.f, kza = 0.f, kzb = 0.f, mac = 0.f, mbc = 0.f;
        if (jb >= 0) {
            const float s = __expf(-(best - cmin) / P.T) / Z;
            const float rho_k = plane_dot(pl, ray) / pl.d;
            const float gC = gE * (-s * (rho_k - E) / P.T) + gs * s;
            const float gz = -0.5f * gC;
            ka = gz / zb.sab;
            kza = gz * zb.z / zb.va;
            kzb = gz * zb.z / zb.vb;
            mac = zb.ma - ca;
            mbc = zb.mb - centre(jb);
        }
        {
            float* F = FV + ly * FS + lx;
            for (int j = 0; j < nc; ++j) {
                const bool mine = j == jb;
                F[(4 * j + 0) * DT * FS] = mine ? ka : 0.f;
                F[(4 * j + 1) * DT * FS] = mine ? ka * mac : 0.f;
                F[(4 * j + 2) * DT * FS] = mine ? kzb : 0.f;
                F[(4 * j + 3) * DT * FS] = mine ? kzb * mbc : 0.f;
            }
            F[(4 * nc + 0) * DT * FS] = ka * mbc;
            F[(4 * nc + 1) * DT * FS] = kza;
            F[(4 * nc + 2) * DT * FS] = kza * mac;
        }
        __syncthreads();
        // 3a. horizontal box sums: halo column c collects pixels c - 2 RHO .. c of the row.
        // Direct sums, not running ones: coefficients of low-texture windows are
        // large, and a running sum would leave their rounding residue where the
        // exact sum is zero
        for (int it = tid; it < nf * DT; it += DNT) {
            const float* fr = FV + it * FS;
            float* hr = Hx + it * HS;
            float v[DT];
#pragma unroll
            for (int x = 0; x < DT; ++x) v[x] = fr[x];
#pragma unroll
            for (int c = 0; c < HW; ++c) {
                float acc = 0.f;
#pragma unroll
                for (int x = (c - 2 * RHO > 0 ? c - 2 * RHO : 0); x <= (c < DT - 1 ? c : DT - 1); ++x) acc += v[x];
                hr[c] = acc;
            }
        }
        __syncthreads();
        // 3b. vertical box sums: halo row r collects rows r - 2 RHO .. r
        for (int it = tid; it < nf * HW; it += DNT) {
            const int f = it / HW, c = it - f * HW;
            const float* hc = Hx + f * DT * HS + c;
            float* vc = FV + f * NPOS + c;
            float v[DT];
#pragma unroll
            for (int y = 0; y < DT; ++y) v[y] = hc[y * HS];
#pragma unroll
            for (int r = 0; r < HW; ++r) {
                float acc = 0.f;
#pragma unroll
                for (int y = (r - 2 * RHO > 0 ? r - 2 * RHO : 0); y <= (r < DT - 1 ? r : DT - 1); ++y) acc += v[y];
                vc[r * HW] = acc;
            }
        }
        __syncthreads();
        // 3c. per halo sample: dL/dw of every camera and this plane's part of dL/dref
        for (int p = tid; p < NPOS; p += DNT) {
            const int hx = p % HW, hy = p / HW, q = hy * DS + hx;
            const float* V = FV + p;
            const float a = Rs[q] - ca;
            float g = -V[(4 * nc + 0) * NPOS] - a * V[(4 * nc + 1) * NPOS] + V[(4 * nc + 2) * NPOS];
            for (int j = 0; j < nc; ++j) {
                const float A1 = V[(4 * j + 0) * NPOS], A2 = V[(4 * j + 1) * NPOS];
                const float A3 = V[(4 * j + 2) * NPOS], A4 = V[(4 * j + 3) * NPOS];
                const float bw = Ws[j * BUF + q];
                float gw = 0.f;
                if (!isnan(bw)) {  // an invalid sample is in no used window: all its sums are zero
                    const float b = bw - centre(j);
                    gw = a * A1 - A2 - b * A3 + A4;
                    g += b * A1;
                }
                gW[j * BUF + q] = gw;
            }
            gR[q] += g;
        }
        __syncthreads();
        // 4. chain dL/dw of every warped halo sample to the image and the pose
        for (int p = tid; p < NPOS; p += DNT) {
            const int hx = p % HW, hy = p / HW;
#pragma unroll
            for (int j = 0; j < PS_MAX_CAMS; ++j) {
                if (j >= nc) break;
                const float gw = gW[j * BUF + hy * DS + hx];
                const int cell = Cc[j * NPOS + p];
                if (gw == 0.f || cell < 0) continue;
                const float* cm = Cm + j * 8 * NPOS + p;
#pragma unroll
                for (int i = 0; i < 6; ++i) pose_acc[6 * j + i] = fmaf(gw, cm[i * NPOS], pose_acc[6 * j + i]);
                if (G.cam[j]) {
                    const DiffCam& C = P.cams[j];
                    const int Wc = C.c.width, xa = cell & 0xffff, ya = cell >> 16;
                    if (!PS_DCHECK(xa < Wc && ya < C.c.height, CHK_GATHER)) continue;
                    const int xb = min(xa + 1, Wc - 1), yb = min(ya + 1, C.c.height - 1);
                    const float ax = cm[6 * NPOS], ay = cm[7 * NPOS];
                    float* Gj = G.cam[j];
                    atomicAdd(&Gj[(size_t)ya * Wc + xa], gw * (1.f - ax) * (1.f - ay));
                    atomicAdd(&Gj[(size_t)ya * Wc + xb], gw * ax * (1.f - ay));
                    atomicAdd(&Gj[(size_t)yb * Wc + xa], gw * (1.f - ax) * ay);
                    atomicAdd(&Gj[(size_t)yb * Wc + xb], gw * ax * ay);
                }
            }
        }
    }
    __syncthreads();
    if (g_ref)
        for (int p = tid; p < NPOS; p += DNT) {
            const int hx = p % HW, hy = p / HW;
            float g = gR[hy * DS + hx];
            if (g != 0.f && PS_DCHECK(x0 + hx >= 0 && y0 + hy >= 0 && x0 + hx < P.W && y0 + hy < P.H, CHK_PIXEL))
                atomicAdd(&g_ref[(size_t)(y0 + hy) * P.W + (x0 + hx)], g);
        }
    if (g_pose) {
        const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
        for (int i = 0; i < 6 * PS_MAX_CAMS; ++i) {
            float v = pose_acc[i];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0) red[wid][i] = v;
        }
        __syncthreads();
        if (tid < 6 * P.n_cams) {
            double s = 0.0;
            for (int w = 0; w < DNT / 32; ++w) s += (double)red[w][tid];
            atomicAdd(&g_pose[tid], s);
        }
    }
}

}  // namespace
}  // namespace ps

using namespace ps;

struct psdiff_s {
    ps_camera ref;
    int n_cams = 0;
    ps_camera cams[PS_MAX_CAMS];
    int rho = 0, K = 0;
    double T = 0.05;
    float4* rays = nullptr;
    PlaneD* planes = nullptr;
};

namespace {

void free_diff(psdiff_t* h) {
    if (!h) return;
    cudaFree(h->rays);
    cudaFree(h->planes);
    delete h;
}

int fill_params(const psdiff_t* h, const float* const* images, const ps_pose* ref_to_cam, DiffP& P) {
    std::memset(&P, 0, sizeof(P));
    P.W = h->ref.width;
    P.H = h->ref.height;
    P.rho = h->rho;
    P.K = h->K;
    P.n_cams = h->n_cams;
    P.T = (float)h->T;
    P.rays = h->rays;
    P.planes = h->planes;
    PS_ARG(images != nullptr && images[0] != nullptr, "psdiff: images[0] is NULL");
    PS_ARG(ref_to_cam != nullptr, "psdiff: ref_to_cam is NULL");
    P.ref = images[0];
    for (int j = 0; j < h->n_cams; ++j) {
        PS_ARG(images[1 + j] != nullptr, "psdiff: images[%d] is NULL", 1 + j);
        for (int i = 0; i < 12; ++i)
            PS_ARG(std::isfinite(i < 9 ? ref_to_cam[j].R[i] : ref_to_cam[j].t[i - 9]), "psdiff: pose %d not finite", j);
        for (int i = 0; i < 9; ++i) P.cams[j].R[i] = (float)ref_to_cam[j].R[i];
        for (int i = 0; i < 3; ++i) P.cams[j].t[i] = (float)ref_to_cam[j].t[i];
        P.cams[j].c = to_camf(h->cams[j]);
        P.cams[j].img = images[1 + j];
    }
    return PS_OK;
}

}  // namespace

extern "C" int psdiff_create(const ps_diff_desc* d, psdiff_t** out) {
    clear_error();
    PS_ARG(out != nullptr, "psdiff_create: out is NULL");
    *out = nullptr;
    PS_ARG(d != nullptr && d->cams != nullptr, "psdiff_create: desc or cams is NULL");
    PS_ARG(d->n_cams >= 1 && d->n_cams <= PS_MAX_CAMS, "psdiff_create: n_cams must be in 1..%d", PS_MAX_CAMS);
    PS_ARG(d->ref.width > 0 && d->ref.height > 0 && d->ref.width <= 16384 && d->ref.height <= 16384 &&
               d->ref.fx > 0 && d->ref.fy > 0 && d->ref.xi >= 0,
           "psdiff_create: bad reference camera");
    for (int j = 0; j < d->n_cams; ++j)
        PS_ARG(d->cams[j].width > 1 && d->cams[j].height > 1 && d->cams[j].fx > 0 && d->cams[j].fy > 0 &&
                   d->cams[j].xi >= 0,
               "psdiff_create: bad matching camera %d", j);
    const ps_level& L = d->level;
    PS_ARG(L.kind == PS_LEVEL_DOWNSAMPLE && L.factor == 1, "psdiff_create: one full-resolution level (factor 1)");
    PS_ARG(L.window == 5 || L.window == 7 || L.window == 9, "psdiff_create: window must be 5, 7 or 9");
    PS_ARG(L.n_sets >= 1 && L.n_sets <= PS_MAX_SETS, "psdiff_create: n_sets must be in 1..%d", PS_MAX_SETS);
    PS_ARG(d->temperature > 0 && std::isfinite(d->temperature), "psdiff_create: temperature must be > 0");
    std::vector<PlaneD> planes;
    for (int s = 0; s < L.n_sets; ++s) {
        const ps_plane_set& S = L.sets[s];
        PS_ARG(S.count >= 1 && S.count <= 4096 && S.a > 0 && S.b >= S.a, "psdiff_create: bad plane set %d", s);
        PS_ARG(S.family == PS_PLANES_FRONTO || S.family == PS_PLANES_GROUND, "psdiff_create: bad family");
        double n[3] = {0, 0, 1};
        if (S.family == PS_PLANES_GROUND) {
            double nn = std::sqrt(S.n[0] * S.n[0] + S.n[1] * S.n[1] + S.n[2] * S.n[2]);
            PS_ARG(nn > 0, "psdiff_create: ground normal is zero");
            for (int i = 0; i < 3; ++i) n[i] = S.n[i] / nn;
        }
        for (int i = 0; i < S.count; ++i) {
            double t = S.count > 1 ? (double)i / (S.count - 1) : 0.0;
            double dd = S.family == PS_PLANES_FRONTO ? 1.0 / (1.0 / S.b + t * (1.0 / S.a - 1.0 / S.b))
                                                     : S.a + t * (S.b - S.a);
            planes.push_back({(float)n[0], (float)n[1], (float)n[2], (float)dd});
        }
    }
    psdiff_t* h = new psdiff_t();
    h->ref = d->ref;
    h->n_cams = d->n_cams;
    for (int j = 0; j < d->n_cams; ++j) h->cams[j] = d->cams[j];
    h->rho = L.window / 2;
    h->K = (int)planes.size();
    h->T = d->temperature;
    const size_t npx = (size_t)d->ref.width * d->ref.height;
    cudaError_t e = cudaMalloc(&h->rays, sizeof(float4) * npx);
    if (e == cudaSuccess) e = cudaMalloc(&h->planes, sizeof(PlaneD) * planes.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(h->planes, planes.data(), sizeof(PlaneD) * planes.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_diff(h);
        set_error("psdiff_create: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA;
    }
    if (build_rays(d->ref, h->rays, nullptr) != PS_OK || cudaDeviceSynchronize() != cudaSuccess) {
        free_diff(h);
        return PS_ERR_CUDA;
    }
    *out = h;
    return PS_OK;
}

extern "C" void psdiff_destroy(psdiff_t* h) { free_diff(h); }

extern "C" int psdiff_forward(psdiff_t* h, const float* const* images, const ps_pose* ref_to_cam, float* range,
                              float* cost, float* aux, void* stream) {
    clear_error();
    PS_ARG(h != nullptr && range != nullptr, "psdiff_forward: handle or range is NULL");
    DiffP P;
    int st = fill_params(h, images, ref_to_cam, P);
    if (st) return st;
    dim3 grid((P.W + DT - 1) / DT, (P.H + DT - 1) / DT);
    cudaStream_t s = (cudaStream_t)stream;
    if (P.rho == 2)
        soft_fwd_kernel<2><<<grid, DNT, 0, s>>>(P, range, cost, aux);
    else if (P.rho == 3)
        soft_fwd_kernel<3><<<grid, DNT, 0, s>>>(P, range, cost, aux);
    else
        soft_fwd_kernel<4><<<grid, DNT, 0, s>>>(P, range, cost, aux);
    PS_CUDA(cudaGetLastError());
    return PS_OK;
}

extern "C" int psdiff_backward(psdiff_t* h, const float* const* images, const ps_pose* ref_to_cam, const float* aux,
                               const float* g_range, const float* g_cost, float* const* g_images, double* g_pose,
                               void* stream) {
    clear_error();
    PS_ARG(h != nullptr && aux != nullptr, "psdiff_backward: handle or aux is NULL");
    DiffP P;
    int st = fill_params(h, images, ref_to_cam, P);
    if (st) return st;
    float* g_ref = g_images ? g_images[0] : nullptr;
    GradOut G;
    for (int j = 0; j < PS_MAX_CAMS; ++j) G.cam[j] = (g_images && j < h->n_cams) ? g_images[1 + j] : nullptr;
    // at most 202 KB (window 9, 4 cameras)
    const size_t smem = sizeof(float) * (P.rho == 2   ? BwdLayout<2>::floats(P.n_cams)
                                         : P.rho == 3 ? BwdLayout<3>::floats(P.n_cams)
                                                      : BwdLayout<4>::floats(P.n_cams));
    dim3 grid((P.W + 15) / 16, (P.H + 15) / 16);
    cudaStream_t s = (cudaStream_t)stream;
    if (P.rho == 2) {
        PS_CUDA(cudaFuncSetAttribute(soft_bwd_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        soft_bwd_kernel<2><<<grid, DNT, smem, s>>>(P, aux, g_range, g_cost, g_ref, G, g_pose);
    } else if (P.rho == 3) {
        PS_CUDA(cudaFuncSetAttribute(soft_bwd_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        soft_bwd_kernel<3><<<grid, DNT, smem, s>>>(P, aux, g_range, g_cost, g_ref, G, g_pose);
    } else {
        PS_CUDA(cudaFuncSetAttribute(soft_bwd_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        soft_bwd_kernel<4><<<grid, DNT, smem, s>>>(P, aux, g_range, g_cost, g_ref, G, g_pose);
    }
    PS_CUDA(cudaGetLastError());
    return PS_OK;
}

namespace ps {
PS_DEFINE_CHECK_READER(check_bits_diff)
}  // namespace ps

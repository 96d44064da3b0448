// Oracle: a plain, slow FP64 CPU restatement of the fisheye plane-sweep +
// TSDF fusion path of "Real-Time Dense Mapping for Self-Driving Vehicles
// using Fisheye Cameras" (Cui et al.), written to check the CUDA library.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
// benchmark's CPU-baseline leg may load this code.  It shares no code, header,
// table or helper with the CUDA library; the two meet only in the seeded
// inputs produced by the scene generator.
//
// Every function follows one step of the method in the paper's order, in
// double precision, with direct loops (no running sums, no tiling, no fusion):
//   unified camera model ............ Sec. III-C, Eq. (1) and its forward map
//   plane families .................. Sec. III-A (fronto-parallel + ground-parallel)
//   per-plane warp + bilinear sample  Sec. III-A (plane-sweeping stereo)
//   ZNCC matching cost .............. Sec. III-A (cost 0 <-> ZNCC 1, cost 1 <-> ZNCC -1)
//   min over matching cameras, winner-take-all, parabola sub-plane fit
//   multi-scale: downsample / crop / merge ... Sec. III-A "Multi-scale strategy"
//   dynamic-object boxes as masks ... Sec. III (overview) and III-B
//   voxel-block allocation along [d - mu, d + mu] ... Sec. III-C
//   TSDF running average ............ Sec. III-C, Eq. (2), weight cap
//   local-map allocation gate ....... Sec. III-C (60 m x 60 m x 3 m)
//   depth filters ................... Sec. III-A "Depth map filtering"
//   block swap-out / load ........... Sec. III-C (blocks leaving the local map)
//   surface points of the map ....... the map as a point set (Sec. IV-C)
//   differentiable forms (not in the paper): soft-argmin depth over the
//   plane hypotheses and dense fusion, each with its gradient
//
// Readings where the paper is silent are stated beside the code that takes
// them.  Built with OpenMP, the independent loops (pixels of a sweep, rows of
// a ray table, blocks of an integration) are shared among threads; each
// pixel, ray and voxel is still computed by the same sequential code, so the
// results do not depend on the thread count.  Parity pins: see tests/test_oracle_*.py.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <set>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double INF = std::numeric_limits<double>::infinity();
const int MAX_WINDOW = 15;  // largest matching window side the oracle accepts

struct OrCamera {
    double xi, fx, fy, cx, cy, k1, k2, p1, p2, r2_max;
    int32_t width, height;
};

struct OrPose {      // X_dst = R X_src + t, R row-major
    double R[9];
    double t[3];
};

struct OrPlaneSet {  // family 0: fronto, inverse depth uniform on [1/b, 1/a], index 0 farthest
    int32_t family;  // family 1: ground-parallel, offset uniform on [a, b], normal n
    int32_t count;
    double a, b;
    double n[3];
};

struct OrLevel {     // kind 0: downsample by factor; kind 1: centred crop at full resolution
    int32_t kind, factor, crop_w, crop_h, window, n_sets;
    OrPlaneSet sets[4];
};

// ---------------------------------------------------------------- camera

// Radial-tangential distortion of undistorted normalised coordinates.
// (Distortion is not part of Eq. (1); the unified model it extends is Mei's.)
void distort(const OrCamera& c, double x, double y, double* xd, double* yd) {
    double r2 = x * x + y * y;
    double radial = 1.0 + c.k1 * r2 + c.k2 * r2 * r2;
    *xd = x * radial + 2.0 * c.p1 * x * y + c.p2 * (r2 + 2.0 * x * x);
    *yd = y * radial + c.p1 * (r2 + 2.0 * y * y) + 2.0 * c.p2 * x * y;
}

// Invert the distortion by Newton's method on the 2x2 system.  Converged when
// the residual is below 1e-13; not converged after 100 iterations = invalid.
bool undistort(const OrCamera& c, double xd, double yd, double* x, double* y) {
    double X = xd, Y = yd;
    for (int it = 0; it < 100; ++it) {
        double fx, fy;
        distort(c, X, Y, &fx, &fy);
        double ex = fx - xd, ey = fy - yd;
        if (std::fabs(ex) < 1e-13 && std::fabs(ey) < 1e-13) {
            *x = X;
            *y = Y;
            return true;
        }
        double r2 = X * X + Y * Y;
        double radial = 1.0 + c.k1 * r2 + c.k2 * r2 * r2;
        double dr = c.k1 + 2.0 * c.k2 * r2;  // d radial / d r2
        double j11 = radial + 2.0 * X * X * dr + 2.0 * c.p1 * Y + 6.0 * c.p2 * X;
        double j12 = 2.0 * X * Y * dr + 2.0 * c.p1 * X + 2.0 * c.p2 * Y;
        double j21 = 2.0 * X * Y * dr + 2.0 * c.p1 * X + 2.0 * c.p2 * Y;
        double j22 = radial + 2.0 * Y * Y * dr + 6.0 * c.p1 * Y + 2.0 * c.p2 * X;
        double det = j11 * j22 - j12 * j21;
        if (det == 0.0) return false;
        X -= (j22 * ex - j12 * ey) / det;
        Y -= (-j21 * ex + j11 * ey) / det;
    }
    return false;
}

// Back-projection, Eq. (1): unit ray of pixel (u, v).
// Invalid when undistortion fails, when the undistorted radius exceeds the
// camera's r2_max, or when 1 + (1 - xi^2)(x^2 + y^2) < 0.
bool unproject(const OrCamera& c, double u, double v, double r[3]) {
    double x, y;
    if (!undistort(c, (u - c.cx) / c.fx, (v - c.cy) / c.fy, &x, &y)) return false;
    double s = x * x + y * y;
    if (s > c.r2_max) return false;
    double disc = 1.0 + (1.0 - c.xi * c.xi) * s;
    if (disc < 0.0) return false;
    double f = (c.xi + std::sqrt(disc)) / (s + 1.0);
    r[0] = f * x;
    r[1] = f * y;
    r[2] = f - c.xi;
    return true;
}

// Forward unified projection: point -> unit sphere -> shift by xi along z ->
// perspective division -> distortion -> pixel.  Valid where the sphere point
// satisfies z_s > -min(xi, 1/xi) (the side of the sphere on which the map
// is one-to-one and inverted by Eq. (1)) and the undistorted radius is within
// r2_max.
bool project(const OrCamera& c, const double X[3], double* u, double* v) {
    double n = std::sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    if (!(n > 0.0)) return false;
    double xs = X[0] / n, ys = X[1] / n, zs = X[2] / n;
    double lim = c.xi > 0.0 ? std::min(c.xi, 1.0 / c.xi) : 0.0;
    if (!(zs > -lim)) return false;
    double mx = xs / (zs + c.xi), my = ys / (zs + c.xi);
    if (mx * mx + my * my > c.r2_max) return false;
    double xd, yd;
    distort(c, mx, my, &xd, &yd);
    *u = c.fx * xd + c.cx;
    *v = c.fy * yd + c.cy;
    return true;
}

void apply(const OrPose& P, const double X[3], double Y[3]) {
    for (int i = 0; i < 3; ++i)
        Y[i] = P.R[3 * i] * X[0] + P.R[3 * i + 1] * X[1] + P.R[3 * i + 2] * X[2] + P.t[i];
}

// ---------------------------------------------------------------- levels

struct Image {
    int W = 0, H = 0;
    std::vector<double> px;  // intensities in [0, 1]
    double at(int x, int y) const { return px[(size_t)y * W + x]; }
};

// Downsampled level intrinsics: pixel centres of an s x s block average sit at
// full-resolution coordinate s*u' + (s-1)/2.
OrCamera scaled(const OrCamera& c, int s) {
    OrCamera o = c;
    o.fx = c.fx / s;
    o.fy = c.fy / s;
    o.cx = (c.cx - (s - 1) / 2.0) / s;
    o.cy = (c.cy - (s - 1) / 2.0) / s;
    o.width = c.width / s;
    o.height = c.height / s;
    return o;
}

// s x s box mean of a uint8 image, intensities scaled to [0, 1].
Image downsample(const uint8_t* img, int W, int H, int s) {
    Image o;
    o.W = W / s;
    o.H = H / s;
    o.px.assign((size_t)o.W * o.H, 0.0);
    for (int y = 0; y < o.H; ++y)
        for (int x = 0; x < o.W; ++x) {
            double acc = 0.0;
            for (int dy = 0; dy < s; ++dy)
                for (int dx = 0; dx < s; ++dx) acc += img[(size_t)(s * y + dy) * W + (s * x + dx)];
            o.px[(size_t)y * o.W + x] = acc / (s * s) / 255.0;
        }
    return o;
}

Image crop(const uint8_t* img, int W, int x0, int y0, int w, int h) {
    Image o;
    o.W = w;
    o.H = h;
    o.px.resize((size_t)w * h);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) o.px[(size_t)y * w + x] = img[(size_t)(y0 + y) * W + (x0 + x)] / 255.0;
    return o;
}

struct PlaneH {          // plane n . X = d in the reference frame
    double n[3];
    double d;
    int family_set;      // index of the plane set it belongs to
    int local;           // index within that set
};

struct LevelCtx {
    OrCamera ref;
    std::vector<OrCamera> cams;
    Image ref_img;
    std::vector<Image> cam_img;
    std::vector<PlaneH> planes;
    std::vector<int> set_start, set_count;
    int rho = 0;
    // reference-level ray table (Eq. 1 per pixel)
    std::vector<std::array<double, 3>> ray;
    std::vector<uint8_t> ray_ok;
};

// Plane hypotheses of a level (Sec. III-A): the sets in order, planes of a set in index order.
void make_planes(const OrLevel& L, LevelCtx& ctx) {
    for (int s = 0; s < L.n_sets; ++s) {
        const OrPlaneSet& P = L.sets[s];
        ctx.set_start.push_back((int)ctx.planes.size());
        ctx.set_count.push_back(P.count);
        for (int i = 0; i < P.count; ++i) {
            PlaneH h;
            h.family_set = s;
            h.local = i;
            double t = P.count > 1 ? (double)i / (P.count - 1) : 0.0;
            if (P.family == 0) {
                h.n[0] = 0.0;
                h.n[1] = 0.0;
                h.n[2] = 1.0;
                double inv = 1.0 / P.b + t * (1.0 / P.a - 1.0 / P.b);
                h.d = 1.0 / inv;
            } else {
                double nn = std::sqrt(P.n[0] * P.n[0] + P.n[1] * P.n[1] + P.n[2] * P.n[2]);
                for (int k = 0; k < 3; ++k) h.n[k] = P.n[k] / nn;
                h.d = P.a + t * (P.b - P.a);
            }
            ctx.planes.push_back(h);
        }
    }
}

// Plane parameter of a set at fractional index i (fronto: inverse depth is
// the uniformly spaced quantity; ground: the offset is).
double plane_param(const OrPlaneSet& P, double i) {
    double t = P.count > 1 ? i / (P.count - 1) : 0.0;
    if (P.family == 0) return 1.0 / (1.0 / P.b + t * (1.0 / P.a - 1.0 / P.b));
    return P.a + t * (P.b - P.a);
}

void build_level(const OrCamera& ref_full, int n_cams, const OrCamera* cams_full, const OrLevel& L,
                 const uint8_t* const* images, LevelCtx& ctx) {
    const int W = ref_full.width, H = ref_full.height;
    if (L.kind == 0) {
        int s = L.factor;
        ctx.ref = scaled(ref_full, s);
        ctx.ref_img = downsample(images[0], W, H, s);
        for (int j = 0; j < n_cams; ++j) {
            ctx.cams.push_back(scaled(cams_full[j], s));
            ctx.cam_img.push_back(downsample(images[1 + j], cams_full[j].width, cams_full[j].height, s));
        }
    } else {
        // Centred crop of the reference image at full resolution; the matching
        // cameras keep their full images (a warped ray may land anywhere in them).
        int x0 = (W - L.crop_w) / 2, y0 = (H - L.crop_h) / 2;
        ctx.ref = ref_full;
        ctx.ref.cx -= x0;
        ctx.ref.cy -= y0;
        ctx.ref.width = L.crop_w;
        ctx.ref.height = L.crop_h;
        ctx.ref_img = crop(images[0], W, x0, y0, L.crop_w, L.crop_h);
        for (int j = 0; j < n_cams; ++j) {
            ctx.cams.push_back(cams_full[j]);
            ctx.cam_img.push_back(downsample(images[1 + j], cams_full[j].width, cams_full[j].height, 1));
        }
    }
    ctx.rho = std::min(L.window, MAX_WINDOW) / 2;
    make_planes(L, ctx);
    size_t N = (size_t)ctx.ref.width * ctx.ref.height;
    ctx.ray.resize(N);
    ctx.ray_ok.resize(N);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ctx.ref.height; ++y)
        for (int x = 0; x < ctx.ref.width; ++x) {
            double r[3];
            bool ok = unproject(ctx.ref, x, y, r);
            size_t i = (size_t)y * ctx.ref.width + x;
            ctx.ray_ok[i] = ok;
            ctx.ray[i] = {r[0], r[1], r[2]};
        }
}

// Bilinear sample at (u, v); valid only inside [0, W-1] x [0, H-1].
bool bilinear(const Image& I, double u, double v, double* out) {
    if (!(u >= 0.0 && u <= I.W - 1 && v >= 0.0 && v <= I.H - 1)) return false;
    int x0 = (int)std::floor(u), y0 = (int)std::floor(v);
    double ax = u - x0, ay = v - y0;
    int x1 = std::min(x0 + 1, I.W - 1), y1 = std::min(y0 + 1, I.H - 1);
    *out = (1 - ay) * ((1 - ax) * I.at(x0, y0) + ax * I.at(x1, y0)) +
           ay * ((1 - ax) * I.at(x0, y1) + ax * I.at(x1, y1));
    return true;
}

// Plane-induced warp of reference pixel q into matching camera j, then sample.
bool warped_sample(const LevelCtx& ctx, const OrPose& ref_to_cam, int j, const PlaneH& P, int qx, int qy,
                   double* w) {
    size_t i = (size_t)qy * ctx.ref.width + qx;
    if (!ctx.ray_ok[i]) return false;
    const double* r = ctx.ray[i].data();
    double nr = P.n[0] * r[0] + P.n[1] * r[1] + P.n[2] * r[2];
    if (!(nr > 0.0)) return false;
    double lam = P.d / nr;
    double X[3] = {lam * r[0], lam * r[1], lam * r[2]};
    double Xj[3];
    apply(ref_to_cam, X, Xj);
    double u, v;
    if (!project(ctx.cams[j], Xj, &u, &v)) return false;
    return bilinear(ctx.cam_img[j], u, v, w);
}

// Zero-normalised cross-correlation of two N-sample windows by its two-pass
// definition.  Returns false when either window's per-sample variance is below
// 1e-8 (a flat window has no defined correlation).
bool zncc(const double* a, const double* b, int N, double* out) {
    double ma = 0, mb = 0;
    for (int i = 0; i < N; ++i) {
        ma += a[i];
        mb += b[i];
    }
    ma /= N;
    mb /= N;
    double cov = 0, va = 0, vb = 0;
    for (int i = 0; i < N; ++i) {
        cov += (a[i] - ma) * (b[i] - mb);
        va += (a[i] - ma) * (a[i] - ma);
        vb += (b[i] - mb) * (b[i] - mb);
    }
    if (va / N < 1e-8 || vb / N < 1e-8) return false;
    *out = cov / std::sqrt(va * vb);
    return true;
}

// Matching cost of reference pixel p, plane P, camera j over the
// (2 rho + 1)^2 window around p in reference-image space: (1 - ZNCC) / 2,
// so that ZNCC 1 -> 0 and ZNCC -1 -> 1.  +inf when any window sample is
// invalid or the window is flat.
double window_cost(const LevelCtx& ctx, const OrPose& pose, int j, const PlaneH& P, int px, int py) {
    int rho = ctx.rho;
    double a[MAX_WINDOW * MAX_WINDOW], b[MAX_WINDOW * MAX_WINDOW];
    int N = 0;
    for (int dy = -rho; dy <= rho; ++dy)
        for (int dx = -rho; dx <= rho; ++dx) {
            double w;
            if (!warped_sample(ctx, pose, j, P, px + dx, py + dy, &w)) return INF;
            a[N] = ctx.ref_img.at(px + dx, py + dy);
            b[N] = w;
            ++N;
        }
    double z;
    if (!zncc(a, b, N, &z)) return INF;
    return (1.0 - z) / 2.0;
}

// Winner-take-all over the aggregated costs C[0..K) (+inf = invalid):
// the lowest index among the minima wins, the second best is the minimum over
// every other plane, and a parabola through the winner and its two neighbours
// in the same plane set gives the sub-plane offset delta in [-1/2, 1/2]
// (0 at a set's ends, next to an invalid neighbour, or on a flat triple).
void wta(const double* C, int K, const std::vector<int>& set_start, const std::vector<int>& set_count, int* kstar,
         double* c1, double* c2, double* delta) {
    int ks = -1;
    for (int k = 0; k < K; ++k)
        if (C[k] < INF && (ks < 0 || C[k] < C[ks])) ks = k;
    *kstar = ks;
    *c1 = INF;
    *c2 = INF;
    *delta = 0.0;
    if (ks < 0) return;
    *c1 = C[ks];
    for (int k = 0; k < K; ++k)
        if (k != ks && C[k] < *c2) *c2 = C[k];
    int s = 0;
    while (s + 1 < (int)set_start.size() && set_start[s + 1] <= ks) ++s;
    int i = ks - set_start[s], cnt = set_count[s];
    if (i > 0 && i < cnt - 1 && C[ks - 1] < INF && C[ks + 1] < INF) {
        double cm = C[ks - 1], c0 = C[ks], cp = C[ks + 1];
        double den = cm - 2.0 * c0 + cp;
        if (den > 0.0) {
            double dl = (cm - cp) / (2.0 * den);
            *delta = std::max(-0.5, std::min(0.5, dl));
        }
    }
}

struct PixelResult {
    double depth, c1, c2;
    int32_t kstar;
};

// One reference pixel of one level: costs over all planes (min over
// cameras), winner-take-all with ties to the lowest index, second best over
// all other planes, parabola through the winner and its two neighbours in the
// same plane set, and the range along the pixel's ray.
PixelResult sweep_pixel(const LevelCtx& ctx, const OrLevel& L, const OrPose* poses, int px, int py,
                        double* cost_row) {
    PixelResult R{0.0, INF, INF, -1};
    int rho = ctx.rho;
    int K = (int)ctx.planes.size();
    bool inside = px >= rho && py >= rho && px < ctx.ref.width - rho && py < ctx.ref.height - rho;
    std::vector<double> C(K, INF);
    if (inside) {
        for (int k = 0; k < K; ++k) {
            double best = INF;
            for (int j = 0; j < (int)ctx.cams.size(); ++j) {
                double c = window_cost(ctx, poses[j], j, ctx.planes[k], px, py);
                if (c < best) best = c;
            }
            C[k] = best;
        }
    }
    if (cost_row)
        for (int k = 0; k < K; ++k) cost_row[k] = C[k];
    int ks;
    double delta;
    wta(C.data(), K, ctx.set_start, ctx.set_count, &ks, &R.c1, &R.c2, &delta);
    if (ks < 0) return R;
    R.kstar = ks;
    const PlaneH& P = ctx.planes[ks];
    int s = P.family_set, i = P.local;
    double d = plane_param(L.sets[s], i + delta);
    const double* r = ctx.ray[(size_t)py * ctx.ref.width + px].data();
    double nr = P.n[0] * r[0] + P.n[1] * r[1] + P.n[2] * r[2];
    R.depth = d / nr;
    return R;
}

// ---------------------------------------------------------------- TSDF

using Key = std::array<int64_t, 3>;

struct TsdfDesc {
    double voxel_size, mu, w_max;
    int32_t block_dim;
    int32_t dense_dim[3];     // voxels per axis; all zero = hashed blocks
    double origin[3];
    double local_half[3];     // all zero = no local-map gate
};

struct Block {
    std::vector<double> D, W;
    std::vector<uint8_t> amb;  // voxel's history may differ under float rounding
    uint8_t block_amb = 0;     // block's first allocation frame may differ
};

struct Tsdf {
    TsdfDesc d;
    std::map<Key, Block> blocks;
    std::set<Key> ever_maybe;  // blocks ever in a frame's ambiguous allocation band
    std::set<Key> last_strict, last_maybe;
    // ambiguity bands used to mark rounding-sensitive decisions
    double tau_len = 1e-4;     // m, segment / block intersection length
    double tau_px = 2e-3;      // px, nearest-pixel rounding
    double tau_m = 1e-4;       // m, eta >= -mu threshold
    double tau_rel = 1e-6;     // projection validity margins
};

Block new_block(int B3) {
    Block b;
    b.D.assign(B3, 0.0);
    b.W.assign(B3, 0.0);
    b.amb.assign(B3, 0);
    return b;
}

// Length of segment [A, B] inside the box [lo, hi] (slab method); 0 if disjoint.
double segment_box_length(const double A[3], const double B[3], const double lo[3], const double hi[3]) {
    double t0 = 0.0, t1 = 1.0;
    for (int k = 0; k < 3; ++k) {
        double d = B[k] - A[k];
        if (d == 0.0) {
            if (A[k] < lo[k] || A[k] > hi[k]) return 0.0;
            continue;
        }
        double ta = (lo[k] - A[k]) / d, tb = (hi[k] - A[k]) / d;
        if (ta > tb) std::swap(ta, tb);
        t0 = std::max(t0, ta);
        t1 = std::min(t1, tb);
        if (t0 > t1) return 0.0;
    }
    double len = std::sqrt((B[0] - A[0]) * (B[0] - A[0]) + (B[1] - A[1]) * (B[1] - A[1]) +
                           (B[2] - A[2]) * (B[2] - A[2]));
    return (t1 - t0) * len;
}

bool gate_on(const TsdfDesc& d) { return d.local_half[0] > 0 || d.local_half[1] > 0 || d.local_half[2] > 0; }

// Voxel-block allocation (Sec. III-C): every block that the segment from
// d - mu to d + mu along each valid pixel's ray crosses, restricted to the
// local map around the vehicle.  The segment starts no closer than the
// camera centre.
void allocate(Tsdf& T, const float* depth, const OrCamera& cam, const OrPose& w2c, const double* lc) {
    const TsdfDesc& d = T.d;
    const int B = d.block_dim;
    const double L = B * d.voxel_size;
    const double tau = T.tau_len;
    T.last_strict.clear();
    T.last_maybe.clear();
    std::set<Key> alloc_now;
    double C[3], Rt[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) Rt[3 * i + k] = w2c.R[3 * k + i];
    for (int i = 0; i < 3; ++i) C[i] = -(Rt[3 * i] * w2c.t[0] + Rt[3 * i + 1] * w2c.t[1] + Rt[3 * i + 2] * w2c.t[2]);
    for (int v = 0; v < cam.height; ++v)
        for (int u = 0; u < cam.width; ++u) {
            double dep = depth[(size_t)v * cam.width + u];
            if (!(dep > 0.0) || !std::isfinite(dep)) continue;
            double r[3];
            if (!unproject(cam, u, v, r)) continue;
            double dw[3];
            for (int i = 0; i < 3; ++i) dw[i] = Rt[3 * i] * r[0] + Rt[3 * i + 1] * r[1] + Rt[3 * i + 2] * r[2];
            double s0 = std::max(0.0, dep - d.mu), s1 = dep + d.mu;
            double A[3], Bp[3], Ae[3], Be[3];
            for (int i = 0; i < 3; ++i) {
                A[i] = C[i] + s0 * dw[i] - d.origin[i];
                Bp[i] = C[i] + s1 * dw[i] - d.origin[i];
                Ae[i] = A[i] - tau * dw[i];
                Be[i] = Bp[i] + tau * dw[i];
            }
            int64_t lo[3], hi[3];
            for (int i = 0; i < 3; ++i) {
                lo[i] = (int64_t)std::floor((std::min(A[i], Bp[i]) - tau) / L);
                hi[i] = (int64_t)std::floor((std::max(A[i], Bp[i]) + tau) / L);
            }
            for (int64_t bz = lo[2]; bz <= hi[2]; ++bz)
                for (int64_t by = lo[1]; by <= hi[1]; ++by)
                    for (int64_t bx = lo[0]; bx <= hi[0]; ++bx) {
                        Key key = {bx, by, bz};
                        double blo[3] = {bx * L, by * L, bz * L};
                        double bhi[3] = {(bx + 1) * L, (by + 1) * L, (bz + 1) * L};
                        double bloe[3], bhie[3];
                        for (int i = 0; i < 3; ++i) {
                            bloe[i] = blo[i] - tau;
                            bhie[i] = bhi[i] + tau;
                        }
                        double len = segment_box_length(A, Bp, blo, bhi);
                        double len_loose = segment_box_length(Ae, Be, bloe, bhie);
                        if (len_loose <= 0.0) continue;
                        bool inside = true;
                        double margin = INF;
                        if (gate_on(d) && lc) {
                            for (int i = 0; i < 3; ++i) {
                                double c = d.origin[i] + (key[i] + 0.5) * L;
                                double m = d.local_half[i] - std::fabs(c - lc[i]);
                                margin = std::min(margin, m);
                            }
                            inside = margin >= 0.0;
                        }
                        bool strict = len >= tau && (margin >= tau);
                        bool maybe = !strict && (std::fabs(margin) < tau || inside);
                        if (len > 0.0 && inside) alloc_now.insert(key);
                        if (strict)
                            T.last_strict.insert(key);
                        else if (maybe)
                            T.last_maybe.insert(key);
                    }
        }
    for (const Key& k : T.last_strict) T.last_maybe.erase(k);
    const int B3 = B * B * B;
    for (const Key& k : alloc_now) {
        if (T.blocks.count(k)) continue;
        Block b = new_block(B3);
        b.block_amb = (!T.last_strict.count(k)) || T.ever_maybe.count(k);
        T.blocks.emplace(k, std::move(b));
    }
    for (const Key& k : T.last_maybe)
        if (!T.blocks.count(k)) T.ever_maybe.insert(k);
}

double frac_dist(double x) {  // distance of x to the nearest integer
    return std::fabs(x - std::floor(x + 0.5));
}

// Integration, Eq. (2), over every voxel of every allocated block (the brute
// force definition; no visible-block list).  eta = d(pi(X_d)) - |X_d| with the
// depth taken at the nearest pixel; voxels with eta < -mu are left alone.
void integrate(Tsdf& T, const float* depth, const OrCamera& cam, const OrPose& w2c) {
    const TsdfDesc& d = T.d;
    const int B = d.block_dim;
    const double lim = cam.xi > 0.0 ? std::min(cam.xi, 1.0 / cam.xi) : 0.0;
    // Blocks are independent: with OpenMP they are shared among threads.
    std::vector<std::pair<const Key*, Block*>> list;
    list.reserve(T.blocks.size());
    for (auto& kv : T.blocks) list.emplace_back(&kv.first, &kv.second);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t bi = 0; bi < (int64_t)list.size(); ++bi) {
        const Key& key = *list[bi].first;
        Block& blk = *list[bi].second;
        for (int z = 0; z < B; ++z)
            for (int y = 0; y < B; ++y)
                for (int x = 0; x < B; ++x) {
                    int vi = (z * B + y) * B + x;
                    double X[3] = {d.origin[0] + (key[0] * B + x + 0.5) * d.voxel_size,
                                   d.origin[1] + (key[1] * B + y + 0.5) * d.voxel_size,
                                   d.origin[2] + (key[2] * B + z + 0.5) * d.voxel_size};
                    double Xd[3];
                    apply(w2c, X, Xd);
                    double nrm = std::sqrt(Xd[0] * Xd[0] + Xd[1] * Xd[1] + Xd[2] * Xd[2]);
                    // rounding-sensitive validity of the projection
                    if (nrm > 0) {
                        double zs = Xd[2] / nrm;
                        if (std::fabs(zs + lim) < T.tau_rel) blk.amb[vi] = 1;
                        double den = zs + cam.xi;
                        if (den != 0.0) {
                            double mx = Xd[0] / nrm / den, my = Xd[1] / nrm / den;
                            if (std::fabs(mx * mx + my * my - cam.r2_max) < T.tau_rel * (1 + cam.r2_max))
                                blk.amb[vi] = 1;
                        }
                    }
                    double u, v;
                    if (!project(cam, Xd, &u, &v)) continue;
                    if (frac_dist(u + 0.5) < T.tau_px || frac_dist(v + 0.5) < T.tau_px) blk.amb[vi] = 1;
                    double pu = std::floor(u + 0.5), pv = std::floor(v + 0.5);
                    if (pu < 0 || pv < 0 || pu >= cam.width || pv >= cam.height) continue;
                    double dm = depth[(size_t)pv * cam.width + (size_t)pu];
                    if (!(dm > 0.0) || !std::isfinite(dm)) continue;
                    double eta = dm - nrm;
                    if (std::fabs(eta + d.mu) < T.tau_m) blk.amb[vi] = 1;
                    if (eta < -d.mu) continue;
                    double sdf = std::min(1.0, eta / d.mu);
                    double w = blk.W[vi];
                    blk.D[vi] = (w * blk.D[vi] + sdf) / (w + 1.0);
                    blk.W[vi] = std::min(w + 1.0, d.w_max);
                }
    }
}

// ---------------------------------------------------------------- differentiable forms
//
// Not in the paper: the winner-take-all depth is piecewise constant in the
// images and the poses, so for gradients the plane hypotheses are averaged
// with softmax weights of their aggregated costs (soft-argmin):
//   s_k   = exp(-C_k / T) / sum over valid k' of exp(-C_k' / T)
//   E     = sum_k s_k rho_k,   rho_k = (n_k . r) / d_k   (inverse range of plane k along the ray)
//   range = 1 / E
// C_k is the minimum over the matching cameras, as in the sweep; its
// gradient goes to the camera that attains it (the lowest index on a tie).
// Beside the range, the soft minimum of the costs
//   S = -T log sum over valid k of exp(-C_k / T),   dS/dC_k = s_k,
// is a photometric loss that needs no ground truth.
// Images are real-valued here (intensities as given, no quantisation).

double norm3(const double X[3]) { return std::sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]); }

// d(u, v)/dX of project() at X (row-major 2 x 3), by the chain rule through
// the sphere shift, the perspective division and the distortion polynomial.
void project_jacobian(const OrCamera& c, const double X[3], double J[6]) {
    double n = norm3(X);
    double den = X[2] + c.xi * n;  // mx = X / den, my = Y / den
    double dden[3] = {c.xi * X[0] / n, c.xi * X[1] / n, 1.0 + c.xi * X[2] / n};
    double mx = X[0] / den, my = X[1] / den;
    double dmx[3], dmy[3];
    for (int i = 0; i < 3; ++i) {
        dmx[i] = (i == 0 ? 1.0 / den : 0.0) - X[0] * dden[i] / (den * den);
        dmy[i] = (i == 1 ? 1.0 / den : 0.0) - X[1] * dden[i] / (den * den);
    }
    double r2 = mx * mx + my * my;
    double rad = 1.0 + c.k1 * r2 + c.k2 * r2 * r2, drad = c.k1 + 2.0 * c.k2 * r2;
    double a = rad + 2.0 * mx * mx * drad + 2.0 * c.p1 * my + 6.0 * c.p2 * mx;  // dxd/dmx
    double b = 2.0 * mx * my * drad + 2.0 * c.p1 * mx + 2.0 * c.p2 * my;        // dxd/dmy = dyd/dmx
    double d = rad + 2.0 * my * my * drad + 6.0 * c.p1 * my + 2.0 * c.p2 * mx;  // dyd/dmy
    for (int i = 0; i < 3; ++i) {
        J[i] = c.fx * (a * dmx[i] + b * dmy[i]);
        J[3 + i] = c.fy * (b * dmx[i] + d * dmy[i]);
    }
}

// Level of real-valued images at full resolution (the differentiable forms
// use one full-resolution level).
void build_level_real(const OrCamera& ref, int n_cams, const OrCamera* cams, const OrLevel& L,
                      const double* const* images, LevelCtx& ctx) {
    ctx.ref = ref;
    ctx.ref_img.W = ref.width;
    ctx.ref_img.H = ref.height;
    ctx.ref_img.px.assign(images[0], images[0] + (size_t)ref.width * ref.height);
    for (int j = 0; j < n_cams; ++j) {
        ctx.cams.push_back(cams[j]);
        Image I;
        I.W = cams[j].width;
        I.H = cams[j].height;
        I.px.assign(images[1 + j], images[1 + j] + (size_t)I.W * I.H);
        ctx.cam_img.push_back(I);
    }
    ctx.rho = std::min(L.window, MAX_WINDOW) / 2;
    make_planes(L, ctx);
    size_t N = (size_t)ref.width * ref.height;
    ctx.ray.resize(N);
    ctx.ray_ok.resize(N);
    for (int y = 0; y < ref.height; ++y)
        for (int x = 0; x < ref.width; ++x) {
            double r[3];
            bool ok = unproject(ref, x, y, r);
            size_t i = (size_t)y * ref.width + x;
            ctx.ray_ok[i] = ok;
            ctx.ray[i] = {r[0], r[1], r[2]};
        }
}

// Soft-argmin of one pixel: costs C (K, +inf = invalid) and inverse ranges
// rho; weights s (K), E = sum s rho and (if S != NULL) the soft minimum S.
// False when no plane is valid.
bool soft_argmin(const double* C, const double* rho, int K, double T, double* s, double* E, double* S = nullptr) {
    double m = INF;
    for (int k = 0; k < K; ++k)
        if (C[k] < m) m = C[k];
    if (!(m < INF)) return false;
    double Z = 0.0;
    for (int k = 0; k < K; ++k) {
        s[k] = C[k] < INF ? std::exp(-(C[k] - m) / T) : 0.0;
        Z += s[k];
    }
    *E = 0.0;
    for (int k = 0; k < K; ++k) {
        s[k] /= Z;
        *E += s[k] * rho[k];
    }
    if (S) *S = m - T * std::log(Z);
    return true;
}

// Costs (min over cameras), the attaining camera and inverse ranges of one pixel.
bool soft_pixel_costs(const LevelCtx& ctx, const OrPose* poses, int px, int py, std::vector<double>& C,
                      std::vector<int>& jbest, std::vector<double>& rho) {
    int K = (int)ctx.planes.size();
    C.assign(K, INF);
    jbest.assign(K, -1);
    rho.assign(K, 0.0);
    int r = ctx.rho;
    if (!(px >= r && py >= r && px < ctx.ref.width - r && py < ctx.ref.height - r)) return false;
    size_t i = (size_t)py * ctx.ref.width + px;
    if (!ctx.ray_ok[i]) return false;
    const double* ray = ctx.ray[i].data();
    for (int k = 0; k < K; ++k) {
        const PlaneH& P = ctx.planes[k];
        rho[k] = (P.n[0] * ray[0] + P.n[1] * ray[1] + P.n[2] * ray[2]) / P.d;
        for (int j = 0; j < (int)ctx.cams.size(); ++j) {
            double c = window_cost(ctx, poses[j], j, P, px, py);
            if (c < C[k]) {
                C[k] = c;
                jbest[k] = j;
            }
        }
    }
    return true;
}

// Dense TSDF grid (differentiable fusion): voxel v of block b holds {D, w}
// at vox[2 (512 b + v)], block b = bx + nbx (by + nby bz), v = x + 8 y + 64 z.
struct DenseGrid {
    int nbx, nby, nbz;
    double origin[3], voxel, mu, w_max;
};

// Observation of one voxel by one depth map (Sec. III-C): eta and the pixel,
// or false when the voxel is not updated (no projection, no depth, eta < -mu).
bool dense_voxel_obs(const DenseGrid& G, int gx, int gy, int gz, const float* depth, const OrCamera& cam,
                     const OrPose& w2c, double Xc[3], double* eta, size_t* pix) {
    double X[3] = {G.origin[0] + (gx + 0.5) * G.voxel, G.origin[1] + (gy + 0.5) * G.voxel,
                   G.origin[2] + (gz + 0.5) * G.voxel};
    apply(w2c, X, Xc);
    double u, v;
    if (!project(cam, Xc, &u, &v)) return false;
    double pu = std::floor(u + 0.5), pv = std::floor(v + 0.5);
    if (pu < 0 || pv < 0 || pu >= cam.width || pv >= cam.height) return false;
    *pix = (size_t)pv * cam.width + (size_t)pu;
    double dm = depth[*pix];
    if (!(dm > 0.0) || !std::isfinite(dm)) return false;
    *eta = dm - norm3(Xc);
    return *eta >= -G.mu;
}

}  // namespace

// ===================================================================== C ABI

extern "C" {

// Threads the pixel and block loops use (OpenMP build); returns the count in
// effect.  n <= 0 leaves it unchanged.  Without OpenMP everything runs on one.
int orc_set_threads(int32_t n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_project(const OrCamera* c, const double* X, double* uv) { return project(*c, X, &uv[0], &uv[1]); }

int orc_unproject(const OrCamera* c, double u, double v, double* r) { return unproject(*c, u, v, r); }

void orc_distort(const OrCamera* c, double x, double y, double* out) { distort(*c, x, y, &out[0], &out[1]); }

int orc_undistort(const OrCamera* c, double xd, double yd, double* out) {
    return undistort(*c, xd, yd, &out[0], &out[1]);
}

// ZNCC of two n-vectors; returns 0 if undefined (flat), else 1 and *out.
int orc_zncc(const double* a, const double* b, int32_t n, double* out) { return zncc(a, b, n, out); }

// Plane list of a level: n (K x 3), d (K), set index (K), local index (K).
int32_t orc_level_planes(const OrLevel* L, double* n, double* d, int32_t* set, int32_t* local) {
    LevelCtx ctx;
    make_planes(*L, ctx);
    for (size_t k = 0; k < ctx.planes.size(); ++k) {
        for (int i = 0; i < 3; ++i) n[3 * k + i] = ctx.planes[k].n[i];
        d[k] = ctx.planes[k].d;
        set[k] = ctx.planes[k].family_set;
        local[k] = ctx.planes[k].local;
    }
    return (int32_t)ctx.planes.size();
}

// Level camera and level image of the reference (for tests of the multi-scale step).
void orc_level_ref(const OrCamera* ref_full, const OrLevel* L, const uint8_t* ref_img, OrCamera* cam_out,
                   double* img_out) {
    const uint8_t* imgs[1] = {ref_img};
    LevelCtx ctx;
    OrLevel L2 = *L;
    L2.n_sets = 0;
    build_level(*ref_full, 0, nullptr, L2, imgs, ctx);
    *cam_out = ctx.ref;
    std::memcpy(img_out, ctx.ref_img.px.data(), ctx.ref_img.px.size() * sizeof(double));
}

// Warped sample for tests of the warp: value of camera j's level image at the
// warp of reference level pixel (qx, qy) through plane k.  Returns validity.
int orc_warped_sample(const OrCamera* ref_full, int32_t n_cams, const OrCamera* cams_full, const OrPose* poses,
                      const OrLevel* L, const uint8_t* const* images, int32_t j, int32_t k, int32_t qx, int32_t qy,
                      double* w) {
    LevelCtx ctx;
    build_level(*ref_full, n_cams, cams_full, *L, images, ctx);
    return warped_sample(ctx, poses[j], j, ctx.planes[k], qx, qy, w);
}

// Sweep of one level.  pix: n_pix (x, y) pairs in level coordinates, or NULL
// for every level pixel in row-major order (n_pix is then ignored).  Outputs
// per pixel: range depth (0 = invalid), best and second-best cost (+inf when
// absent), winning plane index (-1 = none) and, if costs != NULL, the K
// aggregated costs.  Returns the number of pixels computed.
int64_t orc_sweep_level(const OrCamera* ref_full, int32_t n_cams, const OrCamera* cams_full, const OrPose* poses,
                        const OrLevel* L, const uint8_t* const* images, int64_t n_pix, const int32_t* pix,
                        double* depth, double* c1, double* c2, int32_t* kstar, double* costs) {
    LevelCtx ctx;
    build_level(*ref_full, n_cams, cams_full, *L, images, ctx);
    int64_t n = pix ? n_pix : (int64_t)ctx.ref.width * ctx.ref.height;
    int K = (int)ctx.planes.size();
    // Pixels are independent: with OpenMP they are shared among threads, each
    // pixel still computed by the same sequential code.
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        int x = pix ? pix[2 * i] : (int)(i % ctx.ref.width);
        int y = pix ? pix[2 * i + 1] : (int)(i / ctx.ref.width);
        PixelResult R = sweep_pixel(ctx, *L, poses, x, y, costs ? costs + i * K : nullptr);
        depth[i] = R.depth;
        c1[i] = R.c1;
        c2[i] = R.c2;
        kstar[i] = R.kstar;
    }
    return n;
}

// Winner-take-all step alone (for tests): C has K costs, sets given by
// n_sets counts in order.  Outputs kstar, c1, c2, delta.
void orc_wta(const double* C, int32_t K, int32_t n_sets, const int32_t* counts, int32_t* kstar, double* out3) {
    std::vector<int> start, cnt;
    int acc = 0;
    for (int i = 0; i < n_sets; ++i) {
        start.push_back(acc);
        cnt.push_back(counts[i]);
        acc += counts[i];
    }
    int ks;
    wta(C, K, start, cnt, &ks, &out3[0], &out3[1], &out3[2]);
    *kstar = ks;
}

// Multi-scale merge and masking at full resolution.  low: depth of the
// downsampled level (factor s, NULL if none); crop: depth of the centred crop
// (crop_w x crop_h, NULL if none).  A pixel takes the crop's depth where it
// lies in the crop and that depth is valid, else the low level's depth at
// (floor(u/s), floor(v/s)); pixels inside any half-open box become 0.
void orc_merge(int32_t W, int32_t H, const double* low, int32_t s, const double* crop_d, int32_t crop_w,
               int32_t crop_h, const int32_t* boxes, int32_t n_boxes, double* out) {
    int x0 = (W - crop_w) / 2, y0 = (H - crop_h) / 2;
    int Wl = s > 0 ? W / s : 0, Hl = s > 0 ? H / s : 0;
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            double val = 0.0;
            if (low) {
                int lu = std::min(u / s, Wl - 1), lv = std::min(v / s, Hl - 1);
                val = low[(size_t)lv * Wl + lu];
            }
            if (crop_d && u >= x0 && u < x0 + crop_w && v >= y0 && v < y0 + crop_h) {
                double c = crop_d[(size_t)(v - y0) * crop_w + (u - x0)];
                if (c > 0.0) val = c;
            }
            for (int b = 0; b < n_boxes; ++b)
                if (u >= boxes[4 * b] && u < boxes[4 * b + 2] && v >= boxes[4 * b + 1] && v < boxes[4 * b + 3])
                    val = 0.0;
            out[(size_t)v * W + u] = val;
        }
}

// Depth map filtering (Sec. III-A, "Depth map filtering"), then merging and
// masking.  Per level: a pixel is an outlier when its best cost exceeds
// alpha of its image part (alpha_upper above the full-resolution row
// split_row, alpha_lower below), or when its second-best cost is below
// ratio_min times its best cost (the ratio of second to first best measures
// uniqueness).  The surviving level depths are merged as in orc_merge.  On the
// merged map, a pixel keeps its depth only if at least a fraction delta of
// the other pixels of its (2w+1)^2 window inside the image have a depth
// within gamma of it.  Finally the boxes are zeroed.  amb (optional, W x H)
// marks pixels whose outcome a float rounding of a cost (1e-4) or a depth
// (1e-5 relative) could flip.
struct FilterParams {
    double alpha_upper, alpha_lower, split_row, ratio_min, gamma, delta;
    int32_t window;
};

static bool keep_level(double c1, double c2, double alpha, double ratio, bool* amb) {
    const double tol = 1e-4;
    if (std::isfinite(c1) && std::fabs(c1 - alpha) < tol) *amb = true;
    if (std::isfinite(c1) && std::isfinite(c2) && std::fabs(c2 - ratio * c1) < tol * (1.0 + c1)) *amb = true;
    return c1 <= alpha && c2 >= ratio * c1;
}

void orc_filter_frame(int32_t W, int32_t H, const double* low_d, const double* low_c1, const double* low_c2,
                      int32_t s, const double* crop_d, const double* crop_c1, const double* crop_c2, int32_t crop_w,
                      int32_t crop_h, const FilterParams* f, const int32_t* boxes, int32_t n_boxes, double* out,
                      uint8_t* amb) {
    const double split = f->split_row >= 0 ? f->split_row : H / 2.0;
    int x0 = (W - crop_w) / 2, y0 = (H - crop_h) / 2;
    int Wl = s > 0 ? W / s : 0, Hl = s > 0 ? H / s : 0;
    std::vector<double> merged((size_t)W * H, 0.0);
    std::vector<uint8_t> am((size_t)W * H, 0);
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            double val = 0.0;
            bool a = false;
            if (low_d) {
                int lu = std::min(u / s, Wl - 1), lv = std::min(v / s, Hl - 1);
                size_t i = (size_t)lv * Wl + lu;
                double row = s * lv + (s - 1) / 2.0;  // full-resolution row of the level pixel's centre
                double alpha = row < split ? f->alpha_upper : f->alpha_lower;
                if (low_d[i] > 0.0 && keep_level(low_c1[i], low_c2[i], alpha, f->ratio_min, &a)) val = low_d[i];
            }
            if (crop_d && u >= x0 && u < x0 + crop_w && v >= y0 && v < y0 + crop_h) {
                size_t i = (size_t)(v - y0) * crop_w + (u - x0);
                double alpha = v < split ? f->alpha_upper : f->alpha_lower;
                if (crop_d[i] > 0.0 && keep_level(crop_c1[i], crop_c2[i], alpha, f->ratio_min, &a)) val = crop_d[i];
            }
            merged[(size_t)v * W + u] = val;
            am[(size_t)v * W + u] = a;
        }
    const int w = f->window / 2;
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            double d = merged[(size_t)v * W + u];
            double res = 0.0;
            bool a = am[(size_t)v * W + u];
            if (d > 0.0) {
                int cons = 0, tot = 0;
                for (int dy = -w; dy <= w; ++dy)
                    for (int dx = -w; dx <= w; ++dx) {
                        if (dx == 0 && dy == 0) continue;
                        int uu = u + dx, vv = v + dy;
                        if (uu < 0 || vv < 0 || uu >= W || vv >= H) continue;
                        ++tot;
                        double dn = merged[(size_t)vv * W + uu];
                        if (am[(size_t)vv * W + uu]) a = true;  // a neighbour's own depth may flip
                        if (dn > 0.0 && std::fabs(std::fabs(dn - d) - f->gamma) < 1e-5 * (d + dn)) a = true;
                        if (dn > 0.0 && std::fabs(dn - d) < f->gamma) ++cons;
                    }
                if (tot > 0 && cons >= f->delta * tot) res = d;
            }
            for (int b = 0; b < n_boxes; ++b)
                if (u >= boxes[4 * b] && u < boxes[4 * b + 2] && v >= boxes[4 * b + 1] && v < boxes[4 * b + 3]) {
                    res = 0.0;
                    a = false;
                }
            out[(size_t)v * W + u] = res;
            if (amb) amb[(size_t)v * W + u] = a;
        }
}

void* orc_tsdf_new(const TsdfDesc* d) {
    Tsdf* T = new Tsdf();
    T->d = *d;
    if (d->dense_dim[0] > 0) {
        const int B = d->block_dim;
        for (int z = 0; z < d->dense_dim[2] / B; ++z)
            for (int y = 0; y < d->dense_dim[1] / B; ++y)
                for (int x = 0; x < d->dense_dim[0] / B; ++x)
                    T->blocks.emplace(Key{x, y, z}, new_block(B * B * B));
    }
    return T;
}

void orc_tsdf_free(void* h) { delete static_cast<Tsdf*>(h); }

void orc_tsdf_set_bands(void* h, double tau_len, double tau_px, double tau_m, double tau_rel) {
    Tsdf* T = static_cast<Tsdf*>(h);
    T->tau_len = tau_len;
    T->tau_px = tau_px;
    T->tau_m = tau_m;
    T->tau_rel = tau_rel;
}

// One frame: allocation (hashed maps only), then integration.
// depth: H x W float32 range map (0 = invalid); lc: local-map centre or NULL.
void orc_tsdf_integrate(void* h, const float* depth, const OrCamera* cam, const OrPose* w2c, const double* lc) {
    Tsdf* T = static_cast<Tsdf*>(h);
    if (T->d.dense_dim[0] == 0) allocate(*T, depth, *cam, *w2c, lc);
    integrate(*T, depth, *cam, *w2c);
}

int64_t orc_tsdf_count(void* h) { return (int64_t) static_cast<Tsdf*>(h)->blocks.size(); }

// All blocks in key order: keys (n x 3), D and W (n x B^3, voxel x fastest),
// amb (n x B^3: 1 where the voxel's history is rounding-sensitive or its
// block's allocation frame may differ).
void orc_tsdf_dump(void* h, int64_t* keys, double* D, double* W, uint8_t* amb) {
    Tsdf* T = static_cast<Tsdf*>(h);
    const int B3 = T->d.block_dim * T->d.block_dim * T->d.block_dim;
    int64_t i = 0;
    for (auto& kv : T->blocks) {
        for (int k = 0; k < 3; ++k) keys[3 * i + k] = kv.first[k];
        for (int v = 0; v < B3; ++v) {
            D[i * B3 + v] = kv.second.D[v];
            W[i * B3 + v] = kv.second.W[v];
            amb[i * B3 + v] = kv.second.amb[v] | kv.second.block_amb;
        }
        ++i;
    }
}

// Surface points of a block map (Sec. III-C, the extracted map): for every
// voxel a and its +x, +y and +z neighbour b (in the same block or the next
// block along that axis) that both have w >= max(min_w, 1), a sign change of
// D (positive on one side, zero or negative on the other) gives the point
// X_a + t (X_b - X_a), t = D_a / (D_a - D_b), voxel centres at
// origin + (i + 1/2) voxel.  keys: n x 3 block indices; D, W: n x 512 (voxel
// x + 8 y + 64 z).  Writes up to cap points (x, y, z) and edges (global voxel
// index of a, axis); returns the number of points found.
int64_t orc_tsdf_points(int64_t n, const int32_t* keys, const double* D, const double* W, double min_w,
                        const double* origin, double voxel, int64_t cap, double* points, int32_t* edges) {
    std::map<Key, int64_t> index;
    for (int64_t i = 0; i < n; ++i) index[Key{keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]}] = i;
    const double wmin = std::max(min_w, 1.0);
    int64_t found = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t* k = keys + 3 * i;
        for (int v = 0; v < 512; ++v) {
            const int x = v % 8, y = (v / 8) % 8, z = v / 64;
            const double da = D[i * 512 + v];
            if (!(W[i * 512 + v] >= wmin)) continue;
            for (int axis = 0; axis < 3; ++axis) {
                int c[3] = {x, y, z};
                int32_t kb[3] = {k[0], k[1], k[2]};
                c[axis] += 1;
                if (c[axis] == 8) {  // the neighbour lies in the next block along the axis
                    c[axis] = 0;
                    kb[axis] += 1;
                }
                auto it = index.find(Key{kb[0], kb[1], kb[2]});
                if (it == index.end()) continue;
                const int64_t j = it->second;
                const int vb = c[0] + 8 * c[1] + 64 * c[2];
                if (!(W[j * 512 + vb] >= wmin)) continue;
                const double db = D[j * 512 + vb];
                if ((da > 0.0) == (db > 0.0)) continue;
                const double t = da / (da - db);
                const int g[3] = {k[0] * 8 + x, k[1] * 8 + y, k[2] * 8 + z};
                if (found < cap) {
                    for (int q = 0; q < 3; ++q) {
                        double xa = origin[q] + (g[q] + 0.5) * voxel;
                        points[3 * found + q] = xa + (q == axis ? t * voxel : 0.0);
                        edges[4 * found + q] = g[q];
                    }
                    edges[4 * found + 3] = axis;
                }
                ++found;
            }
        }
    }
    return found;
}

// Last frame's allocation report: counts of the strict set (blocks any
// correct implementation allocates) and the ambiguous band.
void orc_tsdf_alloc_counts(void* h, int64_t* n_strict, int64_t* n_maybe) {
    Tsdf* T = static_cast<Tsdf*>(h);
    *n_strict = (int64_t)T->last_strict.size();
    *n_maybe = (int64_t)T->last_maybe.size();
}

void orc_tsdf_alloc_sets(void* h, int64_t* strict, int64_t* maybe) {
    Tsdf* T = static_cast<Tsdf*>(h);
    int64_t i = 0;
    for (const Key& k : T->last_strict) {
        for (int j = 0; j < 3; ++j) strict[3 * i + j] = k[j];
        ++i;
    }
    i = 0;
    for (const Key& k : T->last_maybe) {
        for (int j = 0; j < 3; ++j) maybe[3 * i + j] = k[j];
        ++i;
    }
}

// Local-map swap-out (Sec. III-C: blocks that are no longer in the local map
// are swapped out of GPU memory): remove every block whose centre lies
// outside the box of half extents local_half around lc, returning the removed
// blocks in key order.  n_amb counts removed or kept blocks whose centre lies
// within tau_len of the box (a float rounding may decide them either way);
// their keys come first in amb_keys when given.
int64_t orc_tsdf_swap_out(void* h, const double* lc, int64_t* keys, double* D, double* W, int64_t* n_amb,
                          int64_t* amb_keys) {
    Tsdf* T = static_cast<Tsdf*>(h);
    const TsdfDesc& d = T->d;
    const int B = d.block_dim;
    const int B3 = B * B * B;
    const double L = B * d.voxel_size;
    int64_t n = 0, na = 0;
    for (auto it = T->blocks.begin(); it != T->blocks.end();) {
        double margin = INF;
        for (int i = 0; i < 3; ++i) {
            double c = d.origin[i] + (it->first[i] + 0.5) * L;
            margin = std::min(margin, d.local_half[i] - std::fabs(c - lc[i]));
        }
        if (std::fabs(margin) < T->tau_len) {
            if (amb_keys)
                for (int k = 0; k < 3; ++k) amb_keys[3 * na + k] = it->first[k];
            ++na;
        }
        if (margin < 0.0) {
            if (keys) {
                for (int k = 0; k < 3; ++k) keys[3 * n + k] = it->first[k];
                for (int v = 0; v < B3; ++v) {
                    D[n * B3 + v] = it->second.D[v];
                    W[n * B3 + v] = it->second.W[v];
                }
            }
            ++n;
            it = T->blocks.erase(it);
        } else {
            ++it;
        }
    }
    if (n_amb) *n_amb = na;
    return n;
}

// Load blocks (checkpoint resume, swap-in): insert or overwrite each block's voxels.
void orc_tsdf_load(void* h, int64_t n, const int64_t* keys, const double* D, const double* W) {
    Tsdf* T = static_cast<Tsdf*>(h);
    const int B3 = T->d.block_dim * T->d.block_dim * T->d.block_dim;
    for (int64_t i = 0; i < n; ++i) {
        Key k = {keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]};
        auto it = T->blocks.find(k);
        if (it == T->blocks.end()) it = T->blocks.emplace(k, new_block(B3)).first;
        for (int v = 0; v < B3; ++v) {
            it->second.D[v] = D[i * B3 + v];
            it->second.W[v] = W[i * B3 + v];
            it->second.amb[v] = 0;
        }
        it->second.block_amb = 0;
    }
}

// Blocks ever in an ambiguous allocation band (for set comparisons).
int64_t orc_tsdf_ever_maybe(void* h, int64_t* keys) {
    Tsdf* T = static_cast<Tsdf*>(h);
    int64_t i = 0;
    if (keys)
        for (const Key& k : T->ever_maybe) {
            for (int j = 0; j < 3; ++j) keys[3 * i + j] = k[j];
            ++i;
        }
    return (int64_t)T->ever_maybe.size();
}

// ---------------------------------------------------------------- differentiable forms (C API)

void orc_project_jacobian(const OrCamera* c, const double* X, double* J) { project_jacobian(*c, X, J); }

int orc_soft_argmin(const double* C, const double* rho, int32_t K, double T, double* s, double* E, double* S) {
    return soft_argmin(C, rho, K, T, s, E, S);
}

// Soft-argmin range map of one full-resolution level of real-valued images
// (ref, then the matching cameras) and the soft-minimum cost map (cost may be
// NULL); both 0 where no plane is valid.
void orc_soft_depth(const OrCamera* ref, int32_t n_cams, const OrCamera* cams, const OrPose* poses,
                    const OrLevel* L, const double* const* images, double T, double* range, double* cost) {
    LevelCtx ctx;
    build_level_real(*ref, n_cams, cams, *L, images, ctx);
    const int K = (int)ctx.planes.size();
    std::vector<double> C, rho, sw(K);
    std::vector<int> jb;
    for (int y = 0; y < ref->height; ++y)
        for (int x = 0; x < ref->width; ++x) {
            double E = 0.0, S = 0.0;
            size_t i = (size_t)y * ref->width + x;
            range[i] = 0.0;
            if (cost) cost[i] = 0.0;
            if (soft_pixel_costs(ctx, poses, x, y, C, jb, rho) &&
                soft_argmin(C.data(), rho.data(), K, T, sw.data(), &E, &S)) {
                range[i] = 1.0 / E;
                if (cost) cost[i] = S;
            }
        }
}

// Pixels whose soft-argmin gradient depends on a floating-point decision:
// some valid plane's two lowest camera costs lie within tau of each other
// (float rounding may route that plane's gradient to either camera), or a
// window sample of the winning camera lies within tau_px of a pixel-grid
// line (the bilinear slope, which the pose gradient uses, jumps there).
// amb: one byte per pixel, 1 = marked.
void orc_soft_depth_ties(const OrCamera* ref, int32_t n_cams, const OrCamera* cams, const OrPose* poses,
                         const OrLevel* L, const double* const* images, double tau, double tau_px, uint8_t* amb) {
    LevelCtx ctx;
    build_level_real(*ref, n_cams, cams, *L, images, ctx);
    const int K = (int)ctx.planes.size(), r = ctx.rho;
    for (int y = 0; y < ref->height; ++y)
        for (int x = 0; x < ref->width; ++x) {
            uint8_t a = 0;
            if (x >= r && y >= r && x < ref->width - r && y < ref->height - r)
                for (int k = 0; k < K && !a; ++k) {
                    double c1 = INF, c2 = INF;
                    int jb = -1;
                    for (int j = 0; j < n_cams; ++j) {
                        double c = window_cost(ctx, poses[j], j, ctx.planes[k], x, y);
                        if (c < c1) {
                            c2 = c1;
                            c1 = c;
                            jb = j;
                        } else if (c < c2) {
                            c2 = c;
                        }
                    }
                    if (c2 < INF && c2 - c1 < tau) a = 1;
                    if (jb < 0 || tau_px <= 0.0) continue;
                    const PlaneH& P = ctx.planes[k];
                    for (int dy = -r; dy <= r && !a; ++dy)
                        for (int dx = -r; dx <= r && !a; ++dx) {
                            const double* ray = ctx.ray[(size_t)(y + dy) * ref->width + (x + dx)].data();
                            const double lam = P.d / (P.n[0] * ray[0] + P.n[1] * ray[1] + P.n[2] * ray[2]);
                            double X[3] = {lam * ray[0], lam * ray[1], lam * ray[2]}, Xj[3], u, v;
                            apply(poses[jb], X, Xj);
                            project(ctx.cams[jb], Xj, &u, &v);
                            if (frac_dist(u) < tau_px || frac_dist(v) < tau_px) a = 1;
                        }
                }
            amb[(size_t)y * ref->width + x] = a;
        }
}

// Gradient of L = sum_p g(p) range(p) + gs(p) S(p) (gs may be NULL) with respect to the images (g_images:
// one array per image, ADDED to) and to left perturbations of each
// ref_to_cam pose, T_j <- exp([w]x, v) T_j (g_pose: 6 per camera, (w, v),
// ADDED to).  Chain: range = 1/E; dE/dC_k = -s_k (rho_k - E) / T; C_k is the
// winning camera's (1 - ZNCC) / 2; ZNCC's derivative with respect to each
// window sample of either window; bilinear weights (image) and the bilinear
// slope times the projection Jacobian (pose: dX_j = w x X_j + v).
void orc_soft_depth_grad(const OrCamera* ref, int32_t n_cams, const OrCamera* cams, const OrPose* poses,
                         const OrLevel* L, const double* const* images, double T, const double* g,
                         const double* gs, double* const* g_images, double* g_pose) {
    LevelCtx ctx;
    build_level_real(*ref, n_cams, cams, *L, images, ctx);
    const int K = (int)ctx.planes.size(), r = ctx.rho, N = (2 * r + 1) * (2 * r + 1);
    std::vector<double> C, rho, sw(K);
    std::vector<int> jb;
    std::vector<double> a(N), b(N);
    for (int py = 0; py < ref->height; ++py)
        for (int px = 0; px < ref->width; ++px) {
            const double gp = g ? g[(size_t)py * ref->width + px] : 0.0;
            const double gsp = gs ? gs[(size_t)py * ref->width + px] : 0.0;
            double E = 0.0;
            if (gp == 0.0 && gsp == 0.0) continue;
            if (!soft_pixel_costs(ctx, poses, px, py, C, jb, rho)) continue;
            if (!soft_argmin(C.data(), rho.data(), K, T, sw.data(), &E)) continue;
            const double gE = -gp / (E * E);
            for (int k = 0; k < K; ++k) {
                if (!(C[k] < INF)) continue;
                const double gC = gE * (-sw[k] * (rho[k] - E) / T) + gsp * sw[k];
                const int j = jb[k];
                const PlaneH& P = ctx.planes[k];
                // the two windows of the winning camera
                int n = 0;
                for (int dy = -r; dy <= r; ++dy)
                    for (int dx = -r; dx <= r; ++dx) {
                        a[n] = ctx.ref_img.at(px + dx, py + dy);
                        warped_sample(ctx, poses[j], j, P, px + dx, py + dy, &b[n]);
                        ++n;
                    }
                double ma = 0, mb = 0;
                for (int q = 0; q < N; ++q) {
                    ma += a[q];
                    mb += b[q];
                }
                ma /= N;
                mb /= N;
                double cov = 0, va = 0, vb = 0;
                for (int q = 0; q < N; ++q) {
                    cov += (a[q] - ma) * (b[q] - mb);
                    va += (a[q] - ma) * (a[q] - ma);
                    vb += (b[q] - mb) * (b[q] - mb);
                }
                const double sab = std::sqrt(va * vb), z = cov / sab;
                const double gz = -0.5 * gC;  // cost = (1 - z) / 2
                n = 0;
                for (int dy = -r; dy <= r; ++dy)
                    for (int dx = -r; dx <= r; ++dx, ++n) {
                        const int qx = px + dx, qy = py + dy;
                        const double dza = (b[n] - mb) / sab - z * (a[n] - ma) / va;
                        const double dzb = (a[n] - ma) / sab - z * (b[n] - mb) / vb;
                        g_images[0][(size_t)qy * ref->width + qx] += gz * dza;
                        const double gb = gz * dzb;
                        // the warp of q: X on the plane, X_j in camera j, (u, v), bilinear
                        const double* ray = ctx.ray[(size_t)qy * ref->width + qx].data();
                        const double lam = P.d / (P.n[0] * ray[0] + P.n[1] * ray[1] + P.n[2] * ray[2]);
                        double X[3] = {lam * ray[0], lam * ray[1], lam * ray[2]}, Xj[3];
                        apply(poses[j], X, Xj);
                        double u, v;
                        project(ctx.cams[j], Xj, &u, &v);
                        const Image& I = ctx.cam_img[j];
                        int x0 = (int)std::floor(u), y0 = (int)std::floor(v);
                        double ax = u - x0, ay = v - y0;
                        int x1 = std::min(x0 + 1, I.W - 1), y1 = std::min(y0 + 1, I.H - 1);
                        double* G = g_images[1 + j];
                        G[(size_t)y0 * I.W + x0] += gb * (1 - ax) * (1 - ay);
                        G[(size_t)y0 * I.W + x1] += gb * ax * (1 - ay);
                        G[(size_t)y1 * I.W + x0] += gb * (1 - ax) * ay;
                        G[(size_t)y1 * I.W + x1] += gb * ax * ay;
                        const double dwdu = (1 - ay) * (I.at(x1, y0) - I.at(x0, y0)) + ay * (I.at(x1, y1) - I.at(x0, y1));
                        const double dwdv = (1 - ax) * (I.at(x0, y1) - I.at(x0, y0)) + ax * (I.at(x1, y1) - I.at(x1, y0));
                        double J[6];
                        project_jacobian(ctx.cams[j], Xj, J);
                        double gX[3];
                        for (int i = 0; i < 3; ++i) gX[i] = gb * (dwdu * J[i] + dwdv * J[3 + i]);
                        double* gp6 = g_pose + 6 * j;
                        gp6[0] += Xj[1] * gX[2] - Xj[2] * gX[1];  // w: X_j x gX
                        gp6[1] += Xj[2] * gX[0] - Xj[0] * gX[2];
                        gp6[2] += Xj[0] * gX[1] - Xj[1] * gX[0];
                        gp6[3] += gX[0];                          // v
                        gp6[4] += gX[1];
                        gp6[5] += gX[2];
                    }
            }
        }
}

// Differentiable fusion of one depth map into a dense grid (Sec. III-C,
// Eq. 2 with unit observation weight): out = in, then every observed voxel
// D <- (w D + min(1, eta/mu)) / (w + 1), w <- min(w + 1, w_max).
void orc_dense_fuse(const int32_t* nb, const double* origin, double voxel, double mu, double w_max,
                    const double* vox_in, const float* depth, const OrCamera* cam, const OrPose* w2c,
                    double* vox_out) {
    DenseGrid G{nb[0], nb[1], nb[2], {origin[0], origin[1], origin[2]}, voxel, mu, w_max};
    const size_t n = (size_t)nb[0] * nb[1] * nb[2] * 512;
    std::memcpy(vox_out, vox_in, sizeof(double) * 2 * n);
    for (size_t i = 0; i < n; ++i) {
        size_t b = i / 512, v = i % 512;
        int gx = (int)(b % nb[0]) * 8 + (int)(v % 8), gy = (int)((b / nb[0]) % nb[1]) * 8 + (int)((v / 8) % 8),
            gz = (int)(b / ((size_t)nb[0] * nb[1])) * 8 + (int)(v / 64);
        double Xc[3], eta;
        size_t pix;
        if (!dense_voxel_obs(G, gx, gy, gz, depth, *cam, *w2c, Xc, &eta, &pix)) continue;
        double w = vox_in[2 * i + 1];
        vox_out[2 * i] = (w * vox_in[2 * i] + std::min(1.0, eta / mu)) / (w + 1.0);
        vox_out[2 * i + 1] = std::min(w + 1.0, w_max);
    }
}

// Gradient of L = sum_i gD[i] D_out[i] (the weights are counts: no gradient)
// with respect to D_in (written), the depth map (ADDED to) and a left
// perturbation of world_to_cam, X_c <- exp([w]x, v) X_c (6 values, ADDED to).
// An observed voxel passes w / (w + 1) to D_in; when eta < mu it passes
// 1 / (mu (w + 1)) to its pixel's depth, and minus that times X_c / |X_c| to X_c.
void orc_dense_fuse_grad(const int32_t* nb, const double* origin, double voxel, double mu, double w_max,
                         const double* vox_in, const float* depth, const OrCamera* cam, const OrPose* w2c,
                         const double* gD, double* gD_in, double* g_depth, double* g_pose) {
    DenseGrid G{nb[0], nb[1], nb[2], {origin[0], origin[1], origin[2]}, voxel, mu, w_max};
    const size_t n = (size_t)nb[0] * nb[1] * nb[2] * 512;
    for (size_t i = 0; i < n; ++i) {
        size_t b = i / 512, v = i % 512;
        int gx = (int)(b % nb[0]) * 8 + (int)(v % 8), gy = (int)((b / nb[0]) % nb[1]) * 8 + (int)((v / 8) % 8),
            gz = (int)(b / ((size_t)nb[0] * nb[1])) * 8 + (int)(v / 64);
        double Xc[3], eta;
        size_t pix;
        gD_in[i] = gD[i];
        if (!dense_voxel_obs(G, gx, gy, gz, depth, *cam, *w2c, Xc, &eta, &pix)) continue;
        double w = vox_in[2 * i + 1];
        gD_in[i] = gD[i] * w / (w + 1.0);
        if (!(eta < mu)) continue;  // truncated at 1: no dependence on eta
        double ge = gD[i] / (mu * (w + 1.0));
        g_depth[pix] += ge;
        double nrm = norm3(Xc), gX[3];
        for (int k = 0; k < 3; ++k) gX[k] = -ge * Xc[k] / nrm;
        g_pose[0] += Xc[1] * gX[2] - Xc[2] * gX[1];
        g_pose[1] += Xc[2] * gX[0] - Xc[0] * gX[2];
        g_pose[2] += Xc[0] * gX[1] - Xc[1] * gX[0];
        g_pose[3] += gX[0];
        g_pose[4] += gX[1];
        g_pose[5] += gX[2];
    }
}

}  // extern "C"

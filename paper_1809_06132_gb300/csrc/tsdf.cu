// TSDF fusion of fisheye depth maps into voxel blocks (Sec. III-C) on sm_103a.
//
// Per frame (all asynchronous on the caller's stream, no host sync):
//   depth_max_kernel  largest range of the frame (bounds the visible test)
//   alloc_kernel      per valid pixel: the blocks crossed by the segment
//                     [d - mu, d + mu] of its ray (slab test of the segment
//                     against each block of its bounding box), gated by the
//                     local map, inserted into an open-addressing hash table
//                     (bounded linear probing; overflow latches a status)
//   visible_kernel    allocated blocks that some pixel of this frame can
//                     update: a conservative sphere test on range and view
//                     angle, compacted into a list
//   integrate_kernel  Eq. 2 on every voxel of the listed blocks: one CTA per
//                     block, 256 threads x 2 voxels, 16-byte loads and
//                     stores of the interleaved {D, w} pairs
//   extract_kernel    copy-out with the minimum-observation filter
//   points_kernel     surface points at sign changes between observed neighbour voxels
//
// The signed distance eta = d - |X_d| subtracts two ranges of tens of
// metres; float32 alone would lose ~1e-5 m there.  The kernel therefore
// carries the voxel-to-camera offset as an exact integer voxel offset plus a
// sub-voxel remainder, forms |X_d|^2 with an exact integer part, and
// refines sqrt with one Newton step in split (hi + lo) float arithmetic, so
// eta keeps ~1e-7 m absolute accuracy at any range.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace ps {
namespace {

constexpr int B = 8;            // voxels per block edge
constexpr int B3 = B * B * B;   // voxels per block
constexpr int IT = 256;         // integrate threads per block (2 voxels each)
constexpr unsigned long long EMPTY = ~0ull;
constexpr int MAX_PROBE = 4096;
constexpr long long MAX_CANDIDATES = 4096;  // blocks in one segment's bounding box

__host__ __device__ __forceinline__ unsigned long long pack_key(int x, int y, int z) {
    return ((unsigned long long)(x + (1 << 20)) & 0x1FFFFF) | (((unsigned long long)(y + (1 << 20)) & 0x1FFFFF) << 21) |
           (((unsigned long long)(z + (1 << 20)) & 0x1FFFFF) << 42);
}

// The 64-bit finalising mix of MurmurHash3 (fmix64): two multiplications
// and three xor-shifts that spread every key bit over the whole word.
__device__ __forceinline__ unsigned long long hash64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

struct FrameP {
    // camera (float) and pose
    CamF cam;
    float R[9];        // world -> camera rotation
    float Rt[9];       // camera -> world rotation
    float C[3];        // camera centre relative to the grid origin (m)
    int ic[3];         // camera centre in voxel units: ic + fc = (C_world - origin) / voxel
    float fb[3];       // 1/2 - fc: sub-voxel part of a voxel centre's offset from the camera
    float vox, vox_lo; // voxel size split into float hi + lo
    float mu, inv_mu, w_max;
    float block;       // block edge (m)
    // local-map gate (block centre within half of centre), relative to origin
    int gate;
    float lc[3], lh[3];
    // visible test
    float cos_view;    // cosine of the widest view angle of a valid ray (margin included)
    float view_angle;
};

struct TsdfDev {
    unsigned long long* hkeys;
    int* hvals;
    long long slot_mask;
    float2* vox;
    int4* pool_keys;     // (bx, by, bz, 0); w = -1 marks a freed slot
    int* n_alloc;        // slots handed out so far (freed ones included)
    int* free_stack;     // freed slots, reused before the pool grows
    int* free_top;       // entries on the free stack (may run below zero while allocating)
    int pool_cap;
    int* vis;
    int* n_vis;
    unsigned* status;
    unsigned* dmax_bits;
    const float4* rays;  // depth camera rays (camera frame), NaN = none
    int n_parts, part;   // hash partition: allocate only blocks with owner(key) == part
};

// Owner of a block among n_parts maps: the high half of the key's hash (the
// slot index uses the low bits, so each part still spreads over the table).
__device__ __forceinline__ int block_owner(int bx, int by, int bz, int n_parts) {
    return (int)((hash64(pack_key(bx, by, bz)) >> 32) % (unsigned long long)n_parts);
}

// ----------------------------------------------------------------- hash

// Insert (or find) a block key; returns its pool index or -1 on failure.
__device__ int hash_insert(const TsdfDev& T, int bx, int by, int bz) {
    unsigned long long key = pack_key(bx, by, bz);
    long long h = (long long)(hash64(key) & (unsigned long long)T.slot_mask);
    for (int probe = 0; probe < MAX_PROBE; ++probe) {
        unsigned long long k = *((volatile unsigned long long*)&T.hkeys[h]);
        if (k == key) {
            // a block that found no room in the pool stays unstored; say so on every frame that needs it
            if (*((volatile int*)&T.hvals[h]) == -2) atomicOr(T.status, DEV_CAPACITY);
            return 0;
        }
        if (k == EMPTY) {
            unsigned long long prev = atomicCAS(&T.hkeys[h], EMPTY, key);
            if (prev == EMPTY) {
                int idx = -1;
                if (T.free_top) {
                    int top = atomicSub(T.free_top, 1);
                    if (top > 0) idx = T.free_stack[top - 1];
                }
                if (idx < 0) idx = atomicAdd(T.n_alloc, 1);
                if (idx >= T.pool_cap) {
                    atomicOr(T.status, DEV_CAPACITY);
                    T.hvals[h] = -2;
                    return -1;
                }
                T.pool_keys[idx] = make_int4(bx, by, bz, 0);
                T.hvals[h] = idx;
                return 0;
            }
            if (prev == key) {
                if (*((volatile int*)&T.hvals[h]) == -2) atomicOr(T.status, DEV_CAPACITY);
                return 0;
            }
        }
        h = (h + 1) & T.slot_mask;
    }
    atomicOr(T.status, DEV_TIMEOUT | DEV_CAPACITY);
    return -1;
}

// ----------------------------------------------------------------- kernels

__global__ void depth_max_kernel(const float* depth, int n, unsigned* dmax_bits) {
    float m = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float d = depth[i];
        if (d > m && d < 3.0e38f) m = d;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(dmax_bits, __float_as_uint(m));
}

// Length of segment [A, B] inside box [lo, hi] (slab method).
__device__ __forceinline__ float seg_box(const float A[3], const float D[3], const float lo[3], const float hi[3]) {
    float t0 = 0.f, t1 = 1.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (D[k] == 0.f) {
            if (A[k] < lo[k] || A[k] > hi[k]) return 0.f;
            continue;
        }
        float inv = 1.0f / D[k];
        float ta = (lo[k] - A[k]) * inv, tb = (hi[k] - A[k]) * inv;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    }
    return t1 > t0 ? (t1 - t0) : 0.f;
}

__global__ void alloc_kernel(const __grid_constant__ FrameP F, TsdfDev T, const float* depth) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y;
    if (u >= F.cam.width || v >= F.cam.height) return;
    size_t o = (size_t)v * F.cam.width + u;
    float d = depth[o];
    if (!(d > 0.f) || !(d < 3.0e38f)) return;
    float4 r = T.rays[o];
    if (isnan(r.x)) return;
    float dw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dw[i] = F.Rt[3 * i] * r.x + F.Rt[3 * i + 1] * r.y + F.Rt[3 * i + 2] * r.z;
    float s0 = fmaxf(0.f, d - F.mu), s1 = d + F.mu;
    float A[3], Dv[3];
    int lo[3], hi[3];
    long long n_cand = 1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        A[i] = fmaf(s0, dw[i], F.C[i]);
        float Bp = fmaf(s1, dw[i], F.C[i]);
        Dv[i] = Bp - A[i];
        float flo = floorf(fminf(A[i], Bp) / F.block), fhi = floorf(fmaxf(A[i], Bp) / F.block);
        if (F.gate) {
            // only blocks whose centre lies in the local map can be allocated:
            // clip the candidates to the gate's index range (one block of slack;
            // the exact centre test below decides)
            flo = fmaxf(flo, floorf((F.lc[i] - F.lh[i]) / F.block - 0.5f) - 1.0f);
            fhi = fminf(fhi, floorf((F.lc[i] + F.lh[i]) / F.block - 0.5f) + 1.0f);
            if (flo > fhi) return;
        }
        // block keys hold 21-bit signed indices; a segment outside that range cannot be stored
        if (!(flo >= -1048575.f && fhi <= 1048575.f)) {
            atomicOr(T.status, DEV_CAPACITY);
            return;
        }
        lo[i] = (int)flo;
        hi[i] = (int)fhi;
        n_cand *= (long long)(hi[i] - lo[i] + 1);
    }
    if (n_cand > MAX_CANDIDATES) {  // segment spans more blocks than any sane mu / block ratio gives
        atomicOr(T.status, DEV_CAPACITY);
        return;
    }
    for (int bz = lo[2]; bz <= hi[2]; ++bz)
        for (int by = lo[1]; by <= hi[1]; ++by)
            for (int bx = lo[0]; bx <= hi[0]; ++bx) {
                float blo[3] = {bx * F.block, by * F.block, bz * F.block};
                float bhi[3] = {(bx + 1) * F.block, (by + 1) * F.block, (bz + 1) * F.block};
                if (seg_box(A, Dv, blo, bhi) <= 0.f) continue;
                if (F.gate) {
                    float c0 = (bx + 0.5f) * F.block, c1 = (by + 0.5f) * F.block, c2 = (bz + 0.5f) * F.block;
                    if (fabsf(c0 - F.lc[0]) > F.lh[0] || fabsf(c1 - F.lc[1]) > F.lh[1] ||
                        fabsf(c2 - F.lc[2]) > F.lh[2])
                        continue;
                }
                if (T.n_parts > 1 && block_owner(bx, by, bz, T.n_parts) != T.part) continue;
                hash_insert(T, bx, by, bz);
            }
}

// Blocks a pixel of this frame can update: within range dmax + mu of the
// camera (eta >= -mu needs |X_d| <= d + mu) and inside the widest view cone
// (both tested on the block's bounding sphere).
__global__ void visible_kernel(const __grid_constant__ FrameP F, TsdfDev T) {
    int n = min(*T.n_alloc, T.pool_cap);
    float dmax = __uint_as_float(*T.dmax_bits);
    float rb = F.block * 0.8660254f * 1.001f + 1e-4f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int4 k = T.pool_keys[i];
        if (k.w < 0) continue;  // freed slot
        float c[3] = {(k.x + 0.5f) * F.block - F.C[0], (k.y + 0.5f) * F.block - F.C[1],
                      (k.z + 0.5f) * F.block - F.C[2]};
        float Xc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) Xc[a] = F.R[3 * a] * c[0] + F.R[3 * a + 1] * c[1] + F.R[3 * a + 2] * c[2];
        float dist = sqrtf(Xc[0] * Xc[0] + Xc[1] * Xc[1] + Xc[2] * Xc[2]);
        bool vis = dmax > 0.f && dist - rb <= dmax + F.mu;
        if (vis && dist > rb) {
            float ang = acosf(fminf(1.f, fmaxf(-1.f, Xc[2] / dist)));
            float half = asinf(fminf(1.f, rb / dist));
            vis = ang - half <= F.view_angle;
        }
        if (vis) {
            int slot = atomicAdd(T.n_vis, 1);
            T.vis[slot] = i;
        }
    }
}

// Observation of a voxel by the depth map (Sec. III-C): eta, the pixel index
// and the point in the camera frame.  a = voxel index - camera voxel (exact
// int), F.fb the sub-voxel part, so the voxel centre sits at vox * (a + fb)
// from the camera.  False when the voxel does not project into the image or
// its pixel has no depth; eta < -mu is left to the caller.
__device__ __forceinline__ bool observe_voxel(const FrameP& F, const float* depth, int ax, int ay, int az, float* eta_out,
                                              size_t* pix_out, float Xc[3]) {
    const CamF& c = F.cam;
    float bx = F.fb[0], by = F.fb[1], bz = F.fb[2];
    float vx = ((float)ax + bx) * F.vox, vy = ((float)ay + by) * F.vox, vz = ((float)az + bz) * F.vox;
    float X = F.R[0] * vx + F.R[1] * vy + F.R[2] * vz;
    float Y = F.R[3] * vx + F.R[4] * vy + F.R[5] * vz;
    float Z = F.R[6] * vx + F.R[7] * vy + F.R[8] * vz;
    // projection (unified model + distortion) and nearest pixel
    float n = sqrtf(fmaf(X, X, fmaf(Y, Y, Z * Z)));
    float inv = 1.0f / fmaf(c.xi, n, Z);
    float mx = X * inv, my = Y * inv;
    float r2 = fmaf(mx, mx, my * my);
    float rad = fmaf(r2, fmaf(c.k2, r2, c.k1), 1.0f);
    float mxy = mx * my;
    float xd = fmaf(mx, rad, fmaf(2.0f * c.p1, mxy, c.p2 * fmaf(2.0f * mx, mx, r2)));
    float yd = fmaf(my, rad, fmaf(c.p1, fmaf(2.0f * my, my, r2), 2.0f * c.p2 * mxy));
    float u = fmaf(c.fx, xd, c.cx), v = fmaf(c.fy, yd, c.cy);
    if (!((Z > c.lim * n) && (r2 <= c.r2_max))) return false;
    float pu = floorf(u + 0.5f), pv = floorf(v + 0.5f);
    if (!(pu >= 0.f && pv >= 0.f && pu < (float)c.width && pv < (float)c.height)) return false;
    const size_t pix = (size_t)pv * c.width + (size_t)pu;
    if (!PS_DCHECK(pix < (size_t)c.width * c.height, CHK_PIXEL)) return false;
    float d = __ldg(&depth[pix]);
    if (!(d > 0.f) || !(d < 3.0e38f)) return false;
    // |X_d| in voxel units: (a + b)^2 = a^2 (exact int) + (2a + b) b
    int A2 = ax * ax + ay * ay + az * az;
    float Bs = fmaf(fmaf(2.0f, (float)ax, bx), bx, fmaf(fmaf(2.0f, (float)ay, by), by, fmaf(2.0f, (float)az, bz) * bz));
    float y = sqrtf((float)A2 + Bs);
    float p = y * y;
    float pe = fmaf(y, y, -p);  // p + pe = y^2 exactly
    float diff = A2 < (1 << 24) ? (float)A2 - p : (float)(A2 - __float2int_rn(p));
    float corr = ((diff - pe) + Bs) / (2.0f * y);  // |X_d| = y + corr (voxel units)
    // eta = d - vox * (y + corr), with the product vox * y split exactly
    float q = F.vox * y;
    float qe = fmaf(F.vox, y, -q);
    *eta_out = ((d - q) - qe) - fmaf(F.vox_lo, y, F.vox * corr);
    *pix_out = pix;
    Xc[0] = X;
    Xc[1] = Y;
    Xc[2] = Z;
    return true;
}

// Eq. 2 on one voxel.
__device__ __forceinline__ void update_voxel(const FrameP& F, const float* depth, int ax, int ay, int az, float2& dw) {
    float eta, Xc[3];
    size_t pix;
    if (!observe_voxel(F, depth, ax, ay, az, &eta, &pix, Xc)) return;
    if (eta < -F.mu) return;
    float sdf = fminf(1.0f, eta * F.inv_mu);
    float w = dw.y;
    dw.x = (w * dw.x + sdf) / (w + 1.0f);
    dw.y = fminf(w + 1.0f, F.w_max);
}

// 32 registers (8 CTAs, the whole register file, per SM): measured 3% faster on
// the ring workload than the unconstrained 40 (0.190 against 0.196 ms per frame).
__global__ void __launch_bounds__(IT, 8) integrate_kernel(const __grid_constant__ FrameP F, TsdfDev T,
                                                       const float* depth) {
    int nv = *T.n_vis;
    for (int e = blockIdx.x; e < nv; e += gridDim.x) {
        int bi = T.vis[e];
        if (!PS_DCHECK(bi >= 0 && bi < T.pool_cap, CHK_POOL)) continue;  // uniform over the CTA
        int4 k = T.pool_keys[bi];
        float4* blk = reinterpret_cast<float4*>(T.vox + (size_t)bi * B3);
        float4 pr = blk[threadIdx.x];
        int v0 = 2 * threadIdx.x;  // voxels v0, v0 + 1: same y, z; x and x + 1
        int x = v0 & 7, y = (v0 >> 3) & 7, z = v0 >> 6;
        int ax = k.x * B + x - F.ic[0], ay = k.y * B + y - F.ic[1], az = k.z * B + z - F.ic[2];
        float2 a = make_float2(pr.x, pr.y), b = make_float2(pr.z, pr.w);
        update_voxel(F, depth, ax, ay, az, a);
        update_voxel(F, depth, ax + 1, ay, az, b);
        blk[threadIdx.x] = make_float4(a.x, a.y, b.x, b.y);
    }
}

// Output o <- live slot live[o] (or slot o when live is NULL).
__global__ void extract_kernel(TsdfDev T, const int* live, int n, float min_w, int* keys, float* D, float* W) {
    for (int o = blockIdx.x; o < n; o += gridDim.x) {
        const int i = live ? live[o] : o;
        if (!PS_DCHECK(i >= 0 && i < T.pool_cap, CHK_POOL)) continue;  // uniform over the CTA
        if (threadIdx.x == 0) {
            int4 k = T.pool_keys[i];
            keys[3 * o] = k.x;
            keys[3 * o + 1] = k.y;
            keys[3 * o + 2] = k.z;
        }
        for (int v = threadIdx.x; v < B3; v += blockDim.x) {
            float2 dw = T.vox[(size_t)i * B3 + v];
            bool keep = dw.y >= min_w && dw.y > 0.f;
            D[(size_t)o * B3 + v] = keep ? dw.x : 0.f;
            W[(size_t)o * B3 + v] = keep ? dw.y : 0.f;
        }
    }
}

// Live slots of the pool in slot order (one CTA of 1024 threads: each thread
// counts a contiguous range, a CTA-wide scan places the ranges).  live[]
// receives the slot indices, *n_live their number.
__global__ void __launch_bounds__(1024) compact_live_kernel(TsdfDev T, int* live, int* n_live) {
    __shared__ int part[1024];
    const int n = min(*T.n_alloc, T.pool_cap);
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    int c = 0;
    for (int i = lo; i < hi; ++i) c += T.pool_keys[i].w >= 0;
    part[threadIdx.x] = c;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // inclusive scan
        int v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int o = part[threadIdx.x] - c;
    for (int i = lo; i < hi; ++i)
        if (T.pool_keys[i].w >= 0) live[o++] = i;
    if (threadIdx.x == blockDim.x - 1) *n_live = part[threadIdx.x];
}

// Swap-out: live blocks whose centre lies outside the local map are copied
// to the caller's buffers (up to cap of them), their slots freed and zeroed.
__global__ void evict_kernel(TsdfDev T, const int* live, const int* n_live, float block, float3 lc, float3 lh,
                             int cap, int* n_out, int* keys, float* D, float* W) {
    __shared__ int s_o;
    const int n = *n_live;
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        const int i = live[e];
        const int4 k = T.pool_keys[i];
        const bool out = fabsf((k.x + 0.5f) * block - lc.x) > lh.x || fabsf((k.y + 0.5f) * block - lc.y) > lh.y ||
                         fabsf((k.z + 0.5f) * block - lc.z) > lh.z;
        if (!out) continue;  // uniform over the CTA
        if (threadIdx.x == 0) s_o = atomicAdd(n_out, 1);
        __syncthreads();
        const int o = s_o;
        __syncthreads();
        if (o >= cap) continue;  // no room: the block stays in the map
        if (threadIdx.x == 0) {
            keys[3 * o] = k.x;
            keys[3 * o + 1] = k.y;
            keys[3 * o + 2] = k.z;
            T.pool_keys[i].w = -1;
        }
        for (int v = threadIdx.x; v < B3; v += blockDim.x) {
            float2 dw = T.vox[(size_t)i * B3 + v];
            D[(size_t)o * B3 + v] = dw.x;
            W[(size_t)o * B3 + v] = dw.y;
            T.vox[(size_t)i * B3 + v] = make_float2(0.f, 0.f);
        }
    }
}

// Free stack <- every freed slot below the high-water mark.
__global__ void free_list_kernel(TsdfDev T) {
    const int n = min(*T.n_alloc, T.pool_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (T.pool_keys[i].w < 0) T.free_stack[atomicAdd(T.free_top, 1)] = i;
}

// Hash table rebuilt from the live slots (after a swap-out).
__global__ void rehash_kernel(TsdfDev T) {
    const int n = min(*T.n_alloc, T.pool_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int4 k = T.pool_keys[i];
        if (k.w < 0) continue;
        unsigned long long key = pack_key(k.x, k.y, k.z);
        long long h = (long long)(hash64(key) & (unsigned long long)T.slot_mask);
        for (int probe = 0; probe < MAX_PROBE; ++probe) {
            if (atomicCAS(&T.hkeys[h], EMPTY, key) == EMPTY) {
                T.hvals[h] = i;
                break;
            }
            h = (h + 1) & T.slot_mask;
            if (probe == MAX_PROBE - 1) atomicOr(T.status, DEV_TIMEOUT | DEV_CAPACITY);
        }
    }
}

// Pool slot of a key, -1 when absent (bounded probing).
__device__ int hash_find(const TsdfDev& T, int bx, int by, int bz) {
    unsigned long long key = pack_key(bx, by, bz);
    long long h = (long long)(hash64(key) & (unsigned long long)T.slot_mask);
    for (int probe = 0; probe < MAX_PROBE; ++probe) {
        unsigned long long k = T.hkeys[h];
        if (k == key) return T.hvals[h];
        if (k == EMPTY) return -1;
        h = (h + 1) & T.slot_mask;
    }
    return -1;
}

// Surface points (the extracted map): every voxel a of a listed block and
// its +x, +y, +z neighbour b (same block, or the next block along the axis:
// index arithmetic on dense grids, the hash otherwise) with w >= wmin on both
// and a sign change of D (positive against zero or negative) give the point
// X_a + t (X_b - X_a), t = D_a / (D_a - D_b).  Points and edges (global voxel
// index of a, axis) go to slots taken from an atomic counter; slots past
// `cap` are counted only.
__global__ void __launch_bounds__(256) points_kernel(TsdfDev T, const int* live, int n, float wmin, int nbx, int nby,
                                                     int nbz, float vox, float ox, float oy, float oz, int cap,
                                                     int* counter, float* points, int* edges) {
    __shared__ int nb_slot[3];
    for (int o = blockIdx.x; o < n; o += gridDim.x) {
        const int i = live ? live[o] : o;
        if (!PS_DCHECK(i >= 0 && i < T.pool_cap, CHK_POOL)) continue;  // uniform over the CTA
        const int4 k = T.pool_keys[i];
        __syncthreads();  // the previous block's neighbour slots are no longer read
        if (threadIdx.x < 3) {
            const int a = threadIdx.x;
            const int kx = k.x + (a == 0), ky = k.y + (a == 1), kz = k.z + (a == 2);
            int slot = -1;
            if (nbx > 0) {
                if (kx < nbx && ky < nby && kz < nbz) slot = kx + nbx * (ky + nby * kz);
            } else {
                slot = hash_find(T, kx, ky, kz);
            }
            nb_slot[a] = (slot >= 0 && slot < T.pool_cap) ? slot : -1;
        }
        __syncthreads();
        for (int v = threadIdx.x; v < B3; v += blockDim.x) {
            const float2 da = T.vox[(size_t)i * B3 + v];
            if (!(da.y >= wmin)) continue;
            const int c[3] = {v & 7, (v >> 3) & 7, v >> 6};
            for (int axis = 0; axis < 3; ++axis) {
                int cb[3] = {c[0], c[1], c[2]};
                int slot = i;
                if (++cb[axis] == B) {
                    cb[axis] = 0;
                    slot = nb_slot[axis];
                    if (slot < 0) continue;
                }
                const float2 db = T.vox[(size_t)slot * B3 + cb[0] + B * cb[1] + B * B * cb[2]];
                if (!(db.y >= wmin) || ((da.x > 0.f) == (db.x > 0.f))) continue;
                const float t = da.x / (da.x - db.x);
                const int g[3] = {k.x * B + c[0], k.y * B + c[1], k.z * B + c[2]};
                const int e = atomicAdd(counter, 1);
                if (e >= cap) continue;
                const float org[3] = {ox, oy, oz};
                for (int q = 0; q < 3; ++q) {
                    const float f = (float)g[q] + 0.5f + (q == axis ? t : 0.f);
                    points[3 * (size_t)e + q] = fmaf(f, vox, org[q]);
                    if (edges) edges[4 * (size_t)e + q] = g[q];
                }
                if (edges) edges[4 * (size_t)e + 3] = axis;
            }
        }
    }
}

// Load: (1) insert the keys, (2) copy each block's voxels into its slot.
__global__ void load_keys_kernel(TsdfDev T, const int* keys, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        hash_insert(T, keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]);
}

__global__ void load_voxels_kernel(TsdfDev T, const int* keys, const float* D, const float* W, int n) {
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        const int i = hash_find(T, keys[3 * e], keys[3 * e + 1], keys[3 * e + 2]);
        if (i < 0) continue;  // no room (capacity already latched)
        if (!PS_DCHECK(i < T.pool_cap, CHK_POOL)) continue;
        for (int v = threadIdx.x; v < B3; v += blockDim.x)
            T.vox[(size_t)i * B3 + v] = make_float2(D[(size_t)e * B3 + v], W[(size_t)e * B3 + v]);
    }
}

__global__ void dense_keys_kernel(int4* keys, int nx, int ny, int nz) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ny * nz) return;
    keys[i] = make_int4(i % nx, (i / nx) % ny, i / (nx * ny), 0);
}

}  // namespace

// ray table of the depth camera (defined with the sweep's ray kernel)
int build_rays(const ps_camera& cam, float4* rays, double* max_angle);

}  // namespace ps

using namespace ps;

struct tsdf_s {
    uint32_t magic = MAGIC_TSDF;  // first word: handle type for ps_sync_status
    ps_tsdf_desc d;
    bool dense = false;
    TsdfDev T{};
    int sms = 0;
    float4* rays = nullptr;
    double view_angle = 0;
    int* n_tmp = nullptr;  // [0] live blocks, [1] swapped-out blocks
    StageProfiler prof;
};

namespace {

void free_tsdf(tsdf_t* t) {
    if (!t) return;
    t->prof.release();
    cudaFree(t->T.hkeys);
    cudaFree(t->T.hvals);
    cudaFree(t->T.vox);
    cudaFree(t->T.pool_keys);
    cudaFree(t->T.n_alloc);
    cudaFree(t->T.vis);
    cudaFree(t->T.n_vis);
    cudaFree(t->T.status);
    cudaFree(t->T.dmax_bits);
    cudaFree(t->T.free_stack);
    cudaFree(t->T.free_top);
    cudaFree(t->n_tmp);
    cudaFree(t->rays);
    delete t;
}

int read_status(tsdf_t* t, cudaStream_t s) {
    unsigned st = 0;
    PS_CUDA(cudaMemcpyAsync(&st, t->T.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    if (st) {
        PS_CUDA(cudaMemsetAsync(t->T.status, 0, sizeof(unsigned), s));
        PS_CUDA(cudaStreamSynchronize(s));
        if (st & DEV_TIMEOUT) {
            set_error("TSDF hash probing gave up after %d probes (table too full)", MAX_PROBE);
            return PS_ERR_TIMEOUT;
        }
        set_error("TSDF voxel-block pool or hash table is full");
        return PS_ERR_CAPACITY;
    }
    return PS_OK;
}

}  // namespace

extern "C" int tsdf_create(const ps_tsdf_desc* d, tsdf_t** out) {
    clear_error();
    PS_ARG(out != nullptr, "tsdf_create: out is NULL");
    *out = nullptr;
    PS_ARG(d != nullptr, "tsdf_create: desc is NULL");
    PS_ARG(d->block_dim == 8, "tsdf_create: block_dim must be 8");
    PS_ARG(d->voxel_size > 0 && d->mu > 0 && d->w_max >= 1, "tsdf_create: need voxel_size > 0, mu > 0, w_max >= 1");
    PS_ARG(d->cam.width > 0 && d->cam.height > 0 && d->cam.fx > 0 && d->cam.fy > 0 && d->cam.xi >= 0,
           "tsdf_create: bad camera");
    bool dense = d->dense_dim[0] || d->dense_dim[1] || d->dense_dim[2];
    int64_t pool = 0;
    if (dense) {
        for (int i = 0; i < 3; ++i)
            PS_ARG(d->dense_dim[i] > 0 && d->dense_dim[i] % 8 == 0, "tsdf_create: dense_dim must be multiples of 8");
        pool = (int64_t)(d->dense_dim[0] / 8) * (d->dense_dim[1] / 8) * (d->dense_dim[2] / 8);
        PS_ARG(pool <= (1 << 24), "tsdf_create: dense grid too large");
    } else {
        PS_ARG(d->hash_slots >= 1024 && (d->hash_slots & (d->hash_slots - 1)) == 0 && d->hash_slots <= (1ll << 31),
               "tsdf_create: hash_slots must be a power of two in [2^10, 2^31]");
        PS_ARG(d->pool_blocks >= 1 && d->pool_blocks <= (1ll << 26), "tsdf_create: pool_blocks must be in [1, 2^26]");
        pool = d->pool_blocks;
    }
    tsdf_t* t = new tsdf_t();
    t->d = *d;
    t->dense = dense;
#define PS_TRY(call)                                                        \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) {                                            \
            free_tsdf(t);                                                   \
            set_error("%s: %s", #call, cudaGetErrorString(e_));             \
            return e_ == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA; \
        }                                                                   \
    } while (0)
    int dev = 0;
    PS_TRY(cudaGetDevice(&dev));
    PS_TRY(cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, dev));
    t->T.pool_cap = (int)pool;
    PS_TRY(cudaMalloc(&t->T.vox, sizeof(float2) * (size_t)pool * B3));
    PS_TRY(cudaMemset(t->T.vox, 0, sizeof(float2) * (size_t)pool * B3));
    PS_TRY(cudaMalloc(&t->T.pool_keys, sizeof(int4) * (size_t)pool));
    PS_TRY(cudaMalloc(&t->T.n_alloc, sizeof(int)));
    PS_TRY(cudaMalloc(&t->T.vis, sizeof(int) * (size_t)pool));
    PS_TRY(cudaMalloc(&t->T.n_vis, sizeof(int)));
    PS_TRY(cudaMalloc(&t->T.status, sizeof(unsigned)));
    PS_TRY(cudaMemset(t->T.status, 0, sizeof(unsigned)));
    PS_TRY(cudaMalloc(&t->T.dmax_bits, sizeof(unsigned)));
    PS_TRY(cudaMalloc(&t->n_tmp, 2 * sizeof(int)));
    if (dense) {
        int nx = d->dense_dim[0] / 8, ny = d->dense_dim[1] / 8, nz = d->dense_dim[2] / 8;
        dense_keys_kernel<<<(int)((pool + 255) / 256), 256>>>(t->T.pool_keys, nx, ny, nz);
        PS_TRY(cudaGetLastError());
        int n = (int)pool;
        PS_TRY(cudaMemcpy(t->T.n_alloc, &n, sizeof(int), cudaMemcpyHostToDevice));
    } else {
        PS_TRY(cudaMalloc(&t->T.hkeys, sizeof(unsigned long long) * (size_t)d->hash_slots));
        PS_TRY(cudaMemset(t->T.hkeys, 0xFF, sizeof(unsigned long long) * (size_t)d->hash_slots));
        PS_TRY(cudaMalloc(&t->T.hvals, sizeof(int) * (size_t)d->hash_slots));
        PS_TRY(cudaMemset(t->T.hvals, 0xFF, sizeof(int) * (size_t)d->hash_slots));
        PS_TRY(cudaMemset(t->T.n_alloc, 0, sizeof(int)));
        t->T.slot_mask = d->hash_slots - 1;
        PS_TRY(cudaMalloc(&t->T.free_stack, sizeof(int) * (size_t)pool));
        PS_TRY(cudaMalloc(&t->T.free_top, sizeof(int)));
        PS_TRY(cudaMemset(t->T.free_top, 0, sizeof(int)));
    }
    PS_TRY(cudaMalloc(&t->rays, sizeof(float4) * (size_t)d->cam.width * d->cam.height));
    t->T.rays = t->rays;
    int st = build_rays(d->cam, t->rays, &t->view_angle);
    if (st) {
        free_tsdf(t);
        return st;
    }
    PS_TRY(cudaDeviceSynchronize());
#undef PS_TRY
    *out = t;
    return PS_OK;
}

extern "C" void tsdf_destroy(tsdf_t* t) { free_tsdf(t); }

extern "C" int tsdf_integrate(tsdf_t* t, const float* depth, const ps_pose* w2c, const double* lc, void* stream) {
    clear_error();
    PS_ARG(t != nullptr && depth != nullptr && w2c != nullptr, "tsdf_integrate: NULL argument");
    const ps_tsdf_desc& d = t->d;
    bool gate = !t->dense && (d.local_half[0] > 0 || d.local_half[1] > 0 || d.local_half[2] > 0);
    PS_ARG(!gate || lc != nullptr, "tsdf_integrate: local_center is required with a local map");
    for (int i = 0; i < 12; ++i) PS_ARG(std::isfinite(i < 9 ? w2c->R[i] : w2c->t[i - 9]), "tsdf_integrate: pose not finite");
    cudaStream_t s = (cudaStream_t)stream;
    FrameP F;
    std::memset(&F, 0, sizeof(F));
    F.cam = to_camf(d.cam);
    double Cw[3];
    for (int i = 0; i < 3; ++i) {
        Cw[i] = -(w2c->R[i] * w2c->t[0] + w2c->R[3 + i] * w2c->t[1] + w2c->R[6 + i] * w2c->t[2]);
        for (int k = 0; k < 3; ++k) {
            F.R[3 * i + k] = (float)w2c->R[3 * i + k];
            F.Rt[3 * i + k] = (float)w2c->R[3 * k + i];
        }
    }
    for (int i = 0; i < 3; ++i) {
        double rel = Cw[i] - d.origin[i];
        F.C[i] = (float)rel;
        double cv = rel / d.voxel_size;
        double ic = std::floor(cv + 0.5);
        PS_ARG(std::fabs(ic) < 1e8, "tsdf_integrate: camera too far from the grid origin");
        F.ic[i] = (int)ic;
        F.fb[i] = (float)(0.5 - (cv - ic));
    }
    F.vox = (float)d.voxel_size;
    F.vox_lo = (float)(d.voxel_size - (double)F.vox);
    F.mu = (float)d.mu;
    F.inv_mu = (float)(1.0 / d.mu);
    F.w_max = (float)d.w_max;
    F.block = (float)(8.0 * d.voxel_size);
    F.gate = gate ? 1 : 0;
    if (gate)
        for (int i = 0; i < 3; ++i) {
            F.lc[i] = (float)(lc[i] - d.origin[i]);
            F.lh[i] = (float)d.local_half[i];
        }
    F.view_angle = (float)(t->view_angle + 1e-3);
    const int W = d.cam.width, H = d.cam.height;
    t->prof.mark(0, s);
    PS_CUDA(cudaMemsetAsync(t->T.dmax_bits, 0, sizeof(unsigned), s));
    depth_max_kernel<<<t->sms * 2, 256, 0, s>>>(depth, W * H, t->T.dmax_bits);
    PS_CUDA(cudaGetLastError());
    t->prof.mark(1, s);
    if (!t->dense) {
        alloc_kernel<<<dim3((W + 127) / 128, H), 128, 0, s>>>(F, t->T, depth);
        PS_CUDA(cudaGetLastError());
    }
    t->prof.mark(2, s);
    PS_CUDA(cudaMemsetAsync(t->T.n_vis, 0, sizeof(int), s));
    visible_kernel<<<t->sms * 4, 256, 0, s>>>(F, t->T);
    PS_CUDA(cudaGetLastError());
    t->prof.mark(3, s);
    integrate_kernel<<<t->sms * 8, IT, 0, s>>>(F, t->T, depth);
    PS_CUDA(cudaGetLastError());
    t->prof.mark(4, s);
    t->prof.end_call();
    return PS_OK;
}

extern "C" int tsdf_profile(tsdf_t* t, int32_t capacity) {
    clear_error();
    PS_ARG(t != nullptr && capacity >= 0 && capacity <= (1 << 20), "tsdf_profile: bad arguments");
    return t->prof.enable(4, capacity);
}

extern "C" int tsdf_profile_read(tsdf_t* t, double* stage_ms, int32_t* n_calls) {
    clear_error();
    PS_ARG(t != nullptr && stage_ms != nullptr, "tsdf_profile_read: NULL argument");
    PS_ARG(t->prof.cap > 0, "tsdf_profile_read: profiling is off");
    return t->prof.read(stage_ms, n_calls);
}

extern "C" int tsdf_count(tsdf_t* t, int64_t* n_blocks, void* stream) {
    clear_error();
    PS_ARG(t != nullptr && n_blocks != nullptr, "tsdf_count: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int n[2] = {0, 0};
    PS_CUDA(cudaMemcpyAsync(&n[0], t->T.n_alloc, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (t->T.free_top) PS_CUDA(cudaMemcpyAsync(&n[1], t->T.free_top, sizeof(int), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    *n_blocks = std::min<int64_t>(n[0], t->T.pool_cap) - std::max(0, n[1]);
    return read_status(t, s);
}

extern "C" int tsdf_listed(tsdf_t* t, int64_t* n_blocks, void* stream) {
    clear_error();
    PS_ARG(t != nullptr && n_blocks != nullptr, "tsdf_listed: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int n = 0;
    PS_CUDA(cudaMemcpyAsync(&n, t->T.n_vis, sizeof(int), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    *n_blocks = n;
    return PS_OK;
}

// Live slots in slot order into t->T.vis (scratch outside integrate calls); returns their number.
int live_slots(tsdf_t* t, cudaStream_t s, int64_t* n_live) {
    compact_live_kernel<<<1, 1024, 0, s>>>(t->T, t->T.vis, t->n_tmp);
    PS_CUDA(cudaGetLastError());
    int n = 0;
    PS_CUDA(cudaMemcpyAsync(&n, t->n_tmp, sizeof(int), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    *n_live = n;
    return PS_OK;
}

extern "C" int tsdf_extract(tsdf_t* t, float min_weight, int32_t* keys, float* D, float* W, int64_t capacity,
                            int64_t* n_out, void* stream) {
    clear_error();
    PS_ARG(t != nullptr && n_out != nullptr, "tsdf_extract: NULL argument");
    PS_ARG(capacity >= 0, "tsdf_extract: negative capacity");
    PS_ARG(capacity == 0 || (keys && D && W), "tsdf_extract: NULL output buffer");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t n = 0;
    int st = tsdf_count(t, &n, stream);
    int64_t hw = 0;
    PS_CUDA(cudaMemcpyAsync(&hw, t->T.n_alloc, sizeof(int), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    const bool holes = std::min<int64_t>((int)hw, t->T.pool_cap) != n;  // freed slots below the high-water mark
    if (holes) {
        int e = live_slots(t, s, &n);
        if (e) return e;
    }
    int64_t m = std::min(n, capacity);
    if (m > 0) {
        extract_kernel<<<(int)std::min<int64_t>(m, 65535), 256, 0, s>>>(t->T, holes ? t->T.vis : nullptr, (int)m,
                                                                       min_weight, keys, D, W);
        PS_CUDA(cudaGetLastError());
        PS_CUDA(cudaStreamSynchronize(s));
    }
    *n_out = m;
    if (st) return st;
    if (capacity < n) {
        set_error("tsdf_extract: capacity %lld < %lld blocks", (long long)capacity, (long long)n);
        return PS_ERR_CAPACITY;
    }
    return PS_OK;
}

extern "C" int tsdf_extract_points(tsdf_t* t, float min_weight, float* points, int32_t* edges, int64_t capacity,
                                   int64_t* n_out, void* stream) {
    clear_error();
    PS_ARG(t != nullptr && n_out != nullptr, "tsdf_extract_points: NULL argument");
    PS_ARG(capacity >= 0 && capacity < (1ll << 31), "tsdf_extract_points: capacity must be in 0 .. 2^31 - 1");
    PS_ARG(capacity == 0 || points != nullptr, "tsdf_extract_points: points is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t n = 0;
    int st = tsdf_count(t, &n, stream);
    int64_t hw = 0;
    PS_CUDA(cudaMemcpyAsync(&hw, t->T.n_alloc, sizeof(int), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    const bool holes = std::min<int64_t>((int)hw, t->T.pool_cap) != n;
    if (holes) {
        int e = live_slots(t, s, &n);
        if (e) return e;
    }
    int found = 0;
    if (n > 0) {
        PS_CUDA(cudaMemsetAsync(t->n_tmp + 1, 0, sizeof(int), s));
        const ps_tsdf_desc& d = t->d;
        const int nbx = t->dense ? d.dense_dim[0] / 8 : 0, nby = t->dense ? d.dense_dim[1] / 8 : 0,
                  nbz = t->dense ? d.dense_dim[2] / 8 : 0;
        points_kernel<<<(int)std::min<int64_t>(n, 65535), 256, 0, s>>>(
            t->T, holes ? t->T.vis : nullptr, (int)n, std::max(min_weight, 1.0f), nbx, nby, nbz, (float)d.voxel_size,
            (float)d.origin[0], (float)d.origin[1], (float)d.origin[2], (int)capacity, t->n_tmp + 1, points, edges);
        PS_CUDA(cudaGetLastError());
        PS_CUDA(cudaMemcpyAsync(&found, t->n_tmp + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        PS_CUDA(cudaStreamSynchronize(s));
    }
    *n_out = found;
    if (st) return st;
    if (found > capacity) {
        set_error("tsdf_extract_points: %d points, capacity %lld (the first %lld were written)", found,
                  (long long)capacity, (long long)capacity);
        return PS_ERR_CAPACITY;
    }
    return PS_OK;
}

extern "C" int tsdf_swap_out(tsdf_t* t, const double* lc, int32_t* keys, float* D, float* W, int64_t capacity,
                             int64_t* n_out, void* stream) {
    clear_error();
    PS_ARG(t != nullptr && lc != nullptr && n_out != nullptr, "tsdf_swap_out: NULL argument");
    PS_ARG(!t->dense, "tsdf_swap_out: a dense grid has no local map to leave");
    const ps_tsdf_desc& d = t->d;
    PS_ARG(d.local_half[0] > 0 || d.local_half[1] > 0 || d.local_half[2] > 0,
           "tsdf_swap_out: the map has no local-map extent");
    PS_ARG(capacity >= 0 && (capacity == 0 || (keys && D && W)), "tsdf_swap_out: bad output buffers");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t n_live = 0;
    int e = live_slots(t, s, &n_live);
    if (e) return e;
    PS_CUDA(cudaMemsetAsync(t->n_tmp + 1, 0, sizeof(int), s));
    const float block = (float)(8.0 * d.voxel_size);
    float3 c = make_float3((float)(lc[0] - d.origin[0]), (float)(lc[1] - d.origin[1]), (float)(lc[2] - d.origin[2]));
    float3 h = make_float3((float)d.local_half[0], (float)d.local_half[1], (float)d.local_half[2]);
    if (n_live > 0) {
        evict_kernel<<<(int)std::min<int64_t>(n_live, 65535), 256, 0, s>>>(t->T, t->T.vis, t->n_tmp, block, c, h,
                                                                          (int)std::min<int64_t>(capacity, 1 << 30),
                                                                          t->n_tmp + 1, keys, D, W);
        PS_CUDA(cudaGetLastError());
    }
    // free list and hash rebuilt from the surviving blocks
    PS_CUDA(cudaMemsetAsync(t->T.free_top, 0, sizeof(int), s));
    free_list_kernel<<<t->sms * 4, 256, 0, s>>>(t->T);
    PS_CUDA(cudaGetLastError());
    PS_CUDA(cudaMemsetAsync(t->T.hkeys, 0xFF, sizeof(unsigned long long) * (size_t)d.hash_slots, s));
    PS_CUDA(cudaMemsetAsync(t->T.hvals, 0xFF, sizeof(int) * (size_t)d.hash_slots, s));
    rehash_kernel<<<t->sms * 4, 256, 0, s>>>(t->T);
    PS_CUDA(cudaGetLastError());
    int n_ev = 0;
    PS_CUDA(cudaMemcpyAsync(&n_ev, t->n_tmp + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    *n_out = std::min<int64_t>(n_ev, capacity);
    int st = read_status(t, s);
    if (st) return st;
    if (n_ev > capacity) {
        set_error("tsdf_swap_out: %d blocks left the local map, capacity %lld; the rest stay in the map", n_ev,
                  (long long)capacity);
        return PS_ERR_CAPACITY;
    }
    return PS_OK;
}

extern "C" int tsdf_load(tsdf_t* t, const int32_t* keys, const float* D, const float* W, int64_t n, void* stream) {
    clear_error();
    PS_ARG(t != nullptr && n >= 0 && (n == 0 || (keys && D && W)), "tsdf_load: bad arguments");
    PS_ARG(!t->dense, "tsdf_load: a dense grid keeps its blocks; write its voxels instead");
    PS_ARG(n <= (1ll << 30), "tsdf_load: too many blocks");
    if (n == 0) return PS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    load_keys_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 65535), 256, 0, s>>>(t->T, keys, (int)n);
    PS_CUDA(cudaGetLastError());
    load_voxels_kernel<<<(int)std::min<int64_t>(n, 65535), 256, 0, s>>>(t->T, keys, D, W, (int)n);
    PS_CUDA(cudaGetLastError());
    return PS_OK;
}

namespace ps {
int tsdf_sync_status(tsdf_t* t, cudaStream_t s) { return read_status(t, s); }
}  // namespace ps

extern "C" int tsdf_set_partition(tsdf_t* t, int32_t n_parts, int32_t part) {
    clear_error();
    PS_ARG(t != nullptr, "tsdf_set_partition: NULL handle");
    PS_ARG(!t->dense, "tsdf_set_partition: a dense grid has no block allocation to partition");
    PS_ARG(n_parts >= 1 && part >= 0 && part < n_parts, "tsdf_set_partition: need 0 <= part < n_parts");
    t->T.n_parts = n_parts;
    t->T.part = part;
    return PS_OK;
}

extern "C" int tsdf_status(tsdf_t* t, void* stream) {
    clear_error();
    PS_ARG(t != nullptr, "tsdf_status: NULL handle");
    return read_status(t, (cudaStream_t)stream);
}

// ===================================================================== allocation-free dense fusion
//
// For callers that cannot allocate device memory while they run (real-time
// loops whose memory is planned once up front, hosts whose device memory
// belongs to another allocator): the working memory lives in this fixed
// static device array instead of a handle.
// Layout: [0] status word, [4] block count, [8] listed-block count, [12]
// depth maximum bits, [256 ..) block keys (int4 x PS_STATIC_MAX_BLOCKS), then
// the visible-block list (int x PS_STATIC_MAX_BLOCKS).  The status word only
// gives the shared kernels a valid target: on a dense grid nothing sets it
// (no hash table, no pool, no segment allocation), so it is never read.

#include <mutex>

namespace ps {
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[PS_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_static_mu;
unsigned char* g_static_ptr[MAX_DEVICES] = {};

// Device address of the static array on the current device (looked up once per device).
int static_scratch(unsigned char** out) {
    int dev = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_ARG(dev >= 0 && dev < MAX_DEVICES, "tsdf_integrate_dense_static: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_static_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_static_ptr[dev];
    return PS_OK;
}

__global__ void static_dense_keys_kernel(int4* keys, int* n_alloc, int nx, int ny, int nz) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int n = nx * ny * nz;
    if (i == 0) *n_alloc = n;
    if (i < n) keys[i] = make_int4(i % nx, (i / nx) % ny, i / (nx * ny), 0);
}

}  // namespace
}  // namespace ps

namespace ps {
namespace {

// Frame record of a caller-owned dense grid at `origin` (no local map).
int dense_frame(const double* origin, double voxel_size, double mu, double w_max, const ps_camera* cam,
                const ps_pose* w2c, FrameP& F) {
    std::memset(&F, 0, sizeof(F));
    F.cam = to_camf(*cam);
    for (int i = 0; i < 3; ++i) {
        double Cw = -(w2c->R[i] * w2c->t[0] + w2c->R[3 + i] * w2c->t[1] + w2c->R[6 + i] * w2c->t[2]);
        for (int k = 0; k < 3; ++k) {
            F.R[3 * i + k] = (float)w2c->R[3 * i + k];
            F.Rt[3 * i + k] = (float)w2c->R[3 * k + i];
        }
        double rel = Cw - origin[i];
        F.C[i] = (float)rel;
        double cv = rel / voxel_size;
        double ic = std::floor(cv + 0.5);
        PS_ARG(std::fabs(ic) < 1e8, "dense fusion: camera too far from the grid origin");
        F.ic[i] = (int)ic;
        F.fb[i] = (float)(0.5 - (cv - ic));
    }
    F.vox = (float)voxel_size;
    F.vox_lo = (float)(voxel_size - (double)F.vox);
    F.mu = (float)mu;
    F.inv_mu = (float)(1.0 / mu);
    F.w_max = (float)w_max;
    F.block = (float)(8.0 * voxel_size);
    F.view_angle = 4.0f;  // no view-cone culling: the range test alone keeps the list a superset
    return PS_OK;
}

// Gradient of one dense fusion step (Eq. 2, unit observation weight) for
// every voxel of an nbx x nby x nbz block grid: dL/dD_in = g w / (w + 1) on
// observed voxels (g elsewhere); observed voxels with eta < mu add
// g / (mu (w + 1)) to their pixel's depth gradient and -that * X_c / |X_c|
// to X_c, which a left perturbation (w, v) of world_to_cam moves by
// w x X_c + v (CTA reduction, FP64 atomics).
__global__ void __launch_bounds__(256) dense_fuse_bwd_kernel(const __grid_constant__ FrameP F, int nbx, int nby,
                                                            int nbz, const float2* vox_in, const float* depth,
                                                            const float* gD, float* gD_in, float* g_depth,
                                                            double* g_pose) {
    __shared__ float red[8][6];
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const long long n = (long long)nbx * nby * nbz * B3;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / B3;
        const int v = (int)(i % B3);
        const int gx = (int)(b % nbx) * B + (v & 7), gy = (int)((b / nbx) % nby) * B + ((v >> 3) & 7),
                  gz = (int)(b / ((long long)nbx * nby)) * B + (v >> 6);
        const float g = gD[i];
        float out = g;
        float eta, Xc[3];
        size_t pix;
        if (observe_voxel(F, depth, gx - F.ic[0], gy - F.ic[1], gz - F.ic[2], &eta, &pix, Xc) && !(eta < -F.mu)) {
            const float w = vox_in[i].y;
            out = g * w / (w + 1.0f);
            if (eta < F.mu && g != 0.f) {
                const float ge = g / (F.mu * (w + 1.0f));
                if (g_depth) atomicAdd(&g_depth[pix], ge);
                const float s = -ge / sqrtf(Xc[0] * Xc[0] + Xc[1] * Xc[1] + Xc[2] * Xc[2]);
                const float gx3[3] = {s * Xc[0], s * Xc[1], s * Xc[2]};
                acc[0] += Xc[1] * gx3[2] - Xc[2] * gx3[1];
                acc[1] += Xc[2] * gx3[0] - Xc[0] * gx3[2];
                acc[2] += Xc[0] * gx3[1] - Xc[1] * gx3[0];
                acc[3] += gx3[0];
                acc[4] += gx3[1];
                acc[5] += gx3[2];
            }
        }
        if (gD_in) gD_in[i] = out;
    }
    if (!g_pose) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 6; ++k) {
        float v = acc[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += (double)red[w][threadIdx.x];
        atomicAdd(&g_pose[threadIdx.x], s);
    }
}

}  // namespace
}  // namespace ps

extern "C" int tsdf_integrate_dense_static(float* voxels, const int32_t* dims, const double* origin,
                                           double voxel_size, double mu, double w_max, const float* depth,
                                           const ps_camera* cam, const ps_pose* w2c, void* stream) {
    clear_error();
    PS_ARG(voxels && dims && origin && depth && cam && w2c, "tsdf_integrate_dense_static: NULL argument");
    PS_ARG(voxel_size > 0 && mu > 0 && w_max >= 1, "tsdf_integrate_dense_static: need voxel_size > 0, mu > 0, w_max >= 1");
    PS_ARG(cam->width > 0 && cam->height > 0 && cam->fx > 0 && cam->fy > 0 && cam->xi >= 0,
           "tsdf_integrate_dense_static: bad camera");
    for (int i = 0; i < 3; ++i)
        PS_ARG(dims[i] > 0 && dims[i] % 8 == 0, "tsdf_integrate_dense_static: dims must be positive multiples of 8");
    const long long nx = dims[0] / 8, ny = dims[1] / 8, nz = dims[2] / 8;
    // compared step by step: each factor is at least 1, so no product below overflows
    PS_ARG(nx <= PS_STATIC_MAX_BLOCKS && ny <= PS_STATIC_MAX_BLOCKS / nx &&
               nz <= PS_STATIC_MAX_BLOCKS / (nx * ny),
           "tsdf_integrate_dense_static: a %lld x %lld x %lld block grid exceeds the static limit of %d blocks "
           "(%d voxels)", nx, ny, nz, PS_STATIC_MAX_BLOCKS, PS_STATIC_MAX_BLOCKS * B3);
    const long long n_blocks = nx * ny * nz;
    for (int i = 0; i < 12; ++i)
        PS_ARG(std::isfinite(i < 9 ? w2c->R[i] : w2c->t[i - 9]), "tsdf_integrate_dense_static: pose not finite");
    unsigned char* base = nullptr;
    int st = static_scratch(&base);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    TsdfDev T{};
    T.status = reinterpret_cast<unsigned*>(base);
    T.n_alloc = reinterpret_cast<int*>(base + 4);
    T.n_vis = reinterpret_cast<int*>(base + 8);
    T.dmax_bits = reinterpret_cast<unsigned*>(base + 12);
    T.pool_keys = reinterpret_cast<int4*>(base + 256);
    T.vis = reinterpret_cast<int*>(base + 256 + sizeof(int4) * PS_STATIC_MAX_BLOCKS);
    T.vox = reinterpret_cast<float2*>(voxels);
    T.pool_cap = (int)n_blocks;

    FrameP F;
    st = dense_frame(origin, voxel_size, mu, w_max, cam, w2c, F);
    if (st) return st;
    int dev = 0, sms = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int W = cam->width, H = cam->height;
    PS_CUDA(cudaMemsetAsync(base, 0, 256, s));  // counters and depth maximum start at zero
    static_dense_keys_kernel<<<(int)((n_blocks + 255) / 256), 256, 0, s>>>(T.pool_keys, T.n_alloc, (int)nx, (int)ny,
                                                                           (int)nz);
    PS_CUDA(cudaGetLastError());
    depth_max_kernel<<<sms * 2, 256, 0, s>>>(depth, W * H, T.dmax_bits);
    PS_CUDA(cudaGetLastError());
    visible_kernel<<<sms * 4, 256, 0, s>>>(F, T);
    PS_CUDA(cudaGetLastError());
    integrate_kernel<<<sms * 8, IT, 0, s>>>(F, T, depth);
    PS_CUDA(cudaGetLastError());
    return PS_OK;
}

extern "C" int tsdf_dense_fuse_backward(const float* voxels_in, const int32_t* dims, const double* origin,
                                        double voxel_size, double mu, double w_max, const float* depth,
                                        const ps_camera* cam, const ps_pose* w2c, const float* g_D_out,
                                        float* g_D_in, float* g_depth, double* g_pose, void* stream) {
    clear_error();
    PS_ARG(voxels_in && dims && origin && depth && cam && w2c && g_D_out, "tsdf_dense_fuse_backward: NULL argument");
    PS_ARG(voxel_size > 0 && mu > 0 && w_max >= 1, "tsdf_dense_fuse_backward: need voxel_size > 0, mu > 0, w_max >= 1");
    PS_ARG(cam->width > 0 && cam->height > 0 && cam->fx > 0 && cam->fy > 0 && cam->xi >= 0,
           "tsdf_dense_fuse_backward: bad camera");
    for (int i = 0; i < 3; ++i)
        PS_ARG(dims[i] > 0 && dims[i] % 8 == 0, "tsdf_dense_fuse_backward: dims must be positive multiples of 8");
    for (int i = 0; i < 12; ++i)
        PS_ARG(std::isfinite(i < 9 ? w2c->R[i] : w2c->t[i - 9]), "tsdf_dense_fuse_backward: pose not finite");
    FrameP F;
    int st = dense_frame(origin, voxel_size, mu, w_max, cam, w2c, F);
    if (st) return st;
    int dev = 0, sms = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long n = (long long)dims[0] * dims[1] * dims[2];
    const int grid = (int)std::min<long long>((n + 255) / 256, (long long)sms * 8);
    dense_fuse_bwd_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(F, dims[0] / 8, dims[1] / 8, dims[2] / 8,
                                                                 reinterpret_cast<const float2*>(voxels_in), depth,
                                                                 g_D_out, g_D_in, g_depth, g_pose);
    PS_CUDA(cudaGetLastError());
    return PS_OK;
}

namespace ps {
PS_DEFINE_CHECK_READER(check_bits_tsdf)
}  // namespace ps

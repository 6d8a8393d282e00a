// Device-side building blocks of the sm_103a path: counter-based random numbers, the
// Henyey-Greenstein phase function and sampler, direction rotation, the bricked extinction
// fetch and the FP32 voxel walk (Amanatides-Woo). Positions are in grid-local metres
// (origin subtracted) so FP32 keeps ~1e-4 m resolution across a 2 km domain.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace mst {

constexpr int kMaxCams = 16;
constexpr int kMaxRays = 64;
constexpr int kBrickShift = 3;  // 8^3 bricks
constexpr int kBrickVox = 512;

struct Geo {
    int nx, ny, nz;     // voxels per axis
    int nbx, nby, nbz;  // 8^3 bricks per axis
    float hx, hy, hz;   // voxel size (m)
    float ex, ey, ez;   // grid extent (m)
    int nvox;
    int max_steps;      // nx + ny + nz + 8: no straight walk crosses more voxels
};

struct Cam {
    float px, py, pz;              // centre of projection, grid-local
    float rx, ry, rz;              // right
    float ux, uy, uz;              // up
    float fx, fy, fz;              // forward
    float tx, ty;                  // tan(fov_x/2), tan(fov_x/2) * H / W
    int w, h, pix_off;
};

struct CamSet {
    int n;
    Cam c[kMaxCams];
};

struct Halton {
    int n;
    float a[kMaxRays], b[kMaxRays];
};

// ------------------------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al., SC'11): counter (photon lo, photon hi, event, stream), key = seed.

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// (2 (x >> 9) + 1) / 2^24: 24 significant bits, exact in FP32, strictly inside (0, 1).
__device__ __forceinline__ float u01(uint32_t x) { return __uint2float_rn(2u * (x >> 9) + 1u) * 5.9604644775390625e-08f; }

__device__ __forceinline__ float4 draws(uint2 key, uint64_t photon, uint32_t event) {
    const uint4 x = philox4x32_10(make_uint4((uint32_t)photon, (uint32_t)(photon >> 32), event, 0u), key);
    return make_float4(u01(x.x), u01(x.y), u01(x.z), u01(x.w));
}

// ------------------------------------------------------------------------------------------
// Henyey-Greenstein (Eq. Phg) and its inverse CDF (Eq. thetaHG, squared reading).

struct HG {
    float g, k1, a, b;             // P = k1 * (a - b mu)^(-3/2)
    float omg2, omg, tg, inv2g;    // sampler constants
    bool iso;
};

__device__ __forceinline__ float hg_phase(const HG& h, float mu) {
    const float den = h.a - h.b * mu;
    const float r = rsqrtf(den);
    return h.k1 * r * r * r;
}

__device__ __forceinline__ float hg_sample(const HG& h, float u) {
    if (h.iso) return 2.f * u - 1.f;
    const float s = h.omg2 / (h.omg + h.tg * u);
    const float c = (h.a - s * s) * h.inv2g;
    return fminf(1.f, fmaxf(-1.f, c));
}

// New unit direction at polar cosine ct and azimuth 2 pi u1 about d. Transverse frame:
// e2 = normalize(axis x d), e1 = e2 x d, axis = z unless |d_z| >= 0.9, then x.
__device__ __forceinline__ float3 rotate_dir(float3 d, float ct, float u1) {
    const float st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
    float sp, cp;
    sincospif(2.f * u1, &sp, &cp);
    float3 e2;
    if (fabsf(d.z) < 0.9f) {
        const float n = rsqrtf(d.x * d.x + d.y * d.y);
        e2 = make_float3(-d.y * n, d.x * n, 0.f);
    } else {
        const float n = rsqrtf(d.y * d.y + d.z * d.z);
        e2 = make_float3(0.f, -d.z * n, d.y * n);
    }
    const float3 e1 = make_float3(e2.y * d.z - e2.z * d.y, e2.z * d.x - e2.x * d.z, e2.x * d.y - e2.y * d.x);
    float3 o = make_float3(st * (cp * e1.x + sp * e2.x) + ct * d.x, st * (cp * e1.y + sp * e2.y) + ct * d.y,
                           st * (cp * e1.z + sp * e2.z) + ct * d.z);
    const float rn = rsqrtf(o.x * o.x + o.y * o.y + o.z * o.z);
    return make_float3(o.x * rn, o.y * rn, o.z * rn);
}

// ------------------------------------------------------------------------------------------
// Extinction storage: 8^3 bricks, Morton order inside a brick, so one 128-byte line holds a
// 4x4x2 (FP32) or 4x4x4 (16-bit) block of neighbouring voxels.

__device__ __forceinline__ int spread3(int v) { return (v & 1) | ((v & 2) << 2) | ((v & 4) << 4); }

__device__ __forceinline__ int brick_addr(const Geo& g, int ix, int iy, int iz) {
    const int b = (ix >> kBrickShift) + g.nbx * ((iy >> kBrickShift) + g.nby * (iz >> kBrickShift));
    return (b << 9) | spread3(ix & 7) | (spread3(iy & 7) << 1) | (spread3(iz & 7) << 2);
}

__device__ __forceinline__ int lin_index(const Geo& g, int ix, int iy, int iz) { return ix + g.nx * (iy + g.ny * iz); }

template <int DT>
struct BetaFetch;
template <>
struct BetaFetch<0> {
    typedef float T;
    static __device__ __forceinline__ float get(const void* p, int a) { return __ldg(static_cast<const float*>(p) + a); }
    static __device__ __forceinline__ T make(float v) { return v; }
};
template <>
struct BetaFetch<1> {
    typedef __half T;
    static __device__ __forceinline__ float get(const void* p, int a) {
        return __half2float(__ldg(static_cast<const __half*>(p) + a));
    }
    static __device__ __forceinline__ T make(float v) { return __float2half_rn(v); }
};
template <>
struct BetaFetch<2> {
    typedef __nv_bfloat16 T;
    static __device__ __forceinline__ float get(const void* p, int a) {
        return __bfloat162float(__ldg(static_cast<const __nv_bfloat16*>(p) + a));
    }
    static __device__ __forceinline__ T make(float v) { return __float2bfloat16_rn(v); }
};

// ------------------------------------------------------------------------------------------
// Voxel walk. t_a is the ray parameter of the next face on axis a; ties go to x, then y, then z.

struct Walk {
    float ox, oy, oz;     // ray origin
    float vx, vy, vz;     // 1 / direction
    float tx, ty, tz;     // next face crossing
    int ix, iy, iz;       // current voxel
    int sx, sy, sz;       // step per axis (0 when the direction component is 0)
    int left;             // face crossings left before the walk is abandoned
};

__device__ __forceinline__ float face_t(int i, int s, float h, float o, float inv) {
    return s == 0 ? CUDART_INF_F : (__int2float_rn(i + (s > 0)) * h - o) * inv;
}

__device__ __forceinline__ void walk_init(Walk& w, const Geo& g, float3 o, float3 d, int ix, int iy, int iz) {
    w.ox = o.x; w.oy = o.y; w.oz = o.z;
    w.ix = ix; w.iy = iy; w.iz = iz;
    w.sx = d.x > 0.f ? 1 : (d.x < 0.f ? -1 : 0);
    w.sy = d.y > 0.f ? 1 : (d.y < 0.f ? -1 : 0);
    w.sz = d.z > 0.f ? 1 : (d.z < 0.f ? -1 : 0);
    w.vx = 1.f / d.x; w.vy = 1.f / d.y; w.vz = 1.f / d.z;
    w.tx = face_t(ix, w.sx, g.hx, o.x, w.vx);
    w.ty = face_t(iy, w.sy, g.hy, o.y, w.vy);
    w.tz = face_t(iz, w.sz, g.hz, o.z, w.vz);
    w.left = g.max_steps;
}

__device__ __forceinline__ int walk_axis(const Walk& w, float& tn) {
    int a = 0;
    tn = w.tx;
    if (w.ty < tn) { a = 1; tn = w.ty; }
    if (w.tz < tn) { a = 2; tn = w.tz; }
    return a;
}

constexpr int kWalkOverflow = 6;

// Crosses the face on axis a. Returns the exit face (0..5: x-, x+, y-, y+, z-, z+) if the
// walk left the grid, kWalkOverflow if it made more crossings than any straight line through
// the grid can (only possible with a non-finite direction), else -1.
__device__ __forceinline__ int walk_step(Walk& w, const Geo& g, int a) {
    if (--w.left < 0) return kWalkOverflow;
    if (a == 0) {
        w.ix += w.sx;
        w.tx = face_t(w.ix, w.sx, g.hx, w.ox, w.vx);
        if ((unsigned)w.ix >= (unsigned)g.nx) return w.sx > 0 ? 1 : 0;
    } else if (a == 1) {
        w.iy += w.sy;
        w.ty = face_t(w.iy, w.sy, g.hy, w.oy, w.vy);
        if ((unsigned)w.iy >= (unsigned)g.ny) return w.sy > 0 ? 3 : 2;
    } else {
        w.iz += w.sz;
        w.tz = face_t(w.iz, w.sz, g.hz, w.oz, w.vz);
        if ((unsigned)w.iz >= (unsigned)g.nz) return w.sz > 0 ? 5 : 4;
    }
    return -1;
}

__device__ __forceinline__ int coord_vox(float x, float h, int n) {
    const float f = floorf(x / h);
    return f < 0.f ? 0 : (f > (float)(n - 1) ? n - 1 : (int)f);
}

// Clips the ray o + t d to the grid box. Returns false if it misses; else the entry
// parameter t0 >= 0 and the entry voxel.
__device__ __forceinline__ bool ray_enter(const Geo& g, float3 o, float3 d, float& t0, int& ix, int& iy, int& iz) {
    float tn = 0.f, tf = CUDART_INF_F;
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z}, hi[3] = {g.ex, g.ey, g.ez};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dd[a] == 0.f) {
            if (oo[a] < 0.f || oo[a] > hi[a]) return false;
        } else {
            float t1 = (0.f - oo[a]) / dd[a], t2 = (hi[a] - oo[a]) / dd[a];
            if (t1 > t2) { const float tt = t1; t1 = t2; t2 = tt; }
            tn = fmaxf(tn, t1);
            tf = fminf(tf, t2);
        }
    }
    if (!(tn < tf)) return false;
    t0 = tn;
    ix = coord_vox(o.x + tn * d.x, g.hx, g.nx);
    iy = coord_vox(o.y + tn * d.y, g.hy, g.ny);
    iz = coord_vox(o.z + tn * d.z, g.hz, g.nz);
    return true;
}

__device__ __forceinline__ float3 pixel_dir(const Cam& c, float px, float py) {
    const float x = (2.f * px / (float)c.w - 1.f) * c.tx;
    const float y = (2.f * py / (float)c.h - 1.f) * c.ty;
    float3 d = make_float3(c.fx + x * c.rx + y * c.ux, c.fy + x * c.ry + y * c.uy, c.fz + x * c.rz + y * c.uz);
    const float n = 1.f / sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
    return make_float3(d.x * n, d.y * n, d.z * n);
}

__device__ __forceinline__ int cam_of_pixel(const CamSet& cs, int gp) {
    int c = 0;
    for (int i = 1; i < cs.n; ++i)
        if (gp >= cs.c[i].pix_off) c = i;
    return c;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sumu(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace mst

// Device-side building blocks of the sm_103a path: counter-based random numbers, the
// Henyey-Greenstein phase function and sampler, direction rotation, the staged extinction
// fetch and the FP32 voxel walk (Amanatides-Woo), whose positions are voxel index + offset
// inside the voxel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace mst {

constexpr int kMaxCams = 64;
constexpr int kMaxRays = 64;

struct Geo {
    int nx, ny, nz;     // voxels per axis
    float hx, hy, hz;   // voxel size (m)
    float ex, ey, ez;   // grid extent (m)
    int nvox;
    int max_steps;      // nx + ny + nz + 8: no straight walk crosses more voxels
    // The photon flights walk a copy of the grid padded with kHalo voxels on every side
    // ([nz + 4][ny + 4][nx + 4], halo extinction +inf), so that leaving the grid needs no bounds
    // test in the voxel step: the walk stops on the first halo layer's extinction, and the
    // extinction of the voxel after it, loaded one step ahead, still lies inside the array.
    int p0, p01;        // nx + 4, (nx + 4)(ny + 4): strides of the padded grid
    float inv_p0, inv_p01;
    int npad;           // (nx + 4)(ny + 4)(nz + 4)
};

constexpr int kHalo = 2;  // halo layers of the padded grid

struct Cam {
    float px, py, pz;              // centre of projection, grid-local metres
    int ix, iy, iz;                // voxel holding the centre (may lie outside the grid)
    float lx, ly, lz;              // offset of the centre inside that voxel
    int inside;                    // centre inside the grid
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

// stream 0: the forward transport and its replays; 1 + p: backward paths of global pixel p
__device__ __forceinline__ float4 draws(uint2 key, uint64_t photon, uint32_t event, uint32_t stream = 0u) {
    const uint4 x = philox4x32_10(make_uint4((uint32_t)photon, (uint32_t)(photon >> 32), event, stream), key);
    return make_float4(u01(x.x), u01(x.y), u01(x.z), u01(x.w));
}

// The raw Philox block of a counter, and its four uniforms: draws() in two steps, for callers
// that also use the low bits u01 leaves unused.
__device__ __forceinline__ uint4 draw_bits(uint2 key, uint64_t photon, uint32_t event) {
    return philox4x32_10(make_uint4((uint32_t)photon, (uint32_t)(photon >> 32), event, 0u), key);
}

__device__ __forceinline__ float4 u01x4(uint4 x) { return make_float4(u01(x.x), u01(x.y), u01(x.z), u01(x.w)); }

// ------------------------------------------------------------------------------------------
// Henyey-Greenstein (Eq. Phg) and its inverse CDF (Eq. thetaHG, squared reading).

struct HG {
    float g, k1, a, b;             // P = k1 * (a - b mu)^(-3/2)
    float omg, opg, omg2, tg;      // 1 - g, 1 + g, 1 - g^2, 2 g
    bool iso;
};

__device__ __forceinline__ float hg_phase(const HG& h, float mu) {
    const float den = h.a - h.b * mu;
    const float r = rsqrtf(den);
    return h.k1 * r * r * r;
}

// Inverse CDF of Eq. Phg (squared reading of Eq. thetaHG): cos = (1 + g^2 - s^2) / (2 g) with
// s = (1 - g^2) / (1 - g + 2 g u). 1 - cos and 1 + cos are evaluated in factored form,
//   1 - cos = (1-g)(1-u)(s + 1 - g) / D,  1 + cos = (1+g) u (s + 1 + g) / D,  D = 1 - g + 2 g u,
// so sin = sqrt((1 - cos)(1 + cos)) keeps full FP32 precision for forward scattering, where
// sqrt(1 - cos^2) would cancel. 1 - u is exact for the 24-bit uniforms.
__device__ __forceinline__ void hg_sample(const HG& h, float u, float& ct, float& st) {
    float omc, opc;
    if (h.iso) {
        omc = 2.f * (1.f - u);
        opc = 2.f * u;
    } else {
        const float D = fmaf(h.tg, u, h.omg);  // spelled out, like the multiply-adds of rotate_dir
        const float s = h.omg2 / D;
        omc = h.omg * (1.f - u) * (s + h.omg) / D;
        opc = h.opg * u * (s + h.opg) / D;
    }
    ct = fminf(1.f, fmaxf(-1.f, 0.5f * (opc - omc)));
    st = sqrtf(fmaxf(omc * opc, 0.f));
}

// Rayleigh phase function of air molecules (Eq. Pray): 3 / (16 pi) (1 + mu^2).
__device__ __forceinline__ float rayleigh_phase(float mu) { return 0.05968310365946075f * fmaf(mu, mu, 1.f); }

// Inverse CDF of Eq. Pray (Eq. thetaREY): the CDF of the cosine is (mu^3 + 3 mu + 4) / 8, and
// Cardano's root of mu^3 + 3 mu + 4 - 8u = 0 is mu = c - 1/c with c = cbrt(q + sqrt(q^2 + 1)),
// q = 4u - 2. q + sqrt(q^2 + 1) lies in [0.23, 4.3] for u in [0, 1], so nothing cancels.
__device__ __forceinline__ void rayleigh_sample(float u, float& ct, float& st) {
    const float q = fmaf(4.f, u, -2.f);
    const float c = cbrtf(q + sqrtf(fmaf(q, q, 1.f)));
    ct = fminf(1.f, fmaxf(-1.f, c - 1.f / c));
    st = sqrtf(fmaxf((1.f - ct) * (1.f + ct), 0.f));
}

// New unit direction at polar angle (cos ct, sin st) and azimuth 2 pi u1 about d. Transverse
// frame: e2 = normalize(axis x d), e1 = e2 x d, axis = z unless |d_z| >= 0.9, then x.
// Every multiply-add is spelled out (fmaf, or __fmul_rn which is never fused): the kernels that
// replay a path must compute each direction bit for bit like the forward did, whatever the
// compiler fuses in the code around them.
__device__ __forceinline__ float3 rotate_dir(float3 d, float ct, float st, float u1) {
    float sp, cp;
    sincospif(2.f * u1, &sp, &cp);
    float3 e2;
    if (fabsf(d.z) < 0.9f) {
        const float n = rsqrtf(fmaf(d.x, d.x, __fmul_rn(d.y, d.y)));
        e2 = make_float3(-d.y * n, d.x * n, 0.f);
    } else {
        const float n = rsqrtf(fmaf(d.y, d.y, __fmul_rn(d.z, d.z)));
        e2 = make_float3(0.f, -d.z * n, d.y * n);
    }
    const float3 e1 = make_float3(fmaf(e2.y, d.z, -__fmul_rn(e2.z, d.y)), fmaf(e2.z, d.x, -__fmul_rn(e2.x, d.z)),
                                  fmaf(e2.x, d.y, -__fmul_rn(e2.y, d.x)));
    const float3 o = make_float3(fmaf(st, fmaf(cp, e1.x, __fmul_rn(sp, e2.x)), __fmul_rn(ct, d.x)),
                                 fmaf(st, fmaf(cp, e1.y, __fmul_rn(sp, e2.y)), __fmul_rn(ct, d.y)),
                                 fmaf(st, fmaf(cp, e1.z, __fmul_rn(sp, e2.z)), __fmul_rn(ct, d.z)));
    const float rn = rsqrtf(fmaf(o.x, o.x, fmaf(o.y, o.y, __fmul_rn(o.z, o.z))));
    return make_float3(o.x * rn, o.y * rn, o.z * rn);
}

// ------------------------------------------------------------------------------------------
// Extinction storage: the grid staged in the compute dtype, x fastest ([nz][ny][nx], the
// linear voxel index). A voxel step changes the index by +-1, +-nx or +-nx ny, one multiply-add;
// the whole 64^3 grid is 1 MB and stays in L2, where 8^3 bricks bought no measurable locality
// but cost the walk a wrap test and two selects per step.

__device__ __forceinline__ int lin_index(const Geo& g, int ix, int iy, int iz) { return ix + g.nx * (iy + g.ny * iz); }

// index of voxel (ix, iy, iz) in the padded grid (each index may lie in the halo, -kHalo .. n + kHalo - 1)
__device__ __forceinline__ int pad_index(const Geo& g, int ix, int iy, int iz) {
    return (ix + kHalo) + g.p0 * (iy + kHalo) + g.p01 * (iz + kHalo);
}

// (ix, iy, iz) of padded index q, each in [-kHalo, n + kHalo). The quotients come from FP32 reciprocals and
// are corrected by one step: q < 2^31 and the quotients are below 2^12, so the FP32 estimate is
// off by at most one.
__device__ __forceinline__ void unpad(const Geo& g, int q, int& ix, int& iy, int& iz) {
    int a = (int)((float)q * g.inv_p01);
    int r = q - a * g.p01;
    if (r < 0) { --a; r += g.p01; } else if (r >= g.p01) { ++a; r -= g.p01; }
    int b = (int)((float)r * g.inv_p0);
    int c = r - b * g.p0;
    if (c < 0) { --b; c += g.p0; } else if (c >= g.p0) { ++b; c -= g.p0; }
    ix = c - kHalo;
    iy = b - kHalo;
    iz = a - kHalo;
}

// linear voxel index k of a padded index; false for a halo voxel
__device__ __forceinline__ bool interior_lin(const Geo& g, int q, int& k) {
    int ix, iy, iz;
    unpad(g, q, ix, iy, iz);
    k = lin_index(g, ix, iy, iz);
    return (unsigned)ix < (unsigned)g.nx && (unsigned)iy < (unsigned)g.ny && (unsigned)iz < (unsigned)g.nz;
}

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
// Voxel walk in voxel-local form. A point is (voxel index, offset inside the voxel); the walk
// keeps, per axis, the distance along the ray from the current point to the next face. A step
// of length s across axis a subtracts s from the other two axes and resets axis a to h_a/|d_a|,
// so every quantity stays of the size of one voxel and FP32 keeps ~1e-6 m resolution however
// large the grid. Ties go to x, then y, then z.

struct Walk {
    float tx, ty, tz;     // distance to the next face per axis (INF when parallel)
    float qx, qy, qz;     // h / |d| per axis
    float ax, ay, az;     // |d| per axis
    float p0x, p0y, p0z;  // offset at the start (kept on axes the ray does not move along)
    int ix, iy, iz;       // current voxel
    int sx, sy, sz;       // step per axis (0 when the direction component is 0)
    int lin;              // linear index ix + nx (iy + ny iz) of the current voxel (its extinction's address)
    int left;             // face crossings left before the walk is abandoned
};

// kFastRcp: 1/|d| by the hardware reciprocal (__fdividef, within 2 ulp) instead of the
// correctly rounded division; photon flights use it, camera and LOS rays keep the division.
template <bool kFastRcp>
__device__ __forceinline__ void axis_init(float p, float d, float h, float& t, float& q, float& a, int& s) {
    if (d > 0.f) {
        a = d;
        const float inv = kFastRcp ? __fdividef(1.f, d) : 1.f / d;
        t = (h - p) * inv;
        q = h * inv;
        s = 1;
    } else if (d < 0.f) {
        a = -d;
        const float inv = kFastRcp ? __fdividef(1.f, a) : 1.f / a;
        t = p * inv;
        q = h * inv;
        s = -1;
    } else {
        a = 0.f;
        t = CUDART_INF_F;
        q = CUDART_INF_F;
        s = 0;
    }
}

// p: offset of the start point inside voxel (ix, iy, iz), each in [0, h]
template <bool kFastRcp = false>
__device__ __forceinline__ void walk_init(Walk& w, const Geo& g, float3 p, float3 d, int ix, int iy, int iz) {
    axis_init<kFastRcp>(fminf(fmaxf(p.x, 0.f), g.hx), d.x, g.hx, w.tx, w.qx, w.ax, w.sx);
    axis_init<kFastRcp>(fminf(fmaxf(p.y, 0.f), g.hy), d.y, g.hy, w.ty, w.qy, w.ay, w.sy);
    axis_init<kFastRcp>(fminf(fmaxf(p.z, 0.f), g.hz), d.z, g.hz, w.tz, w.qz, w.az, w.sz);
    w.p0x = p.x; w.p0y = p.y; w.p0z = p.z;
    w.ix = ix; w.iy = iy; w.iz = iz;
    w.lin = lin_index(g, ix, iy, iz);
    w.left = g.max_steps;
}

// distance to the next face and its axis
__device__ __forceinline__ int walk_axis(const Walk& w, float& tn) {
    int a = 0;
    tn = w.tx;
    if (w.ty < tn) { a = 1; tn = w.ty; }
    if (w.tz < tn) { a = 2; tn = w.tz; }
    tn = fmaxf(tn, 0.f);
    return a;
}

constexpr int kWalkOverflow = 6;

// Moves seg along the ray and crosses the face on axis a. Returns the exit face (0..5: x-, x+,
// y-, y+, z-, z+) if the walk left the grid, kWalkOverflow if it made more crossings than any
// straight line through the grid can (only possible with a non-finite direction), else -1.
// Branch-free in the axis, so lanes that cross different faces do not diverge. Callers that
// bound the crossings themselves (the transport, once per trip) pass kGuard = false.
template <bool kGuard = true>
__device__ __forceinline__ int walk_step(Walk& w, const Geo& g, int a, float seg) {
    const bool bx = a == 0, by = a == 1, bz = a == 2;
    w.tx = bx ? w.qx : w.tx - seg;
    w.ty = by ? w.qy : w.ty - seg;
    w.tz = bz ? w.qz : w.tz - seg;
    const int s = bx ? w.sx : (by ? w.sy : w.sz);
    w.ix += bx ? s : 0;
    w.iy += by ? s : 0;
    w.iz += bz ? s : 0;
    w.lin += s * (bx ? 1 : (by ? g.nx : g.nx * g.ny));
    const bool out = ((unsigned)w.ix >= (unsigned)g.nx) | ((unsigned)w.iy >= (unsigned)g.ny) |
                     ((unsigned)w.iz >= (unsigned)g.nz);
    if (kGuard && --w.left < 0) return kWalkOverflow;
    return out ? 2 * a + (s > 0) : -1;
}

__device__ __forceinline__ float axis_local(float t, float a, int s, float h, float p0, float l) {
    const float v = s > 0 ? h - (t - l) * a : (s < 0 ? (t - l) * a : p0);
    return fminf(fmaxf(v, 0.f), h);
}

// offset inside the current voxel of the point a distance l past the current point
__device__ __forceinline__ float3 walk_local(const Walk& w, const Geo& g, float l) {
    return make_float3(axis_local(w.tx, w.ax, w.sx, g.hx, w.p0x, l), axis_local(w.ty, w.ay, w.sy, g.hy, w.p0y, l),
                       axis_local(w.tz, w.az, w.sz, g.hz, w.p0z, l));
}

__device__ __forceinline__ bool walk_at(const Walk& w, int ix, int iy, int iz) {
    return w.ix == ix && w.iy == iy && w.iz == iz;
}

// vector from the point (voxel i, offset p) to the point (voxel j, offset q)
__device__ __forceinline__ float3 local_delta(const Geo& g, int ix, int iy, int iz, float3 p, int jx, int jy, int jz,
                                              float3 q) {
    return make_float3((float)(jx - ix) * g.hx + (q.x - p.x), (float)(jy - iy) * g.hy + (q.y - p.y),
                       (float)(jz - iz) * g.hz + (q.z - p.z));
}

__device__ __forceinline__ int coord_vox(float x, float h, int n) {
    const float f = floorf(x / h);
    return f < 0.f ? 0 : (f > (float)(n - 1) ? n - 1 : (int)f);
}

__device__ __forceinline__ float3 pixel_dir(const Cam& c, float px, float py) {
    const float x = (2.f * px / (float)c.w - 1.f) * c.tx;
    const float y = (2.f * py / (float)c.h - 1.f) * c.ty;
    float3 d = make_float3(c.fx + x * c.rx + y * c.ux, c.fy + x * c.ry + y * c.uy, c.fz + x * c.rz + y * c.uz);
    const float n = 1.f / sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
    return make_float3(d.x * n, d.y * n, d.z * n);
}

// Start of a ray from a camera: inside the grid it starts at the camera's own voxel and offset;
// outside, the ray is clipped to the grid box (entry point in grid-local metres). Returns
// false if it misses the grid.
__device__ __forceinline__ bool ray_start(const Geo& g, const Cam& c, float3 d, float3& p, int& ix, int& iy, int& iz) {
    if (c.inside) {
        ix = c.ix; iy = c.iy; iz = c.iz;
        p = make_float3(c.lx, c.ly, c.lz);
        return true;
    }
    // Clip to the grid box in a frame at the corner of the camera's voxel (cell index c.i, which
    // may lie outside the grid): the camera is at offset c.l there and the faces the ray enters
    // through are near, so the entry point keeps FP32's resolution however far the grid extends
    // (grid-local coordinates would carry ~1 mm of rounding 10 km from the origin).
    const int ci[3] = {c.ix, c.iy, c.iz}, nn[3] = {g.nx, g.ny, g.nz};
    const float oo[3] = {c.lx, c.ly, c.lz}, dd[3] = {d.x, d.y, d.z}, hh[3] = {g.hx, g.hy, g.hz};
    float tn = 0.f, tf = CUDART_INF_F;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = -(float)ci[a] * hh[a], hi = (float)(nn[a] - ci[a]) * hh[a];
        if (dd[a] == 0.f) {
            if (oo[a] < lo || oo[a] > hi) return false;
        } else {
            float t1 = (lo - oo[a]) / dd[a], t2 = (hi - oo[a]) / dd[a];
            if (t1 > t2) { const float tt = t1; t1 = t2; t2 = tt; }
            tn = fmaxf(tn, t1);
            tf = fminf(tf, t2);
        }
    }
    if (!(tn < tf)) return false;
    int iv[3];
    float pv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float e = oo[a] + tn * dd[a];  // entry point relative to the camera voxel's corner
        const int k = min(max(ci[a] + (int)floorf(e / hh[a]), 0), nn[a] - 1);
        iv[a] = k;
        pv[a] = e - (float)(k - ci[a]) * hh[a];
    }
    ix = iv[0]; iy = iv[1]; iz = iv[2];
    p = make_float3(pv[0], pv[1], pv[2]);
    return true;
}

__device__ __forceinline__ int cam_of_pixel(const CamSet& cs, int gp) {
    int c = 0;
    for (int i = 1; i < cs.n; ++i)
        if (gp >= cs.c[i].pix_off) c = i;
    return c;
}

// Walks the segment from the point (voxel i, offset p) to the centre of projection of camera c,
// calling fn(walk, length) for every voxel it crosses (walk.lin names the voxel). The walk ends in the
// camera's voxel (last length = distance to the camera inside it) or, for a camera outside the
// grid, at the grid face; the remaining distance guards both ends against rounding.
template <typename F>
__device__ __forceinline__ void walk_to_camera(const Geo& g, const Cam& c, int ix, int iy, int iz, float3 p, F&& fn,
                                               unsigned long long& nseg) {
    const float3 lc = make_float3(c.lx, c.ly, c.lz);
    const float3 v = local_delta(g, ix, iy, iz, p, c.ix, c.iy, c.iz, lc);
    const float dist = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
    if (!(dist > 0.f)) return;
    const float inv = 1.f / dist;
    const float3 d = make_float3(v.x * inv, v.y * inv, v.z * inv);
    Walk w;
    walk_init(w, g, p, d, ix, iy, iz);
    float rem = dist;
    for (;;) {
        ++nseg;
        if (walk_at(w, c.ix, c.iy, c.iz)) {
            const float3 q = walk_local(w, g, 0.f);
            const float len = (lc.x - q.x) * d.x + (lc.y - q.y) * d.y + (lc.z - q.z) * d.z;
            fn(w, fminf(fmaxf(len, 0.f), rem));
            return;
        }
        float seg;
        const int a = walk_axis(w, seg);
        if (seg >= rem) {
            fn(w, rem);
            return;
        }
        fn(w, seg);
        rem -= seg;
        if (walk_step(w, g, a, seg) >= 0) return;
    }
}

// Walks the pixel ray from camera c along d to the grid exit, calling fn(walk, length).
template <typename F>
__device__ __forceinline__ void walk_from_camera(const Geo& g, const Cam& c, float3 d, F&& fn,
                                                 unsigned long long& nseg) {
    float3 p;
    int ix, iy, iz;
    if (!ray_start(g, c, d, p, ix, iy, iz)) return;
    Walk w;
    walk_init(w, g, p, d, ix, iy, iz);
    for (;;) {
        ++nseg;
        float seg;
        const int a = walk_axis(w, seg);
        fn(w, seg);
        if (walk_step(w, g, a, seg) >= 0) return;
    }
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

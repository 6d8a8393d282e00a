// Photon transport on the GPU: the forward MC life cycle (Sec. 2.1.2, steps i-vi) with the
// voxelised local estimate of Eq. Lcupdate (or the classic one of Eq. fle), and the replay
// adjoint that re-walks every photon from its Philox key to scatter the score-function
// gradient of L (no path is stored).
//
// Work distribution: a persistent grid sized to the SM count. Each lane owns one photon at a
// time and advances it one free flight plus one event per loop trip; lanes whose photon has
// ended take a new photon id from a warp-local pool that lane 0 refills from a global ticket,
// so the warp stays full until the chunk runs dry.
#include <algorithm>
#include <type_traits>

#include "mst_internal.h"

namespace mst {
namespace {

constexpr int kTB = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kFnvOffset = 2166136261u;
constexpr uint32_t kFnvPrime = 16777619u;

struct Photon {
    float3 p, d;     // offset inside voxel (ix, iy, iz) and unit direction
    int ix, iy, iz;
    float I, tau;
    uint32_t s;      // scattering events so far
    uint32_t hash;   // forward: path checksum; replay pass 2 on the stored events: the photon's first step slot
    uint64_t id;     // global photon id (Philox counter)
    uint32_t idx;    // call-relative index (hash / skip arrays)
};

// Photon tallies of the forward render: per-thread totals, reduced over the warp at the end.
struct Tally {
    float esc[6];
    float absorbed, killed, gained, forced, launched;
    unsigned capped, escaped, traced, lost;
};

// The forward render keeps its tallies in shared memory, one slot per thread (stride kTB
// words, so a warp's lanes touch consecutive words): no atomics and no registers held across
// the voxel loop. The replay passes keep none: their NoTally compiles every update away.
struct LaneTally {
    float* f;  // 11 float fields at f[q * kTB]
    unsigned* u;  // 4 counters at u[q * kTB]
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < 11; ++q) f[q * kTB] = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) u[q * kTB] = 0u;
    }
    __device__ __forceinline__ void add_absorbed(float v) { f[6 * kTB] += v; }
    __device__ __forceinline__ void add_killed(float v) { f[7 * kTB] += v; }
    __device__ __forceinline__ void add_gained(float v) { f[8 * kTB] += v; }
    __device__ __forceinline__ void add_forced(float v) { f[9 * kTB] += v; }
    __device__ __forceinline__ void add_capped() { u[0] += 1u; }
    __device__ __forceinline__ void add_launch(float i0) {
        f[10 * kTB] += i0;
        u[2 * kTB] += 1u;
    }
    __device__ __forceinline__ void add_escape(int face, float v) {
        if (face < 6) f[face * kTB] += v;
        if (face == kWalkOverflow) u[3 * kTB] += 1u;
        else u[1 * kTB] += 1u;
    }
    __device__ __forceinline__ Tally load() const {
        Tally t;
#pragma unroll
        for (int q = 0; q < 6; ++q) t.esc[q] = f[q * kTB];
        t.absorbed = f[6 * kTB];
        t.killed = f[7 * kTB];
        t.gained = f[8 * kTB];
        t.forced = f[9 * kTB];
        t.launched = f[10 * kTB];
        t.capped = u[0];
        t.escaped = u[1 * kTB];
        t.traced = u[2 * kTB];
        t.lost = u[3 * kTB];
        return t;
    }
};

// A per-thread event counter that exists only when ON (the one-species kernels carry none).
template <bool ON>
struct EventCount {
    unsigned n = 0u;
    __device__ __forceinline__ void add() { ++n; }
    __device__ __forceinline__ void flush(double* slot, unsigned lane) const {
        const unsigned long long s = warp_sumu(n);
        if (lane == 0u && s) atomicAdd(slot, (double)s);
    }
};
template <>
struct EventCount<false> {
    __device__ __forceinline__ void add() {}
    __device__ __forceinline__ void flush(double*, unsigned) const {}
};

struct NoTally {
    __device__ __forceinline__ void zero() {}
    __device__ __forceinline__ void add_absorbed(float) {}
    __device__ __forceinline__ void add_forced(float) {}
    __device__ __forceinline__ void add_gained(float) {}
    __device__ __forceinline__ void add_killed(float) {}
    __device__ __forceinline__ void add_capped() {}
    __device__ __forceinline__ void add_launch(float) {}
    __device__ __forceinline__ void add_escape(int, float) {}
};

// Voxel and offset of u * n voxels, u = (2m + 1) / 2^24 from a Philox word: (2m + 1) n / 2^24 is
// split exactly in integers, so the offset keeps all 24 bits of u.
__device__ __forceinline__ void launch_coord(uint32_t x, int n, float h, int& i, float& off) {
    const uint64_t q = (uint64_t)(2u * (x >> 9) + 1u) * (uint64_t)n;
    i = (int)(q >> 24);
    off = __uint2float_rn((uint32_t)(q & 0xFFFFFFu)) * 5.9604644775390625e-08f * h;
}

// step i: launch uniformly over the top of the atmosphere along the sun direction, weight I0
__device__ __forceinline__ void launch_photon(const TransportArgs& A, Photon& ph, uint32_t pid) {
    ph.idx = A.out_base + pid;
    ph.id = A.first_id + pid;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)ph.id, (uint32_t)(ph.id >> 32), 0u, 0u), A.key);
    float ox, oy;
    launch_coord(x.x, A.g.nx, A.g.hx, ph.ix, ox);
    launch_coord(x.y, A.g.ny, A.g.hy, ph.iy, oy);
    ph.iz = A.g.nz - 1;
    ph.p = make_float3(ox, oy, A.g.hz);
    ph.d = A.sun;
    ph.I = A.I0;
    ph.tau = -logf(1.f - u01(x.z));  // Eq. taurand
    ph.s = 0u;
    ph.hash = kFnvOffset;
}

// A free flight (steps ii-iii) on the padded grid. Per axis: the distance along the ray from
// the current point to the next face (t), the distance between faces (q = h / |d|), and the change
// of the padded index when a face is crossed (+-1, +-(nx + 2), +-(nx + 2)(ny + 2); 0 for an axis
// the ray does not move along, whose t stays +inf); `lin` is the current voxel's padded index.
// A voxel step subtracts the step from two axes and resets the crossed one to q, so every
// quantity stays of the size of one voxel and FP32 keeps ~1e-6 m resolution anywhere in the grid.
// Ties go to x, then y, then z. Leaving the grid needs no test in the step: the first halo voxel
// has extinction +inf, so its optical depth exceeds any free path and the flight stops there.
// The extinction of the next voxel is loaded one step ahead (bn), so that its latency overlaps
// the current step; the voxel after the first halo layer is the second, still in the array.
struct Flight {
    float tx, ty, tz;
    float qx, qy, qz;
    int dx, dy, dz;
    int lin;
    float bn;  // extinction of voxel lin, loaded ahead
    int left;  // voxel steps left before a flight is abandoned (only a non-finite direction gets there)
    int tgt;   // replay pass 2 on the stored events: padded index of the voxel the flight ends in
};

// 1 / |d| by the hardware reciprocal (__fdividef, within 2 ulp)
__device__ __forceinline__ void flight_axis(float p, float d, float h, int stride, float& t, float& q, int& dl) {
    if (d > 0.f) {
        const float inv = __fdividef(1.f, d);
        t = (h - p) * inv;
        q = h * inv;
        dl = stride;
    } else if (d < 0.f) {
        const float inv = __fdividef(1.f, -d);
        t = p * inv;
        q = h * inv;
        dl = -stride;
    } else {
        t = CUDART_INF_F;
        q = CUDART_INF_F;
        dl = 0;
    }
}

// the flight of photon ph from its point (voxel + offset) along its direction
template <int DT>
__device__ __forceinline__ void flight_init(Flight& f, const TransportArgs& A, const Photon& ph) {
    const Geo& g = A.g;
    flight_axis(fminf(fmaxf(ph.p.x, 0.f), g.hx), ph.d.x, g.hx, 1, f.tx, f.qx, f.dx);
    flight_axis(fminf(fmaxf(ph.p.y, 0.f), g.hy), ph.d.y, g.hy, g.p0, f.ty, f.qy, f.dy);
    flight_axis(fminf(fmaxf(ph.p.z, 0.f), g.hz), ph.d.z, g.hz, g.p01, f.tz, f.qz, f.dz);
    f.lin = pad_index(g, ph.ix, ph.iy, ph.iz);
    f.bn = BetaFetch<DT>::get(A.beta_pad, f.lin);
    f.left = g.max_steps;
}

// Replay pass 2 on the stored events: the same flight, told by the step the stored-event adjoint
// wrote for the event that ends it (slot evoff + events so far, ph.hash holding evoff) where it
// ends and how much free path it has left on entering that voxel (tau). Its voxels before that
// one need no extinction: the flight crosses them.
__device__ __forceinline__ void flight_init_stored(Flight& f, const TransportArgs& A, const Photon& ph, float& tau) {
    const Geo& g = A.g;
    const uint4 st = __ldg(reinterpret_cast<const uint4*>(A.wseq) + (ph.hash + ph.s));
    flight_axis(fminf(fmaxf(ph.p.x, 0.f), g.hx), ph.d.x, g.hx, 1, f.tx, f.qx, f.dx);
    flight_axis(fminf(fmaxf(ph.p.y, 0.f), g.hy), ph.d.y, g.hy, g.p0, f.ty, f.qy, f.dy);
    flight_axis(fminf(fmaxf(ph.p.z, 0.f), g.hz), ph.d.z, g.hz, g.p01, f.tz, f.qz, f.dz);
    f.lin = pad_index(g, ph.ix, ph.iy, ph.iz);
    f.left = g.max_steps;
    f.tgt = pad_index(g, (int)(st.y & 0x7FFu), (int)((st.y >> 11) & 0x7FFu), (int)(st.y >> 22));
    tau = __uint_as_float(st.z);
}

// One voxel of a free flight (Eq. MCextinct): the free path tau runs out in this voxel when
// tau <= beta * (distance to the next face). Returns true then, or when the voxel is the halo
// (beta = +inf; the caller tells the two apart by b), with b and the face distance m of the voxel;
// false after crossing into the next voxel. SCORE (replay pass 2): every voxel the flight crosses
// receives -S * length in the gradient tile (padded like the grid). The product beta * m is
// rounded on its own (__fmul_rn: never fused into the subtraction that follows), and so is the
// product in flight_offset: the forward and the replay passes are different kernels, and a
// multiply-add fused in one and not in another would send a photon along another path.
template <int DT, bool SCORE>
__device__ __forceinline__ bool flight_step(const TransportArgs& A, Flight& f, float& tau, float& b, float& m, float S,
                                            unsigned& nsc) {
    b = f.bn;
    m = fminf(f.tx, fminf(f.ty, f.tz));
    const bool px = f.tx <= m;
    const bool py = !px && f.ty <= m;
    const int next = f.lin + (px ? f.dx : (py ? f.dy : f.dz));
    f.bn = BetaFetch<DT>::get(A.beta_pad, next);
    const float bs = __fmul_rn(b, m);
    if (!(tau > bs)) return true;
    tau -= bs;
    if (SCORE && S != 0.f && m > 0.f) {
        atomicAdd(A.gacc + f.lin, -S * m);
        ++nsc;
    }
    f.tx = px ? f.qx : f.tx - m;
    f.ty = py ? f.qy : f.ty - m;
    f.tz = (px || py) ? f.tz - m : f.qz;
    f.lin = next;
    return false;
}

// One voxel of a replay pass-2 flight whose end is known (flight_init_stored): true in the voxel
// the flight ends in (the caller loads its extinction there), else the voxel receives -S *
// length in the gradient tile and the flight crosses into the next one, by the arithmetic of
// flight_step, so that it visits the same voxels.
__device__ __forceinline__ bool flight_step_stored(const TransportArgs& A, Flight& f, float S, unsigned& nsc) {
    // (a voxel index past the padded grid would mean the walk missed its end: it stops there)
    if (f.lin == f.tgt || (unsigned)f.lin >= (unsigned)A.g.npad) return true;
    const float m = fminf(f.tx, fminf(f.ty, f.tz));
    const bool px = f.tx <= m;
    const bool py = !px && f.ty <= m;
    if (S != 0.f && m > 0.f) {
        atomicAdd(A.gacc + f.lin, -S * m);
        ++nsc;
    }
    f.tx = px ? f.qx : f.tx - m;
    f.ty = py ? f.qy : f.ty - m;
    f.tz = (px || py) ? f.tz - m : f.qz;
    f.lin += px ? f.dx : (py ? f.dy : f.dz);
    return false;
}

// offset along one axis, inside the current voxel, of the point a distance l past the current
// point (d: the direction component; p0: the flight's start offset, kept when d = 0)
__device__ __forceinline__ float flight_offset(float t, float d, float h, float p0, float l) {
    const float v = d > 0.f ? h - __fmul_rn(t - l, d) : (d < 0.f ? (t - l) * -d : p0);
    return fminf(fmaxf(v, 0.f), h);
}

// Exit face (0..5: x-, x+, y-, y+, z-, z+) of a flight that reached halo voxel `lin`.
__device__ __forceinline__ int halo_face(const Geo& g, int lin) {
    int ix, iy, iz;
    unpad(g, lin, ix, iy, iz);
    return ix < 0 ? 0 : (ix >= g.nx ? 1 : (iy < 0 ? 2 : (iy >= g.ny ? 3 : (iz < 0 ? 4 : 5))));
}

// A flight that stopped in voxel f.lin (flight_step returned true) with b, m its extinction and
// face distance: a collision moves the photon to the collision point (offset inside the voxel
// and the voxel's indices) and returns kCollided; the halo returns the exit face. With S != 0 the
// collision voxel receives S * (1/beta - length) (one species) or, with two species (TWO), keeps
// its partial length in ph.tau for the event, which adds S * ([aerosol] / beta_aer - length) once
// the particle is known.
constexpr int kCollided = -2;

template <bool TWO>
__device__ __forceinline__ int flight_end(const TransportArgs& A, Photon& ph, const Flight& f, float tau, float b,
                                          float S, unsigned& nsc) {
    if (isinf(b)) return halo_face(A.g, f.lin);
    const float l = tau / b;
    ph.p = make_float3(flight_offset(f.tx, ph.d.x, A.g.hx, ph.p.x, l), flight_offset(f.ty, ph.d.y, A.g.hy, ph.p.y, l),
                       flight_offset(f.tz, ph.d.z, A.g.hz, ph.p.z, l));
    unpad(A.g, f.lin, ph.ix, ph.iy, ph.iz);
    if (S != 0.f) {
        if constexpr (TWO) {
            ph.tau = l;
        } else {
            atomicAdd(A.gacc + f.lin, S * (1.f / b - l));
            ++nsc;
        }
    }
    return kCollided;
}

// cosine between the photon direction and the direction from the photon to camera c, and the
// squared distance; r2 = 0 when the photon sits on the centre of projection
__device__ __forceinline__ float cam_cosine(const TransportArgs& A, const Photon& ph, const Cam& cm, float& r2) {
    const float3 v = local_delta(A.g, ph.ix, ph.iy, ph.iz, ph.p, cm.ix, cm.iy, cm.iz, make_float3(cm.lx, cm.ly, cm.lz));
    r2 = v.x * v.x + v.y * v.y + v.z * v.z;
    return r2 > 0.f ? (ph.d.x * v.x + ph.d.y * v.y + ph.d.z * v.z) * rsqrtf(r2) : 0.f;
}

// Step iv with two species (Sec. 2): the event's particle is air with probability
// beta_air / (beta_air + beta_aer) in its voxel. The uniform comes from the event's own Philox
// block x (the one its scattering draws use): u01 takes the top 23 bits of each word, so the low
// 9 bits of x.x and x.y and the low 5 bits of x.z give a 23-bit m, independent of those draws,
// and u = (2m + 1) / 2^24 (exact in FP32). The test u (beta_air + beta_aer) < beta_air runs in
// FP64 on the FP32 fields, so it takes the same branch as an FP64 evaluation of the same
// expression; an empty aerosol voxel always gives air (u < 1), an empty air voxel aerosol.
__device__ __forceinline__ bool particle_is_air(const TransportArgs& A, uint4 x, int k) {
    const uint32_t m = (x.x & 511u) | ((x.y & 511u) << 9) | ((x.z & 31u) << 18);
    const float u = __uint2float_rn(2u * m + 1u) * 5.9604644775390625e-08f;
    const double ba = (double)__ldg(A.beta_air + k);
    return (double)u * (ba + (double)__ldg(A.beta_aer + k)) < ba;
}

// phase function of the event's particle: Rayleigh (Eq. Pray) for air, HG (Eq. Phg) otherwise.
// The local estimates take the particle as a template parameter, so the one-species code keeps
// no per-camera select.
template <bool AIR>
__device__ __forceinline__ float phase_of(const TransportArgs& A, float mu) {
    if constexpr (AIR) return rayleigh_phase(mu);
    else return hg_phase(A.hg, mu);
}

// Eq. Lcupdate: L_c(k) += albedo I_s P(angle between the incoming ray and X_c - X_s), for all
// cameras at once, four cameras per vector atomic into the [nvox][cp] FP32 tile.
template <bool AIR>
__device__ __forceinline__ void le_voxel_p(const TransportArgs& A, const Photon& ph, float w, int k) {
    float* row = A.Lacc + (size_t)k * A.cp;
    for (int c0 = 0; c0 < A.cams.n; c0 += 4) {
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + j;
            float val = 0.f;
            if (c < A.cams.n) {
                float r2;
                const float mu = cam_cosine(A, ph, A.cams.c[c], r2);
                if (r2 > 0.f) val = w * phase_of<AIR>(A, mu);
            }
            v[j] = val;
        }
        atomicAdd(reinterpret_cast<float4*>(row + c0), make_float4(v[0], v[1], v[2], v[3]));
    }
}

__device__ __forceinline__ void le_voxel(const TransportArgs& A, const Photon& ph, float w, int k, bool air) {
    if (air) le_voxel_p<true>(A, ph, w, k);
    else le_voxel_p<false>(A, ph, w, k);
}

// w_s = sum_c a_c(k) albedo I_s P_c(s): the event's contribution to <a, L>.
template <bool AIR>
__device__ __forceinline__ float le_adjoint_p(const TransportArgs& A, const Photon& ph, float w, int k) {
    const float4* row = reinterpret_cast<const float4*>(A.adj + (size_t)k * A.cp);
    float acc = 0.f;
    for (int c0 = 0; c0 < A.cams.n; c0 += 4) {
        const float4 a4 = __ldg(row + (c0 >> 2));
        const float aa[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + j;
            if (c < A.cams.n && aa[j] != 0.f) {
                float r2;
                const float mu = cam_cosine(A, ph, A.cams.c[c], r2);
                if (r2 > 0.f) acc += aa[j] * w * phase_of<AIR>(A, mu);
            }
        }
    }
    return acc;
}

__device__ __forceinline__ float le_adjoint(const TransportArgs& A, const Photon& ph, float w, int k, bool air) {
    return air ? le_adjoint_p<true>(A, ph, w, k) : le_adjoint_p<false>(A, ph, w, k);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// A shadow ray of Eq. fle: the segment from a point (voxel (ix, iy, iz) + offset p) to camera
// cm's centre, walked on the padded grid like a free flight: per axis the distance to the next
// face (t) and between faces (q), the padded index stride of a crossing, and the length left.
struct Shadow {
    float tx, ty, tz, qx, qy, qz, rem;
    int dx, dy, dz, lin;
};

__device__ __forceinline__ Shadow shadow_init(const Geo& g, int ix, int iy, int iz, float3 p, const Cam& cm) {
    Shadow r;
    const float3 v = local_delta(g, ix, iy, iz, p, cm.ix, cm.iy, cm.iz, make_float3(cm.lx, cm.ly, cm.lz));
    r.rem = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
    const float inv = 1.f / r.rem;
    flight_axis(fminf(fmaxf(p.x, 0.f), g.hx), v.x * inv, g.hx, 1, r.tx, r.qx, r.dx);
    flight_axis(fminf(fmaxf(p.y, 0.f), g.hy), v.y * inv, g.hy, g.p0, r.ty, r.qy, r.dy);
    flight_axis(fminf(fmaxf(p.z, 0.f), g.hz), v.z * inv, g.hz, g.p01, r.tz, r.qz, r.dz);
    r.lin = pad_index(g, ix, iy, iz);
    return r;
}

// Its optical depth t_{s->c}. The walk ends at the camera or at the grid's boundary (the first
// halo voxel, extinction +inf: nothing outside the grid attenuates); nvox returns the voxels it
// crossed. The extinction is loaded two voxels ahead: the walk starts, and every step stands, in
// the grid, so the voxel after next lies at most in the second halo layer.
template <int DT>
__device__ __forceinline__ float shadow_tau(const TransportArgs& A, int ix, int iy, int iz, float3 p, const Cam& cm,
                                            unsigned& nvox) {
    Shadow r = shadow_init(A.g, ix, iy, iz, p, cm);
    float tx = r.tx, ty = r.ty, tz = r.tz, rem = r.rem;
    const float qx = r.qx, qy = r.qy, qz = r.qz;
    const int dx = r.dx, dy = r.dy, dz = r.dz;
    int lin = r.lin;
    float bn = BetaFetch<DT>::get(A.beta_pad, lin);
    float bn2;
    {
        const float m = fminf(tx, fminf(ty, tz));
        const bool px = tx <= m;
        const bool py = !px && ty <= m;
        bn2 = BetaFetch<DT>::get(A.beta_pad, lin + (px ? dx : (py ? dy : dz)));
    }
    float tau = 0.f;
#pragma unroll 1
    for (;;) {
        const float b = bn;
        if (isinf(b)) break;
        ++nvox;
        const float m = fminf(tx, fminf(ty, tz));
        const bool px = tx <= m;
        const bool py = !px && ty <= m;
        const int next = lin + (px ? dx : (py ? dy : dz));
        const float ux = px ? qx : tx - m;
        const float uy = py ? qy : ty - m;
        const float uz = (px || py) ? tz - m : qz;
        const float m2 = fminf(ux, fminf(uy, uz));
        const bool px2 = ux <= m2;
        const bool py2 = !px2 && uy <= m2;
        const bool last = !(rem > m);
        float bn3 = 0.f;
        if (!last) bn3 = BetaFetch<DT>::get(A.beta_pad, next + (px2 ? dx : (py2 ? dy : dz)));
        tau += b * (last ? rem : m);
        if (last) break;
        rem -= m;
        tx = ux;
        ty = uy;
        tz = uz;
        lin = next;
        bn = bn2;
        bn2 = bn3;
    }
    return tau;
}

// The shadow-ray terms d f / d beta_m = -f * (length in voxel m): the same walk again, its nvox
// voxels known from shadow_tau, so it loads no extinction; every voxel receives sw * length in
// the gradient tile (padded like the grid).
__device__ __forceinline__ void shadow_scatter(const TransportArgs& A, int ix, int iy, int iz, float3 p, const Cam& cm,
                                               float sw, unsigned nvox) {
    Shadow r = shadow_init(A.g, ix, iy, iz, p, cm);
#pragma unroll 1
    for (unsigned k = 0u; k < nvox; ++k) {
        const float m = fminf(r.tx, fminf(r.ty, r.tz));
        const bool px = r.tx <= m;
        const bool py = !px && r.ty <= m;
        const bool last = !(r.rem > m);
        atomicAdd(A.gacc + r.lin, sw * (last ? r.rem : m));
        if (last) break;
        r.rem -= m;
        r.tx = px ? r.qx : r.tx - m;
        r.ty = py ? r.qy : r.ty - m;
        r.tz = (px || py) ? r.tz - m : r.qz;
        r.lin += px ? r.dx : (py ? r.dy : r.dz);
    }
}

// Where an event lands in camera cm (Eq. fle): false when the camera does not see it (behind
// the camera, outside the image, on the centre, or, with a residual, a pixel of zero residual);
// else the pixel gp and f0 = albedo I_s P(mu) / (|X_c - X_s|^2 Omega_p), times the pixel's
// residual when RES.
template <bool RES>
__device__ __forceinline__ bool classic_pixel(const TransportArgs& A, const Photon& ph, const Cam& cm, float w, bool air,
                                              int& gp, float& f0) {
    const float3 v = local_delta(A.g, cm.ix, cm.iy, cm.iz, make_float3(cm.lx, cm.ly, cm.lz), ph.ix, ph.iy, ph.iz, ph.p);
    const float zc = v.x * cm.fx + v.y * cm.fy + v.z * cm.fz;
    if (!(zc > 0.f)) return false;
    const float x = (v.x * cm.rx + v.y * cm.ry + v.z * cm.rz) / zc;
    const float y = (v.x * cm.ux + v.y * cm.uy + v.z * cm.uz) / zc;
    const float px = floorf((x / cm.tx + 1.f) * 0.5f * (float)cm.w);
    const float py = floorf((y / cm.ty + 1.f) * 0.5f * (float)cm.h);
    if (px < 0.f || py < 0.f || px >= (float)cm.w || py >= (float)cm.h) return false;
    gp = cm.pix_off + (int)py * cm.w + (int)px;
    const float r2 = v.x * v.x + v.y * v.y + v.z * v.z;
    if (!(r2 > 0.f)) return false;
    float cr = 1.f;
    if (RES) {
        cr = (float)A.cres[gp];
        if (cr == 0.f) return false;
    }
    const float mu = -(ph.d.x * v.x + ph.d.y * v.y + ph.d.z * v.z) * rsqrtf(r2);
    f0 = cr * (w * (air ? rayleigh_phase(mu) : hg_phase(A.hg, mu)) / (r2 * A.omega[gp]));
    return true;
}

// Per-warp scratch of the classic estimate, in shared memory: for a group of kClassicGroup
// cameras, each (event lane, camera) pair's value f (res) and pixel (pix), and the list of shadow
// rays to walk (job: event lane | camera in the group << 5); per lane, the voxel segments its
// shadow rays walked, and the warp's count of shadow rays (MST_ST_SHADOW_*).
constexpr int kClassicGroup = 8;
constexpr int kClassicWords = kClassicGroup * 32 * 2 + kClassicGroup * 32 / 4 + 32 + 4;  // per warp
struct ClassicScratch {
    float* res;      // [kClassicGroup][32]
    int* pix;        // [kClassicGroup][32]
    uint8_t* job;    // [kClassicGroup * 32]
    unsigned* seg;   // [32]
    unsigned* rays;  // [1]
};

// Eq. fle for the warp's round of events (lane i < n holds event i; act says whether this lane
// holds one), shadow rays issued warp-coherently: the lanes first find, camera by camera, which
// cameras see their event and compact those (event, camera) pairs into a list; then every lane
// walks one shadow ray of the list at a time, 32 rays per pass over the list, so the warp's lanes
// stay busy however few cameras see each event. OP 0 adds each f = f0 exp(-t) to its pixel of
// the classic image; OP 1 returns w_s = sum_c cres[p] f (the event's share of <dE/di, i>, for the
// classic-estimator gradient), summed over the cameras in their order; OP 2 also scatters the
// shadow-ray terms -cres[p] f * (length in voxel m) into the gradient tile.
template <int DT, int OP>
__device__ __forceinline__ float le_classic(const TransportArgs& A, const Photon& e, float w, bool air, bool act,
                                            const ClassicScratch& cs) {
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t vox = (uint32_t)e.ix | ((uint32_t)e.iy << 11) | ((uint32_t)e.iz << 22);
    float acc = 0.f;
    for (int c0 = 0; c0 < A.cams.n; c0 += kClassicGroup) {
        const int gn = min(kClassicGroup, A.cams.n - c0);
        int qn = 0;
        for (int cl = 0; cl < gn; ++cl) {
            int gp = 0;
            float f0 = 0.f;
            const bool vis = act && classic_pixel<(OP > 0)>(A, e, A.cams.c[c0 + cl], w, air, gp, f0);
            cs.res[cl * 32 + lane] = vis ? f0 : 0.f;
            if (OP == 0) cs.pix[cl * 32 + lane] = gp;
            const unsigned vm = __ballot_sync(kFull, vis);
            if (vis) cs.job[qn + __popc(vm & lanemask_lt())] = (uint8_t)(lane | ((unsigned)cl << 5));
            qn += __popc(vm);
        }
        if (lane == 0u) *cs.rays += (unsigned)qn;
        __syncwarp();
        for (int j0 = 0; j0 < qn; j0 += 32) {
            const int j = j0 + (int)lane;
            const unsigned jb = j < qn ? cs.job[j] : 0u;
            const int el = (int)(jb & 31u), cl = (int)(jb >> 5);
            const uint32_t v = __shfl_sync(kFull, vox, el);
            const float3 p = make_float3(__shfl_sync(kFull, e.p.x, el), __shfl_sync(kFull, e.p.y, el),
                                         __shfl_sync(kFull, e.p.z, el));
            if (j < qn) {
                const Cam& cm = A.cams.c[c0 + cl];
                const int ix = (int)(v & 0x7FFu), iy = (int)((v >> 11) & 0x7FFu), iz = (int)(v >> 22);
                const int r = cl * 32 + el;
                unsigned nv = 0u;
                const float f = cs.res[r] * expf(-shadow_tau<DT>(A, ix, iy, iz, p, cm, nv));
                if (OP == 0) {
                    atomicAdd(A.cimg + cs.pix[r], (double)f);
                } else {
                    cs.res[r] = f;
                    if (OP == 2) shadow_scatter(A, ix, iy, iz, p, cm, -f, nv);
                }
                cs.seg[lane] += OP == 2 ? 2u * nv : nv;
            }
        }
        __syncwarp();
        if (OP > 0)
            for (int cl = 0; cl < gn; ++cl) acc += cs.res[cl * 32 + lane];
        __syncwarp();
    }
    return acc;
}

// step v (albedo weighting, Russian roulette) and step vi (new direction by the particle's
// phase function, next free path). Returns 0 to continue or the termination code.
// PRE: x is the event's Philox block, already drawn (two species: the particle came from it).
template <bool PRE, typename TallyT>
__device__ __forceinline__ int after_event(const TransportArgs& A, Photon& ph, TallyT& t, bool air, uint4 x) {
    const float alb = air ? A.albedo_air : A.albedo;
    t.add_absorbed((1.f - alb) * ph.I);
    ph.I *= alb;
    if (ph.I == 0.f) return 2;
    if (A.max_order > 0 && (int)ph.s >= A.max_order) {
        t.add_forced(ph.I);
        return 4;
    }
    if ((int)ph.s >= A.max_events) {
        t.add_forced(ph.I);
        t.add_capped();
        return 5;
    }
    const float4 u = PRE ? u01x4(x) : draws(A.key, ph.id, ph.s);
    if (ph.I < A.rr_below) {
        if (u.z < A.rr_survival) {
            t.add_gained(ph.I * (A.inv_rr_survival - 1.f));
            ph.I *= A.inv_rr_survival;
        } else {
            t.add_killed(ph.I);
            return 3;
        }
    }
    float ct, st;
    if (air) rayleigh_sample(u.x, ct, st);
    else hg_sample(A.hg, u.x, ct, st);
    ph.d = rotate_dir(ph.d, ct, st, u.y);
    ph.tau = -logf(1.f - u.w);
    return 0;
}

__device__ __forceinline__ void finish_photon(const TransportArgs& A, const Photon& ph, int term) {
    uint32_t h = (ph.hash ^ ph.s) * kFnvPrime;
    h = (h ^ (uint32_t)term) * kFnvPrime;
    if (A.hash) A.hash[ph.idx] = h;
    if (A.point)
        A.point[ph.idx] = make_float4(ph.p.x, ph.p.y, ph.p.z,
                                      __uint_as_float((uint32_t)ph.ix | ((uint32_t)ph.iy << 11) | ((uint32_t)ph.iz << 22)));
    if (A.ev_cap) A.nevbuf[ph.idx - A.out_base] = ph.s;  // forward storing events: the count pass 2 stops at
}

// One stored event (forward, full gradient): what w_s = sum_c a_c(k) albedo I_s P_c(s) needs.
// Word 9 holds the event number, with the particle (1: air) in bit 31; word 10 the free path left
// when the flight entered the event's voxel (e.tau, set at the collision), with which replay
// pass 2 ends the flight there.
__device__ __forceinline__ void store_event(const TransportArgs& A, unsigned long long i, const Photon& e, float wgt,
                                            bool air) {
    const unsigned long long C = A.ev_cap;
    uint32_t* r = A.evrec + i;
    r[0] = (uint32_t)e.ix | ((uint32_t)e.iy << 11) | ((uint32_t)e.iz << 22);
    r[C] = __float_as_uint(e.p.x);
    r[2 * C] = __float_as_uint(e.p.y);
    r[3 * C] = __float_as_uint(e.p.z);
    r[4 * C] = __float_as_uint(e.d.x);
    r[5 * C] = __float_as_uint(e.d.y);
    r[6 * C] = __float_as_uint(e.d.z);
    r[7 * C] = __float_as_uint(wgt);
    r[8 * C] = e.idx - A.out_base;
    r[9 * C] = e.s | (air ? 0x80000000u : 0u);
    r[10 * C] = __float_as_uint(e.tau);  // the free path left on entering the event's voxel
}

// ------------------------------------------------------------------------------------------
// Per-warp photon stacks in shared memory (structure of arrays: lane i touches word i, so
// pushes and pops are free of bank conflicts). A warp holds at most 32 flying photons, fewer
// than 32 queued events once a round of events is done (events are processed 32 at a time as
// soon as 32 are queued) and a ready stack: new photons are launched only when the ready stack
// is empty, so right after a launch a warp holds 32 flying + at most 31 queued photons and never
// more than 63 in total. The event and ready stacks therefore share one array of kSlots = 64
// slots, the events growing up from slot 0 and the ready photons down from slot 63: together
// they never hold more than 63. (Two separate 64-slot stacks took 49 KB of shared memory per
// block of the forward, which the SM's L1 gives up to hold the extinction grid.)

constexpr int kScoreTile = 4096;   // photons per block in the list kernels
// Stored events are written in per-warp chunks of kEvChunk slots (one reservation on the global
// counter per chunk). A warp's photons come from its own ticket batches, so a chunk holds the
// events of a few dozen photons, and the adjoint that walks a chunk finds their W and step slots
// together in cache instead of scattered over all photons in flight. The buffer keeps one chunk
// per resident warp of headroom for the chunks' unused tails.
constexpr unsigned kEvChunk = kEventChunk;
static_assert(kTB / 32 == kTransportWarps, "transport block size");
constexpr uint32_t kNoPhoton = 0xFFFFFFFFu;  // photon word of a chunk's unused tail slots
constexpr int kSlots = 64;
// Voxels a flying lane advances per loop trip, and minimum resident blocks per SM (register
// budget), per kernel mode; set from sweeps on the 64^3 cumulus workload.
constexpr int kStepsForward = 12;
constexpr int kStepsPass1 = 8;
constexpr int kStepsPass2 = 6;
constexpr int kMinBlocksForward = 3;
constexpr int kMinBlocksClassic = 3;
constexpr int kMinBlocksPass1 = 3;
constexpr int kMinBlocksPass2 = 3;

// kernel modes
// kPass2W: replay pass 2 reading w_s from the stored events instead of recomputing them;
// kPass1C, kPass2C: passes 1 and 2 of the classic-estimator gradient
constexpr int kFwdVoxel = 0, kFwdClassic = 1, kPass2 = 2, kPass1 = 3, kPass2W = 4, kPass1C = 5, kPass2C = 6;

template <int NW>
struct Stack {
    uint32_t* w;  // NW arrays of cap words
    int cap;
};

template <bool REPLAY>
struct Rec {
    static constexpr int NW = REPLAY ? 15 : 12;
};

template <int NW>
__device__ __forceinline__ void put(const Stack<NW>& q, int slot, const Photon& ph, uint32_t nev, double acc) {
    uint32_t* b = q.w + slot;
    const int c = q.cap;
    b[0 * c] = __float_as_uint(ph.p.x);
    b[1 * c] = __float_as_uint(ph.p.y);
    b[2 * c] = __float_as_uint(ph.p.z);
    b[3 * c] = __float_as_uint(ph.d.x);
    b[4 * c] = __float_as_uint(ph.d.y);
    b[5 * c] = __float_as_uint(ph.d.z);
    b[6 * c] = (uint32_t)ph.ix | ((uint32_t)ph.iy << 11) | ((uint32_t)ph.iz << 22);
    b[7 * c] = __float_as_uint(ph.I);
    b[8 * c] = __float_as_uint(ph.tau);
    b[9 * c] = ph.s;
    b[10 * c] = ph.hash;
    b[11 * c] = ph.idx;
    if (NW > 12) {
        b[12 * c] = nev;
        b[13 * c] = (uint32_t)__double_as_longlong(acc);
        b[14 * c] = (uint32_t)((unsigned long long)__double_as_longlong(acc) >> 32);
    }
}

template <int NW>
__device__ __forceinline__ void get(const Stack<NW>& q, int slot, const TransportArgs& A, Photon& ph, uint32_t& nev,
                                    double& acc) {
    const uint32_t* b = q.w + slot;
    const int c = q.cap;
    ph.p = make_float3(__uint_as_float(b[0]), __uint_as_float(b[c]), __uint_as_float(b[2 * c]));
    ph.d = make_float3(__uint_as_float(b[3 * c]), __uint_as_float(b[4 * c]), __uint_as_float(b[5 * c]));
    const uint32_t v = b[6 * c];
    ph.ix = (int)(v & 0x7FFu);
    ph.iy = (int)((v >> 11) & 0x7FFu);
    ph.iz = (int)(v >> 22);
    ph.I = __uint_as_float(b[7 * c]);
    ph.tau = __uint_as_float(b[8 * c]);
    ph.s = b[9 * c];
    ph.hash = b[10 * c];
    ph.idx = b[11 * c];
    ph.id = A.first_id + (ph.idx - A.out_base);
    if (NW > 12) {
        nev = b[12 * c];
        acc = __longlong_as_double((long long)((unsigned long long)b[13 * c] | ((unsigned long long)b[14 * c] << 32)));
    } else {
        nev = 0u;
        acc = 0.0;
    }
}

// Two species: the event's Philox block waits in the event's own stack slot (popped, so free
// until the next trip pushes events) while the local estimate runs, instead of in registers.
// Volatile, so the compiler reloads it rather than keeping the words live.
template <int NW>
__device__ __forceinline__ void stash_block(const Stack<NW>& q, int slot, uint4 x) {
    volatile uint32_t* b = q.w + slot;
    const int c = q.cap;
    b[0] = x.x;
    b[c] = x.y;
    b[2 * c] = x.z;
    b[3 * c] = x.w;
}

template <int NW>
__device__ __forceinline__ uint4 unstash_block(const Stack<NW>& q, int slot) {
    const volatile uint32_t* b = q.w + slot;
    const int c = q.cap;
    return make_uint4(b[0], b[c], b[2 * c], b[3 * c]);
}

// One slice of the rolling fold (see kFoldSweep): the warp swaps the slice's FP32 bins to zero
// and adds what it took to the FP64 result. Transport lanes keep adding to the same bins with
// 32-bit atomics, so nothing added is lost; each bin's FP32 partial covers at most one sweep.
template <int MODE>
__device__ __forceinline__ void fold_slice(const TransportArgs& A, uint32_t batch, unsigned lane) {
    if constexpr (MODE == kFwdVoxel || MODE == kPass2 || MODE == kPass2W || MODE == kPass2C) {
        if (A.fold_bins == 0u) return;
        const uint64_t i0 = (uint64_t)(batch % A.fold_nslices) * A.fold_slice;
        const uint64_t i1 = min(i0 + A.fold_slice, A.fold_bins);
        for (uint64_t i = i0 + lane; i < i1; i += 32) {
            if (MODE == kFwdVoxel) {  // L tile [nvox][cp] -> L64 [C][nvox]
                const uint64_t k = i / (uint32_t)A.cp;
                const int c = (int)(i - k * (uint32_t)A.cp);
                if (c < A.cams.n) {
                    const float v = atomicExch(A.Lacc + i, 0.f);
                    if (v != 0.f) atomicAdd(A.L64 + (size_t)c * A.g.nvox + k, (double)v);
                }
            } else {  // gradient tile [nvox] -> g64 [nvox]
                const float v = atomicExch(A.gacc + i, 0.f);  // padded tile
                int k;
                if (v != 0.f && interior_lin(A.g, (int)i, k)) atomicAdd(A.g64 + k, (double)v);
            }
        }
    }
}

// Warp-uniform refill from the pool of n work items: lanes without a photon take the next
// items of the warp's slice, lane 0 refilling the slice from the launch's global ticket.
// on_launch(j) starts item j and returns whether the lane now has a photon; on_batch(t0) runs
// on the whole warp after each new batch.
template <typename LaunchFn, typename BatchFn>
__device__ __forceinline__ void refill(const TransportArgs& A, uint32_t n, bool& fly, bool& dry, uint32_t& wbase,
                                       uint32_t& wend, unsigned lane, LaunchFn&& on_launch, BatchFn&& on_batch) {
    unsigned need = __ballot_sync(kFull, !fly);
    while (need != 0u && !dry) {
        if (wbase >= wend) {
            unsigned t0 = 0u;
            if (lane == 0u) t0 = atomicAdd(A.ticket, (unsigned)kTicketBatch);
            t0 = __shfl_sync(kFull, t0, 0);
            if (t0 >= n) {
                dry = true;
                break;
            }
            wbase = t0;
            wend = min(t0 + (unsigned)kTicketBatch, n);
            on_batch(t0);
        }
        const unsigned rank = __popc(need & lanemask_lt());
        const unsigned avail = wend - wbase;
        if (!fly && rank < avail) fly = on_launch(wbase + rank);
        wbase += min((unsigned)__popc(need), avail);
        need = __ballot_sync(kFull, !fly);
    }
}

__device__ __forceinline__ void flush_tally(const TransportArgs& A, const Tally& t, unsigned segments,
                                            unsigned events, unsigned lane) {
    double v[11];
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = warp_sum((double)t.esc[q]);
    v[6] = warp_sum((double)t.absorbed);
    v[7] = warp_sum((double)t.killed);
    v[8] = warp_sum((double)t.gained);
    v[9] = warp_sum((double)t.forced);
    v[10] = warp_sum((double)t.launched);
    const unsigned long long ev = warp_sumu(events), sg = warp_sumu(segments);
    const unsigned long long cap = warp_sumu(t.capped), esc = warp_sumu(t.escaped), tr = warp_sumu(t.traced);
    const unsigned long long lost = warp_sumu(t.lost);
    if (lane == 0u) {
#pragma unroll
        for (int q = 0; q < 6; ++q)
            if (v[q] != 0.0) atomicAdd(A.stats + MST_ST_ESC_XM + q, v[q]);
        atomicAdd(A.stats + MST_ST_ABSORBED, v[6]);
        atomicAdd(A.stats + MST_ST_RR_KILLED, v[7]);
        atomicAdd(A.stats + MST_ST_RR_GAINED, v[8]);
        atomicAdd(A.stats + MST_ST_FORCED, v[9]);
        atomicAdd(A.stats + MST_ST_LAUNCHED, v[10]);
        atomicAdd(A.stats + MST_ST_EVENTS, (double)ev);
        atomicAdd(A.stats + MST_ST_SEGMENTS, (double)sg);
        atomicAdd(A.stats + MST_ST_CAPPED, (double)cap);
        atomicAdd(A.stats + MST_ST_ESCAPED_N, (double)esc);
        atomicAdd(A.stats + MST_ST_TRACED, (double)tr);
        if (lost) atomicAdd(A.stats + MST_ST_LOST, (double)lost);
    }
}

// ------------------------------------------------------------------------------------------
// The transport kernel. MODE 0: forward with the voxelised local estimate; 1: forward with the
// classic local estimate; 3 and 2: the two passes of the replay adjoint. Every loop trip (1) fills empty lanes from the
// ready stack, then from the id pool, (2) advances every flying photon by one voxel, pushing
// collisions onto the event stack, and (3) whenever 32 events are queued (or the chunk is
// draining), processes 32 events at once: local estimate, albedo, roulette, new direction;
// photons that go on are pushed onto the ready stack.
//
// Replay adjoint, two launches per chunk. Pass 1 (MODE 3) walks every photon and stores
// W = sum_s w_s, w_s = sum_c a_c(k_s) albedo I_s P_c(s), and its event count per photon; the
// photons with W != 0 are then gathered into a list, longest first. Pass 2 (MODE 2) walks the
// listed photons again, with S_j = W - sum_{s<j} w_s (FP64), and
// scatters the score of every flight that ends in an event; it stops at pass 1's last event.
// Both passes run the same flight and event arithmetic, so they see the same path.
// TWO: two-species medium (the launch has an air field); one-species kernels carry none of its
// code. TRIP: voxels a flying lane advances per loop trip (0: the mode's default), a compile-time
// constant (a run-time bound cost the forward 2 %); the autotuner picks among the instantiated ones.
constexpr int min_blocks(int mode) {
    return (mode == kPass2 || mode == kPass2W)
               ? kMinBlocksPass2
               : (mode == kPass1 ? kMinBlocksPass1
                                 : ((mode == kFwdClassic || mode == kPass1C || mode == kPass2C) ? kMinBlocksClassic
                                                                                                 : kMinBlocksForward));
}

// One scene's photons, run by every warp of the launch until the scene's pool is dry and the
// warp holds none of its photons (flying, queued for an event or ready).
template <int DT, int MODE, bool TWO, int TRIP>
__device__ __forceinline__ void transport_run(const TransportArgs& A, uint32_t* smem) {
    constexpr bool PASS1 = MODE == kPass1 || MODE == kPass1C;
    constexpr bool PASS2 = MODE == kPass2 || MODE == kPass2W || MODE == kPass2C;
    constexpr bool CLASSIC = MODE == kFwdClassic || MODE == kPass1C || MODE == kPass2C;
    constexpr bool REPLAY = PASS1 || PASS2;
    constexpr int kStepsPerTrip = TRIP > 0 ? TRIP : (PASS2 ? kStepsPass2 : (PASS1 ? kStepsPass1 : kStepsForward));
    constexpr int NW = Rec<REPLAY>::NW;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned warp = threadIdx.x >> 5;
    const Stack<NW> stk{smem + warp * NW * kSlots, kSlots};  // events at slot i, ready photons at kSlots-1-i
    int ev_n = 0, rd_n = 0;  // warp-uniform stack heights
    unsigned long long ch_base = ~0ull;  // forward storing events: the warp's current chunk (none yet) ...
    unsigned ch_fill = kEvChunk;         // ... and its slots in use
    const uint32_t gwarp = blockIdx.x * (kTB / 32) + warp;  // the warp's chunk list

    // photon tallies: forward render only, one shared-memory slot per thread after the stacks
    typename std::conditional<REPLAY, NoTally, LaneTally>::type t;
    if constexpr (!REPLAY) {
        float* tb = reinterpret_cast<float*>(smem + (kTB / 32) * NW * kSlots);
        t.f = tb + threadIdx.x;
        t.u = reinterpret_cast<unsigned*>(tb + 11 * kTB) + threadIdx.x;
    }
    t.zero();
    ClassicScratch cls{};  // the classic estimate's per-warp scratch, after the stacks and tallies
    if constexpr (CLASSIC) {
        uint32_t* cb = smem + (kTB / 32) * NW * kSlots + (REPLAY ? 0 : kTB * 15) + warp * kClassicWords;
        cls.res = reinterpret_cast<float*>(cb);
        cls.pix = reinterpret_cast<int*>(cb + kClassicGroup * 32);
        cls.job = reinterpret_cast<uint8_t*>(cb + 2 * kClassicGroup * 32);
        cls.seg = cb + 2 * kClassicGroup * 32 + kClassicGroup * 8;
        cls.rays = cls.seg + 32;
        cls.seg[lane] = 0u;
        if (lane == 0u) *cls.rays = 0u;
        __syncwarp();
    }

    Photon ph;
    Flight w;
    float tau = 0.f;
    uint32_t nev = 0u;  // pass 2: events of pass 1
    double acc = 0.0;   // pass 1: W; pass 2: S
    bool fly = false, dry = false;
    uint32_t wbase = 0u, wend = 0u;
    unsigned segments = 0u, scatters = 0u, events = 0u;
    EventCount<TWO && !REPLAY> air_events;  // two species: forward events on air
    const uint32_t pool_n = PASS2 ? *A.plist_n : A.n;  // pass 2 walks the list built from pass 1
    if (A.ev_cap) {  // a call whose forward stored its events: one of each pair of kernels works
        const bool fit = *A.ev_count <= A.ev_cap;
        if ((PASS1 || MODE == kPass2) && fit) return;  // W and w_s come from the stored events
        if (MODE == kPass2W && !fit) return;           // they did not fit: pass 1 and kPass2 run
    }

    for (;;) {
        // (1) fill: ready photons first, new photons only when the ready stack is empty
        unsigned empty = __ballot_sync(kFull, !fly);
        if (empty != 0u && rd_n > 0) {
            const int rank = __popc(empty & lanemask_lt());
            const int take = min(__popc(empty), rd_n);
            if (!fly && rank < take) {
                get(stk, kSlots - rd_n + rank, A, ph, nev, acc);
                if constexpr (MODE == kPass2W) {
                    flight_init_stored(w, A, ph, tau);
                } else {
                    flight_init<DT>(w, A, ph);
                    tau = ph.tau;
                }
                fly = true;
            }
            rd_n -= take;
            __syncwarp();
        }
        refill(A, pool_n, fly, dry, wbase, wend, lane, [&](uint32_t j) -> bool {
            uint32_t pid = j;
            nev = 0u;
            acc = 0.0;
            if (PASS2) {  // item j of the pass-1 list
                const ScoreRec r = A.plist[j];
                pid = r.pid;
                nev = r.nev;
                acc = r.W;
            } else if (A.skip && A.skip[A.out_base + j]) {
                if (A.hash) A.hash[A.out_base + j] = 0u;
                if (PASS1) A.wbuf[j] = 0.0;
                if (PASS1 || A.ev_cap) A.nevbuf[j] = 0u;
                return false;
            }
            launch_photon(A, ph, pid);
            if constexpr (MODE == kPass2W) {
                ph.hash = A.evoff[pid];
                flight_init_stored(w, A, ph, tau);
            } else {
                flight_init<DT>(w, A, ph);
                tau = ph.tau;
            }
            t.add_launch(A.I0);
            return true;
        }, [&](uint32_t t0) { fold_slice<MODE>(A, t0 / (uint32_t)kTicketBatch, lane); });
        const bool any_fly = __any_sync(kFull, fly);
        if (!any_fly && ev_n == 0 && rd_n == 0 && dry) break;

        // (2) up to kStepsPerTrip voxels for every flying photon
        int r = -1;
        if (fly) {
            const float S = PASS2 ? (float)acc : 0.f;
            int nstep = 0;
            bool stop = false;
            float b = 0.f, m = 0.f;
            if constexpr (MODE == kPass2W) {  // the flight's last voxel is known: no extinction before it
#pragma unroll 1
                while (nstep < kStepsPerTrip) {
                    ++nstep;
                    if (flight_step_stored(A, w, S, scatters)) {
                        stop = true;
                        break;
                    }
                }
                if (stop) {
                    r = (unsigned)w.lin < (unsigned)A.g.npad
                            ? flight_end<TWO>(A, ph, w, tau, BetaFetch<DT>::get(A.beta_pad, w.lin), S, scatters)
                            : kWalkOverflow;
                    // a stored flight ends in its event; any other end is a replay that left the
                    // forward's path, counted as lost (0 in valid use; the fold drops what such a
                    // walk added to the halo)
                    if (r != kCollided) atomicAdd(A.stats + MST_ST_LOST, 1.0);
                }
            } else {
#pragma unroll 1
                while (nstep < kStepsPerTrip) {
                    ++nstep;
                    if (flight_step<DT, PASS2>(A, w, tau, b, m, S, scatters)) {
                        stop = true;
                        break;
                    }
                }
                if (stop) {
                    r = flight_end<TWO>(A, ph, w, tau, b, S, scatters);
                    if (r >= 0) --nstep;  // the halo voxel is no segment of the path
                    if (MODE == kFwdVoxel && r == kCollided) ph.tau = tau;  // kept for the stored event
                }
            }
            segments += nstep;
            // a flight longer than any straight walk through the grid is abandoned
            w.left -= nstep;
            if (r == -1 && w.left < 0) r = kWalkOverflow;
        }
        const bool collided = fly && r == kCollided;
        const unsigned cmask = __ballot_sync(kFull, collided);
        if (collided) {
            put(stk, ev_n + __popc(cmask & lanemask_lt()), ph, nev, acc);
            fly = false;
        } else if (fly && r >= 0) {
            if (REPLAY) {
                if (PASS1) {
                    A.wbuf[ph.idx - A.out_base] = acc;
                    A.nevbuf[ph.idx - A.out_base] = ph.s;
                }
                fly = false;
            } else {
                t.add_escape(r, ph.I);
                finish_photon(A, ph, 1);
                fly = false;
            }
        }
        ev_n += __popc(cmask);
        __syncwarp();

        // (3) events, 32 at a time (fewer only while draining)
        while (ev_n >= 32 || (ev_n > 0 && dry && rd_n == 0 && !__any_sync(kFull, fly))) {
            const int n = min(32, ev_n);
            Photon e;
            uint32_t enev = 0u;
            double eacc = 0.0;
            int term = -1;  // -1 idle lane, 0 goes on, > 0 ended
            unsigned long long ev_slot = 0ull;  // forward storing events: this lane's record slot
            if (MODE == kFwdVoxel && A.ev_cap) {
                // the round's slots continue the warp's chunk and spill into a new one
                unsigned long long nb = 0ull;
                if (ch_fill + (unsigned)n > kEvChunk) {  // a new chunk, linked after the warp's last one
                    if (lane == 0u) {
                        nb = atomicAdd(A.ev_count, (unsigned long long)kEvChunk);
                        const uint32_t nc = (uint32_t)(nb / kEvChunk);
                        if (ch_base == ~0ull) A.warp_head[gwarp] = nc;
                        else if (ch_base + kEvChunk <= A.ev_cap) A.ch_next[ch_base / kEvChunk] = nc;
                    }
                    nb = __shfl_sync(kFull, nb, 0);
                }
                const unsigned f = ch_fill + lane;
                ev_slot = f < kEvChunk ? ch_base + f : nb + (f - kEvChunk);
                if (ch_fill + (unsigned)n > kEvChunk) {
                    ch_base = nb;
                    ch_fill = ch_fill + (unsigned)n - kEvChunk;
                } else {
                    ch_fill += (unsigned)n;
                }
            }
            if constexpr (CLASSIC) {
                // the classic estimate runs on the whole warp (its shadow rays are spread over all
                // lanes), between the event's per-lane first half and its second
                const bool act = (int)lane < n;
                const int slot = ev_n - 1 - (int)lane;
                bool air = false;
                float wgt = 0.f;
                if (act) {
                    get(stk, slot, A, e, enev, eacc);
                    e.s += 1u;
                    ++events;
                    const int k = lin_index(A.g, e.ix, e.iy, e.iz);
                    if constexpr (TWO) {
                        const uint4 x = draw_bits(A.key, e.id, e.s);
                        air = particle_is_air(A, x, k);
                        stash_block(stk, slot, x);
                    }
                    if (air) air_events.add();
                    wgt = (air ? A.albedo_air : A.albedo) * e.I;
                    if (!REPLAY) e.hash = (e.hash ^ (uint32_t)k) * kFnvPrime;
                }
                const float we = le_classic<DT, REPLAY ? (PASS2 ? 2 : 1) : 0>(A, e, wgt, air, act, cls);
                if (act) {
                    uint4 xb = make_uint4(0u, 0u, 0u, 0u);
                    if constexpr (TWO) xb = unstash_block(stk, slot);
                    if (!REPLAY) {
                        term = after_event<TWO>(A, e, t, air, xb);
                        if (term) finish_photon(A, e, term);
                    } else if (PASS1) {
                        eacc += (double)we;
                        term = after_event<TWO>(A, e, t, air, xb);
                        if (term) {
                            A.wbuf[e.idx - A.out_base] = eacc;
                            A.nevbuf[e.idx - A.out_base] = e.s;
                        }
                    } else {
                        const float S = (float)eacc;  // the score weight of the flight that ended here
                        if (TWO && S != 0.f) {  // two species: the collision voxel's term (see flight_step)
                            atomicAdd(A.gacc + pad_index(A.g, e.ix, e.iy, e.iz),
                                      S * ((air ? 0.f : 1.f / __ldg(A.beta_aer + lin_index(A.g, e.ix, e.iy, e.iz))) -
                                           e.tau));
                            ++scatters;
                        }
                        eacc -= (double)we;
                        term = e.s == enev ? 1 : after_event<TWO>(A, e, t, air, xb);  // stop at pass 1's last event
                    }
                }
            } else {  // the voxelised estimate (or the stored w_s), per lane
                if ((int)lane < n) {
                    get(stk, ev_n - 1 - (int)lane, A, e, enev, eacc);
                    e.s += 1u;
                    ++events;
                    const int k = lin_index(A.g, e.ix, e.iy, e.iz);
                    const int slot = ev_n - 1 - (int)lane;
                    uint4 xb = make_uint4(0u, 0u, 0u, 0u);  // two species: the event's Philox block
                    bool air = false;
                    if constexpr (TWO) {
                        const uint4 x = draw_bits(A.key, e.id, e.s);
                        air = particle_is_air(A, x, k);
                        stash_block(stk, slot, x);
                    }
                    if (air) air_events.add();
                    const float wgt = (air ? A.albedo_air : A.albedo) * e.I;
                    if (!REPLAY) {
                        e.hash = (e.hash ^ (uint32_t)k) * kFnvPrime;
                        if (MODE == kFwdVoxel && A.ev_cap && ev_slot < A.ev_cap) store_event(A, ev_slot, e, wgt, air);
                        le_voxel(A, e, wgt, k, air);
                        if constexpr (TWO) xb = unstash_block(stk, slot);
                        term = after_event<TWO>(A, e, t, air, xb);
                        if (term) finish_photon(A, e, term);
                    } else {
                        float we;
                        if constexpr (MODE == kPass2W) we = A.wseq[e.hash + e.s - 1u].w;
                        else we = le_adjoint(A, e, wgt, k, air);
                        if (PASS1) {
                            eacc += (double)we;
                            if constexpr (TWO) xb = unstash_block(stk, slot);
                            term = after_event<TWO>(A, e, t, air, xb);
                            if (term) {
                                A.wbuf[e.idx - A.out_base] = eacc;
                                A.nevbuf[e.idx - A.out_base] = e.s;
                            }
                        } else {
                            const float S = (float)eacc;  // the score weight of the flight that ended here
                            if (TWO && S != 0.f) {  // two species: the collision voxel's term (see flight_step)
                                atomicAdd(A.gacc + pad_index(A.g, e.ix, e.iy, e.iz),
                                          S * ((air ? 0.f : 1.f / __ldg(A.beta_aer + k)) - e.tau));
                                ++scatters;
                            }
                            if constexpr (TWO) xb = unstash_block(stk, slot);
                            term = e.s == enev ? 1 : after_event<TWO>(A, e, t, air, xb);  // stop at pass 1's last event
                            eacc -= (double)we;  // after the scattering step, which hides the w_s load
                        }
                    }
                }
            }
            ev_n -= n;
            __syncwarp();
            const unsigned gmask = __ballot_sync(kFull, term == 0);
            if (term == 0) put(stk, kSlots - 1 - (rd_n + __popc(gmask & lanemask_lt())), e, enev, eacc);
            rd_n += __popc(gmask);
            __syncwarp();
        }
    }
    if constexpr (CLASSIC) {
        const unsigned long long ss = warp_sumu(cls.seg[lane]);
        if (lane == 0u) {
            atomicAdd(A.stats + MST_ST_SHADOW_RAYS, (double)*cls.rays);
            atomicAdd(A.stats + MST_ST_SHADOW_SEGMENTS, (double)ss);
        }
    }
    if constexpr (REPLAY) {
        const unsigned long long ev = warp_sumu(events), sg = warp_sumu(segments), sc = warp_sumu(scatters);
        if (lane == 0u) {
            atomicAdd(A.stats + MST_ST_REPLAY_EVENTS, (double)ev);
            atomicAdd(A.stats + MST_ST_REPLAY_SEGMENTS, (double)sg);
            atomicAdd(A.stats + MST_ST_REPLAY_SCATTERS, (double)sc);
        }
    } else {
        flush_tally(A, t.load(), segments, events, lane);
        air_events.flush(A.stats + MST_ST_AIR_EVENTS, lane);
        if (MODE == kFwdVoxel && A.ev_cap) {  // close the warp's list; its last chunk's tail holds no event
            if (ch_base == ~0ull) {
                if (lane == 0u) A.warp_head[gwarp] = kEndChunk;
            } else {
                if (lane == 0u && ch_base + kEvChunk <= A.ev_cap) A.ch_next[ch_base / kEvChunk] = kEndChunk;
                for (unsigned f = ch_fill + lane; f < kEvChunk; f += 32u)
                    if (ch_base + f < A.ev_cap) A.evrec[8ull * A.ev_cap + ch_base + f] = kNoPhoton;
            }
        }
    }
}

template <int DT, int MODE, bool TWO, int TRIP = 0>
__global__ void __launch_bounds__(kTB, min_blocks(MODE)) k_transport(const TransportArgs A) {
    extern __shared__ uint32_t smem[];
    transport_run<DT, MODE, TWO, TRIP>(A, smem);
}

// Many scenes in one persistent launch (the batched form): every warp runs the scenes one after
// the other from a table in device memory, each until its photons are done, so the launch ends on
// one tail instead of one per scene and small scenes fill the GPU together with large ones.
template <int DT, int MODE, bool TWO, int TRIP = 0>
__global__ void __launch_bounds__(kTB, min_blocks(MODE))
    k_transport_batch(const TransportArgs* __restrict__ scenes, int n_scenes) {
    extern __shared__ uint32_t smem[];
    for (int s = 0; s < n_scenes; ++s) {
        transport_run<DT, MODE, TWO, TRIP>(scenes[s], smem);
        __syncwarp();
    }
}

// w_s of every event the forward stored, instead of replay pass 1: the same arithmetic
// (le_adjoint) on the same event state, written with the event's voxel and free path to the
// photon's step slot in wseq for pass 2, and added to W in FP64; nevbuf (zeroed after the slot
// scan) receives each photon's last event with w_s != 0. Does nothing when the events did not
// fit (pass 1 then walks the paths).
template <bool TWO>
__device__ __forceinline__ void event_adjoint_run(const TransportArgs& A) {
    const unsigned long long cnt = *A.ev_count;  // reserved slots: whole chunks
    if (cnt > A.ev_cap) return;
    const unsigned long long C = A.ev_cap;
    unsigned long long stored = 0ull;
    // A block follows one forward warp's chunks in the order the warp wrote them (lists taken
    // from a ticket): a photon's events lie in one or two neighbouring chunks of its warp, so its
    // W, offset and step slots are used while they are still cached.
    __shared__ uint32_t list;
    for (;;) {
        if (threadIdx.x == 0) list = atomicAdd(A.ticket, 1u);
        __syncthreads();
        const uint32_t gw = list;
        __syncthreads();
        if (gw >= A.n_warps) break;
        for (uint32_t ch = A.warp_head[gw], next; ch != kEndChunk; ch = next) {
            next = A.ch_next[ch];  // issued first, so its latency overlaps the chunk's work
            for (unsigned q = threadIdx.x; q < kEvChunk; q += kTB) {
                const uint32_t* r = A.evrec + (unsigned long long)ch * kEvChunk + q;
                const uint32_t j = r[8 * C];
                if (j == kNoPhoton) continue;
                ++stored;
                const uint32_t v = r[0];
                Photon e;
                e.ix = (int)(v & 2047u);
                e.iy = (int)((v >> 11) & 2047u);
                e.iz = (int)(v >> 22);
                e.p = make_float3(__uint_as_float(r[C]), __uint_as_float(r[2 * C]), __uint_as_float(r[3 * C]));
                e.d = make_float3(__uint_as_float(r[4 * C]), __uint_as_float(r[5 * C]), __uint_as_float(r[6 * C]));
                const uint32_t sw = r[9 * C];  // event number, particle in bit 31
                const float w = le_adjoint(A, e, __uint_as_float(r[7 * C]), lin_index(A.g, e.ix, e.iy, e.iz),
                                           TWO && (sw >> 31) != 0u);
                const uint32_t s = sw & 0x7FFFFFFFu;
                // event s of photon j: slot evoff[j] + s - 1 (one 16-byte store)
                reinterpret_cast<uint4*>(A.wseq)[A.evoff[j] + s - 1u] = make_uint4(__float_as_uint(w), v, r[10 * C], 0u);
                if (w != 0.f) {
                    atomicAdd(A.wbuf + j, (double)w);
                    // S_j = sum_{s >= j} w_s vanishes past the photon's last event with w_s != 0,
                    // so pass 2 stops there (its list and its walks use this in place of the count)
                    atomicMax(A.nevbuf + j, s);
                }
            }
        }
    }
    stored = warp_sumu(stored);
    if ((threadIdx.x & 31u) == 0u && stored) atomicAdd(A.stats + MST_ST_EVENTS_STORED, (double)stored);
}

template <bool TWO>
__global__ void __launch_bounds__(kTB) k_event_adjoint(const TransportArgs A) {
    event_adjoint_run<TWO>(A);
}

// the batched form: the scenes of a table one after the other (block-uniform)
template <bool TWO>
__global__ void __launch_bounds__(kTB) k_event_adjoint_batch(const TransportArgs* __restrict__ scenes, int n_scenes) {
    for (int s = 0; s < n_scenes; ++s) {
        event_adjoint_run<TWO>(scenes[s]);
        __syncthreads();
    }
}

// Exclusive prefix sum of the photons' event counts (three passes over tiles of kScanTile):
// photon j's steps go to wseq[evoff[j] + s - 1], so pass 2 reads each photon's in event order.
constexpr int kScanPer = 16;                 // consecutive counts per thread
constexpr int kScanTile = kTB * kScanPer;    // counts per block

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t& total) {
    __shared__ uint32_t wsum[kTB / 32 + 1];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, incl, o);
        if (lane >= (unsigned)o) incl += u;
    }
    if (lane == 31u) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = lane < kTB / 32 ? wsum[lane] : 0u;
        uint32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(kFull, xi, o);
            if (lane >= (unsigned)o) xi += u;
        }
        if (lane < kTB / 32) wsum[lane] = xi - x;  // exclusive offset of each warp
        if (lane == 31u) wsum[kTB / 32] = xi;      // block total
    }
    __syncthreads();
    total = wsum[kTB / 32];
    return wsum[warp] + incl - v;
}

// A thread's kScanPer consecutive counts: four 16-byte loads when all lie below n (lo is a
// multiple of 16 counts, the array 16-byte aligned), else one by one.
__device__ __forceinline__ void load_counts(const uint32_t* __restrict__ x, uint32_t n, uint32_t lo,
                                            uint32_t (&v)[kScanPer]) {
    static_assert(kScanPer == 16, "four uint4 per thread");
    if (lo + kScanPer <= n) {
        const uint4* p = reinterpret_cast<const uint4*>(x + lo);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 u = __ldg(p + q);
            v[4 * q] = u.x;
            v[4 * q + 1] = u.y;
            v[4 * q + 2] = u.z;
            v[4 * q + 3] = u.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < kScanPer; ++q) v[q] = lo + q < n ? x[lo + q] : 0u;
    }
}

__global__ void __launch_bounds__(kTB) k_scan_tiles(const uint32_t* __restrict__ x, uint32_t n,
                                                    uint32_t* __restrict__ tsum) {
    const uint32_t lo = blockIdx.x * (uint32_t)kScanTile + threadIdx.x * kScanPer;
    uint32_t c[kScanPer];
    load_counts(x, n, lo, c);
    uint32_t v = 0u;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) v += c[q];
    uint32_t total = 0u;
    block_exclusive_scan(v, total);
    if (threadIdx.x == 0) tsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t* __restrict__ tsum, uint32_t nt) {
    // one block: exclusive scan of the tile sums in place, ceil(nt / 1024) consecutive per thread
    __shared__ uint32_t wsum[32];
    const uint32_t per = (nt + 1023u) / 1024u, lo = threadIdx.x * per;
    uint32_t v = 0u;
    for (uint32_t q = 0; q < per; ++q)
        if (lo + q < nt) v += tsum[lo + q];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, incl, o);
        if (lane >= (unsigned)o) incl += u;
    }
    if (lane == 31u) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = wsum[lane];
        uint32_t xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(kFull, xi, o);
            if (lane >= (unsigned)o) xi += u;
        }
        wsum[lane] = xi - x;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - v;
    for (uint32_t q = 0; q < per; ++q)
        if (lo + q < nt) {
            const uint32_t t = tsum[lo + q];
            tsum[lo + q] = run;
            run += t;
        }
}

__global__ void __launch_bounds__(kTB) k_scan_apply(const uint32_t* __restrict__ x, uint32_t n,
                                                    const uint32_t* __restrict__ tsum, uint32_t* __restrict__ out) {
    const uint32_t lo = blockIdx.x * (uint32_t)kScanTile + threadIdx.x * kScanPer;
    uint32_t v[kScanPer], sum = 0u;
    load_counts(x, n, lo, v);
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) sum += v[q];
    uint32_t total = 0u;
    uint32_t run = tsum[blockIdx.x] + block_exclusive_scan(sum, total);
    if (lo + kScanPer <= n) {  // four 16-byte stores
        uint4* o = reinterpret_cast<uint4*>(out + lo);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint4 u;
            u.x = run;
            run += v[4 * q];
            u.y = run;
            run += v[4 * q + 1];
            u.z = run;
            run += v[4 * q + 2];
            u.w = run;
            run += v[4 * q + 3];
            o[q] = u;
        }
    } else {
#pragma unroll
        for (int q = 0; q < kScanPer; ++q)
            if (lo + q < n) {
                out[lo + q] = run;
                run += v[q];
            }
    }
}

// Pass-2 work list. Photons with W != 0 are binned by their pass-1 event count (the last bin
// takes every count >= kScoreBins - 1) and listed from the highest bin down, so the longest
// replays start first and the launch does not end on a tail of long photons.
__device__ __forceinline__ int score_bin(uint32_t nev) { return (int)min(nev, (uint32_t)(kScoreBins - 1)); }

// Step 1: bin counts cnt[b] over the chunk.
__global__ void __launch_bounds__(kTB) k_score_hist(const double* __restrict__ W, const uint32_t* __restrict__ nev,
                                                    uint32_t n, unsigned* __restrict__ cnt) {
    __shared__ unsigned h[kScoreBins];
    for (int b = threadIdx.x; b < kScoreBins; b += kTB) h[b] = 0u;
    __syncthreads();
    const uint32_t lo = blockIdx.x * kScoreTile, hi = min(lo + (uint32_t)kScoreTile, n);
    for (uint32_t i = lo + threadIdx.x; i < hi; i += kTB) {
        const uint32_t e = nev[i];
        if (e != 0u && W[i] != 0.0) atomicAdd(&h[score_bin(e)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kScoreBins; b += kTB)
        if (h[b]) atomicAdd(&cnt[b], h[b]);
}

// Step 2: each tile reserves its slots in every bin (fill[b]) and writes its records there;
// the list length goes to *total.
__global__ void __launch_bounds__(kTB) k_score_scatter(const double* __restrict__ W, const uint32_t* __restrict__ nev,
                                                       uint32_t n, const unsigned* __restrict__ cnt,
                                                       unsigned* __restrict__ fill, unsigned* __restrict__ total,
                                                       ScoreRec* __restrict__ list) {
    __shared__ unsigned h[kScoreBins], pos[kScoreBins];
    for (int b = threadIdx.x; b < kScoreBins; b += kTB) h[b] = 0u;
    __syncthreads();
    const uint32_t lo = blockIdx.x * kScoreTile, hi = min(lo + (uint32_t)kScoreTile, n);
    for (uint32_t i = lo + threadIdx.x; i < hi; i += kTB) {
        const uint32_t e = nev[i];
        if (e != 0u && W[i] != 0.0) atomicAdd(&h[score_bin(e)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // bin starts, highest bin first: start[b] = sum_{b' > b} cnt[b']
        unsigned run = 0u;
        for (int b0 = kScoreBins - 32; b0 >= 0; b0 -= 32) {
            const int b = b0 + (int)threadIdx.x;
            const unsigned c = cnt[b];
            unsigned incl = c;  // suffix sum within the 32 bins b0 .. b0+31
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_down_sync(kFull, incl, o);
                if ((int)threadIdx.x + o < 32) incl += v;
            }
            const unsigned start = run + incl - c;
            pos[b] = h[b] ? start + atomicAdd(&fill[b], h[b]) : 0u;
            run += __shfl_sync(kFull, incl, 0);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) *total = run;
    }
    __syncthreads();
    for (uint32_t i = lo + threadIdx.x; i < hi; i += kTB) {
        const uint32_t e = nev[i];
        const double w = W[i];
        if (e != 0u && w != 0.0) {
            ScoreRec r;
            r.pid = i;
            r.nev = e;
            r.W = w;
            list[atomicAdd(&pos[score_bin(e)], 1u)] = r;
        }
    }
}

// Folds the FP32 chunk tiles into the FP64 results and clears them.
__global__ void k_fold_L(float* __restrict__ Lacc, double* __restrict__ L64, int nvox, int C, int cp) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nvox; k += gridDim.x * blockDim.x) {
        float* row = Lacc + (size_t)k * cp;
        for (int c = 0; c < C; ++c) {
            const float v = row[c];
            if (v != 0.f) {
                L64[(size_t)c * nvox + k] += (double)v;
                row[c] = 0.f;
            }
        }
    }
}

// the gradient tile is padded like the grid the flights walk; its halo receives nothing in valid
// use, and what a replay that left the forward's path added there is dropped
__global__ void k_fold_grad(float* __restrict__ gacc, double* __restrict__ g64, const Geo g) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.npad; q += gridDim.x * blockDim.x) {
        const float v = gacc[q];
        if (v != 0.f) {
            int k;
            if (interior_lin(g, q, k)) g64[k] += (double)v;
            gacc[q] = 0.f;
        }
    }
}

// dynamic shared memory of a transport block: the warps' photon stacks, the forward's tallies
// and the classic estimate's scratch
template <int MODE>
constexpr size_t smem_bytes() {
    constexpr bool REPLAY = MODE >= 2;
    constexpr bool CLASSIC = MODE == kFwdClassic || MODE == kPass1C || MODE == kPass2C;
    return (size_t)(kTB / 32) * Rec<REPLAY>::NW * kSlots * sizeof(uint32_t) +
           (REPLAY ? 0 : (size_t)kTB * 15 * sizeof(uint32_t)) +
           (CLASSIC ? (size_t)(kTB / 32) * kClassicWords * sizeof(uint32_t) : 0);
}

template <typename K>
int occupancy(K kern, size_t smem) {
    int n = 0;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    {   // shared-memory carveout: enough for three blocks (the register budget allows no more), the
        // rest of the SM's 256 KB to L1, which caches the extinction grid the walks fetch
        const size_t need = 3 * (smem + 1024);
        const int pct = (int)std::min<size_t>(100, (need * 100 + 228 * 1024 - 1) / (228 * 1024));
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kTB, smem) != cudaSuccess || n < 1) n = 1;
    return n;
}

template <int DT, int MODE, bool TWO, int TRIP = 0>
cudaError_t launch_mode(const TransportArgs& a, int blocks, cudaStream_t st) {
    if constexpr (TRIP != 0) {  // a variant of the autotuner: the default's carveout (set by occupancy())
        static const int once = occupancy(k_transport<DT, MODE, TWO, TRIP>, smem_bytes<MODE>());
        (void)once;
    }
    k_transport<DT, MODE, TWO, TRIP><<<blocks, kTB, smem_bytes<MODE>(), st>>>(a);
    return cudaGetLastError();
}

// Trip-length variants of the FP32-grid forward and pass-2 kernels, for the autotuner
// (kForwardTrips / kReplayTrips; the defaults are the un-suffixed kernels).
template <int MODE, bool TWO>
cudaError_t launch_trip(const TransportArgs& a, int trip, int blocks, cudaStream_t st) {
    if constexpr (MODE == kFwdVoxel) {
        switch (trip) {
            case 8: return launch_mode<0, MODE, TWO, 8>(a, blocks, st);
            case 10: return launch_mode<0, MODE, TWO, 10>(a, blocks, st);
            case 16: return launch_mode<0, MODE, TWO, 16>(a, blocks, st);
            default: return launch_mode<0, MODE, TWO>(a, blocks, st);
        }
    } else {
        switch (trip) {
            case 4: return launch_mode<0, MODE, TWO, 4>(a, blocks, st);
            case 8: return launch_mode<0, MODE, TWO, 8>(a, blocks, st);
            case 10: return launch_mode<0, MODE, TWO, 10>(a, blocks, st);
            default: return launch_mode<0, MODE, TWO>(a, blocks, st);
        }
    }
}

template <int DT, bool TWO>
int occupancy_mode(int mode) {
    switch (mode) {
        case kFwdVoxel: return occupancy(k_transport<DT, kFwdVoxel, TWO>, smem_bytes<kFwdVoxel>());
        case kFwdClassic: return occupancy(k_transport<DT, kFwdClassic, TWO>, smem_bytes<kFwdClassic>());
        case kPass2: return occupancy(k_transport<DT, kPass2, TWO>, smem_bytes<kPass2>());
        case kPass2W: return occupancy(k_transport<DT, kPass2W, TWO>, smem_bytes<kPass2W>());
        case kPass1C: return occupancy(k_transport<DT, kPass1C, TWO>, smem_bytes<kPass1C>());
        case kPass2C: return occupancy(k_transport<DT, kPass2C, TWO>, smem_bytes<kPass2C>());
        default: return occupancy(k_transport<DT, kPass1, TWO>, smem_bytes<kPass1>());
    }
}

template <int DT, bool TWO>
cudaError_t launch_dt(const TransportArgs& a, int mode, int trip, int blocks, cudaStream_t st) {
    if constexpr (DT == 0) {
        if (trip > 0 && mode == kFwdVoxel) return launch_trip<kFwdVoxel, TWO>(a, trip, blocks, st);
        if (trip > 0 && mode == kPass2W) return launch_trip<kPass2W, TWO>(a, trip, blocks, st);
        if (trip > 0 && mode == kPass2) return launch_trip<kPass2, TWO>(a, trip, blocks, st);
    }
    switch (mode) {
        case kFwdVoxel: return launch_mode<DT, kFwdVoxel, TWO>(a, blocks, st);
        case kFwdClassic: return launch_mode<DT, kFwdClassic, TWO>(a, blocks, st);
        case kPass2: return launch_mode<DT, kPass2, TWO>(a, blocks, st);
        case kPass2W: return launch_mode<DT, kPass2W, TWO>(a, blocks, st);
        case kPass1C: return launch_mode<DT, kPass1C, TWO>(a, blocks, st);
        case kPass2C: return launch_mode<DT, kPass2C, TWO>(a, blocks, st);
        default: return launch_mode<DT, kPass1, TWO>(a, blocks, st);
    }
}

template <bool TWO>
cudaError_t launch_species(const TransportArgs& a, int dtype, int mode, int trip, int blocks, cudaStream_t st) {
    return dtype == 0 ? launch_dt<0, TWO>(a, mode, trip, blocks, st)
                      : (dtype == 1 ? launch_dt<1, TWO>(a, mode, trip, blocks, st)
                                    : launch_dt<2, TWO>(a, mode, trip, blocks, st));
}

// The batched form: FP32 grid, one species, the modes of the full gradient with stored events.
// Function attributes (shared memory, carveout) are set by batch_occupancy() before any launch,
// outside a stream capture.
template <int MODE, int TRIP = 0>
cudaError_t launch_batch_mode(const TransportArgs* table, int n, int blocks, cudaStream_t st) {
    k_transport_batch<0, MODE, false, TRIP><<<blocks, kTB, smem_bytes<MODE>(), st>>>(table, n);
    return cudaGetLastError();
}

template <int MODE, int TRIP = 0>
int batch_occupancy() {
    return occupancy(k_transport_batch<0, MODE, false, TRIP>, smem_bytes<MODE>());
}

}  // namespace

cudaError_t launch_transport_batch(const TransportArgs* table, int n, int mode, int trip, int blocks,
                                   cudaStream_t st) {
    switch (mode) {
        case kFwdVoxel:
            switch (trip) {
                case 8: return launch_batch_mode<kFwdVoxel, 8>(table, n, blocks, st);
                case 10: return launch_batch_mode<kFwdVoxel, 10>(table, n, blocks, st);
                case 16: return launch_batch_mode<kFwdVoxel, 16>(table, n, blocks, st);
                default: return launch_batch_mode<kFwdVoxel>(table, n, blocks, st);
            }
        case kPass2W:
            switch (trip) {
                case 4: return launch_batch_mode<kPass2W, 4>(table, n, blocks, st);
                case 8: return launch_batch_mode<kPass2W, 8>(table, n, blocks, st);
                case 10: return launch_batch_mode<kPass2W, 10>(table, n, blocks, st);
                default: return launch_batch_mode<kPass2W>(table, n, blocks, st);
            }
        case kPass2: return launch_batch_mode<kPass2>(table, n, blocks, st);
        case kPass1: return launch_batch_mode<kPass1>(table, n, blocks, st);
        default: return cudaErrorInvalidValue;
    }
}

int transport_batch_blocks_per_sm(int mode) {
    static int occ[7] = {0, 0, 0, 0, 0, 0, 0};
    static bool ready = false;
    if (!ready) {  // every instantiation's attributes, once; the default trips give the occupancy
        occ[kFwdVoxel] = batch_occupancy<kFwdVoxel>();
        batch_occupancy<kFwdVoxel, 8>();
        batch_occupancy<kFwdVoxel, 10>();
        batch_occupancy<kFwdVoxel, 16>();
        occ[kPass2W] = batch_occupancy<kPass2W>();
        batch_occupancy<kPass2W, 4>();
        batch_occupancy<kPass2W, 8>();
        batch_occupancy<kPass2W, 10>();
        occ[kPass2] = batch_occupancy<kPass2>();
        occ[kPass1] = batch_occupancy<kPass1>();
        ready = true;
    }
    return mode >= 0 && mode < 7 && occ[mode] > 0 ? occ[mode] : 1;
}

cudaError_t launch_event_adjoint_batch(const TransportArgs* table, int n, int blocks, cudaStream_t st) {
    k_event_adjoint_batch<false><<<blocks, kTB, 0, st>>>(table, n);
    return cudaGetLastError();
}

int transport_blocks_per_sm(int dtype, int mode, bool two) {
    static int cache[2][3][7] = {{{0}}};
    int& c = cache[two ? 1 : 0][dtype][mode];
    if (c) return c;
    if (two)
        c = dtype == 0 ? occupancy_mode<0, true>(mode)
                       : (dtype == 1 ? occupancy_mode<1, true>(mode) : occupancy_mode<2, true>(mode));
    else
        c = dtype == 0 ? occupancy_mode<0, false>(mode)
                       : (dtype == 1 ? occupancy_mode<1, false>(mode) : occupancy_mode<2, false>(mode));
    return c;
}

cudaError_t launch_transport(const mst_grid* g, const TransportArgs& a, int dtype, int mode, int blocks,
                             cudaStream_t st) {
    const int trip = g->wf_trip[mode];  // the handle's wavefront setting (0: the kernel's default)
    return a.beta_air ? launch_species<true>(a, dtype, mode, trip, blocks, st)
                      : launch_species<false>(a, dtype, mode, trip, blocks, st);
}

cudaError_t launch_score_list(const mst_grid* g, uint32_t n, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(g->score_cnt, 0, sizeof(unsigned) * (2 * kScoreBins + 1), st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (n + kScoreTile - 1) / kScoreTile;
    if (blocks == 0u) return cudaSuccess;
    k_score_hist<<<blocks, kTB, 0, st>>>(g->wbuf, g->nevbuf, n, g->score_cnt);
    k_score_scatter<<<blocks, kTB, 0, st>>>(g->wbuf, g->nevbuf, n, g->score_cnt, g->score_cnt + kScoreBins,
                                            g->score_cnt + 2 * kScoreBins, g->plist);
    return cudaGetLastError();
}

cudaError_t launch_event_adjoint(const mst_grid* g, const TransportArgs& a, int dtype, cudaStream_t st) {
    (void)dtype;
    if (a.beta_air) k_event_adjoint<true><<<g->sm_count * 8, kTB, 0, st>>>(a);
    else k_event_adjoint<false><<<g->sm_count * 8, kTB, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_event_offsets(const mst_grid* g, uint32_t n, cudaStream_t st) {
    const uint32_t nt = (n + kScanTile - 1) / kScanTile;
    if (nt == 0u) return cudaSuccess;
    if (nt > 1024u * 64u) return cudaErrorInvalidValue;  // 2^28 photons; calls that store events hold 2^27
    uint32_t* tsum = reinterpret_cast<uint32_t*>(g->plist);  // the list is built after the offsets are used
    k_scan_tiles<<<nt, kTB, 0, st>>>(g->nevbuf, n, tsum);
    k_scan_top<<<1, 1024, 0, st>>>(tsum, nt);
    k_scan_apply<<<nt, kTB, 0, st>>>(g->nevbuf, n, tsum, g->evoff);
    return cudaGetLastError();
}

cudaError_t launch_fold_L(const mst_grid* g, cudaStream_t st) {
    const int nb = (g->geo.nvox + 255) / 256;
    k_fold_L<<<nb < 4096 ? nb : 4096, 256, 0, st>>>(g->Lacc, g->L64, g->geo.nvox, g->n_cams, g->cp);
    return cudaGetLastError();
}

cudaError_t launch_fold_grad(const mst_grid* g, cudaStream_t st) {
    const int nb = (g->geo.npad + 255) / 256;
    k_fold_grad<<<nb < 4096 ? nb : 4096, 256, 0, st>>>(g->gacc, g->g64, g->geo);
    return cudaGetLastError();
}

}  // namespace mst

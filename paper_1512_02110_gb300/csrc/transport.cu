// Photon transport on the GPU: the forward MC life cycle (Sec. 2.1.2, steps i-vi) with the
// voxelised local estimate of Eq. Lcupdate (or the classic one of Eq. fle), and the replay
// adjoint that re-walks every photon from its Philox key to scatter the score-function
// gradient of L (no path is stored).
//
// Work distribution: a persistent grid sized to the SM count. Each lane owns one photon at a
// time and advances it one free flight plus one event per loop trip; lanes whose photon has
// ended take a new photon id from a warp-local pool that lane 0 refills from a global ticket,
// so the warp stays full until the chunk runs dry.
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
    uint32_t hash;
    uint64_t id;     // global photon id (Philox counter)
    uint32_t idx;    // call-relative index (hash / skip arrays)
};

struct Tally {
    float esc[6];
    float absorbed, killed, gained, forced, launched;
    unsigned long long events, segments, scatters;
    unsigned int capped, escaped, traced, lost;
};

__device__ __forceinline__ void tally_zero(Tally& t) {
#pragma unroll
    for (int q = 0; q < 6; ++q) t.esc[q] = 0.f;
    t.absorbed = t.killed = t.gained = t.forced = t.launched = 0.f;
    t.events = t.segments = t.scatters = 0ull;
    t.capped = t.escaped = t.traced = t.lost = 0u;
}

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

// steps ii-iii: free flight of optical depth ph.tau (Eq. MCextinct). Returns -1 on a collision
// (ph.p and the voxel updated) or the exit face 0..5 (kWalkOverflow if the walk was abandoned).
// With S != 0 it also scatters the score of this flight into the gradient tile: -S * length in
// every voxel crossed and S * (1/beta - length) in the collision voxel.
template <int DT>
__device__ __forceinline__ int flight(const TransportArgs& A, Photon& ph, unsigned long long& nseg,
                                      unsigned long long& nsc, float S) {
    Walk w;
    walk_init(w, A.g, ph.p, ph.d, ph.ix, ph.iy, ph.iz);
    float tau = ph.tau;
    for (;;) {
        const float b = BetaFetch<DT>::get(A.beta, brick_addr(A.g, w.ix, w.iy, w.iz));
        ++nseg;
        float seg;
        const int a = walk_axis(w, seg);
        const float bs = b * seg;
        if (tau <= bs) {
            const float l = tau / b;
            ph.p = walk_local(w, A.g, l);
            ph.ix = w.ix;
            ph.iy = w.iy;
            ph.iz = w.iz;
            if (S != 0.f) {
                atomicAdd(A.gacc + lin_index(A.g, w.ix, w.iy, w.iz), S * (1.f / b - l));
                ++nsc;
            }
            return -1;
        }
        if (S != 0.f && seg > 0.f) {
            atomicAdd(A.gacc + lin_index(A.g, w.ix, w.iy, w.iz), -S * seg);
            ++nsc;
        }
        tau -= bs;
        const int f = walk_step(w, A.g, a, seg);
        if (f >= 0) return f;
    }
}

// cosine between the photon direction and the direction from the photon to camera c, and the
// squared distance; r2 = 0 when the photon sits on the centre of projection
__device__ __forceinline__ float cam_cosine(const TransportArgs& A, const Photon& ph, const Cam& cm, float& r2) {
    const float3 v = local_delta(A.g, ph.ix, ph.iy, ph.iz, ph.p, cm.ix, cm.iy, cm.iz, make_float3(cm.lx, cm.ly, cm.lz));
    r2 = v.x * v.x + v.y * v.y + v.z * v.z;
    return r2 > 0.f ? (ph.d.x * v.x + ph.d.y * v.y + ph.d.z * v.z) * rsqrtf(r2) : 0.f;
}

// Eq. Lcupdate: L_c(k) += albedo I_s P(angle between the incoming ray and X_c - X_s), for all
// cameras at once, four cameras per vector atomic into the [nvox][cp] FP32 tile.
__device__ __forceinline__ void le_voxel(const TransportArgs& A, const Photon& ph, float w, int k) {
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
                if (r2 > 0.f) val = w * hg_phase(A.hg, mu);
            }
            v[j] = val;
        }
        atomicAdd(reinterpret_cast<float4*>(row + c0), make_float4(v[0], v[1], v[2], v[3]));
    }
}

// w_s = sum_c a_c(k) albedo I_s P_c(s): the event's contribution to <a, L>.
__device__ __forceinline__ float le_adjoint(const TransportArgs& A, const Photon& ph, float w, int k) {
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
                if (r2 > 0.f) acc += aa[j] * w * hg_phase(A.hg, mu);
            }
        }
    }
    return acc;
}

// Eq. fle: pixel p(X_s) of camera c += albedo I_s P t_{s->c} / (|V|^2 Omega_p)
template <int DT>
__device__ __forceinline__ void le_classic(const TransportArgs& A, const Photon& ph, float w) {
    for (int c = 0; c < A.cams.n; ++c) {
        const Cam& cm = A.cams.c[c];
        // point relative to the camera
        const float3 v = local_delta(A.g, cm.ix, cm.iy, cm.iz, make_float3(cm.lx, cm.ly, cm.lz), ph.ix, ph.iy, ph.iz,
                                     ph.p);
        const float zc = v.x * cm.fx + v.y * cm.fy + v.z * cm.fz;
        if (!(zc > 0.f)) continue;
        const float x = (v.x * cm.rx + v.y * cm.ry + v.z * cm.rz) / zc;
        const float y = (v.x * cm.ux + v.y * cm.uy + v.z * cm.uz) / zc;
        const float px = floorf((x / cm.tx + 1.f) * 0.5f * (float)cm.w);
        const float py = floorf((y / cm.ty + 1.f) * 0.5f * (float)cm.h);
        if (px < 0.f || py < 0.f || px >= (float)cm.w || py >= (float)cm.h) continue;
        const int gp = cm.pix_off + (int)py * cm.w + (int)px;
        const float r2 = v.x * v.x + v.y * v.y + v.z * v.z;
        if (!(r2 > 0.f)) continue;
        const float mu = -(ph.d.x * v.x + ph.d.y * v.y + ph.d.z * v.z) * rsqrtf(r2);
        float tau = 0.f;
        unsigned long long ns = 0;
        walk_to_camera(A.g, cm, ph.ix, ph.iy, ph.iz, ph.p, [&](int jx, int jy, int jz, float len) {
            tau += BetaFetch<DT>::get(A.beta, brick_addr(A.g, jx, jy, jz)) * len;
        }, ns);
        const float val = w * hg_phase(A.hg, mu) * expf(-tau) / (r2 * A.omega[gp]);
        atomicAdd(A.cimg + gp, (double)val);
    }
}

// step v (albedo weighting, Russian roulette) and step vi (HG direction, next free path).
// Returns 0 to continue or the termination code.
__device__ __forceinline__ int after_event(const TransportArgs& A, Photon& ph, Tally& t) {
    t.absorbed += (1.f - A.albedo) * ph.I;
    ph.I *= A.albedo;
    if (ph.I == 0.f) return 2;
    if (A.max_order > 0 && (int)ph.s >= A.max_order) {
        t.forced += ph.I;
        return 4;
    }
    if ((int)ph.s >= A.max_events) {
        t.forced += ph.I;
        t.capped += 1u;
        return 5;
    }
    const float4 u = draws(A.key, ph.id, ph.s);
    if (ph.I < A.rr_below) {
        if (u.z < A.rr_survival) {
            t.gained += ph.I * (A.inv_rr_survival - 1.f);
            ph.I *= A.inv_rr_survival;
        } else {
            t.killed += ph.I;
            return 3;
        }
    }
    float ct, st;
    hg_sample(A.hg, u.x, ct, st);
    ph.d = rotate_dir(ph.d, ct, st, u.y);
    ph.tau = -logf(1.f - u.w);
    return 0;
}

__device__ __forceinline__ void finish_photon(const TransportArgs& A, Photon& ph, int term) {
    uint32_t h = (ph.hash ^ ph.s) * kFnvPrime;
    h = (h ^ (uint32_t)term) * kFnvPrime;
    if (A.hash) A.hash[ph.idx] = h;
}

// Warp-uniform refill: lanes without a photon take the next ids of the warp's pool.
// Returns false once the pool is dry and no lane holds a photon.
template <typename LaunchFn>
__device__ __forceinline__ void refill(const TransportArgs& A, bool& alive, bool& dry, uint32_t& wbase, uint32_t& wend,
                                       unsigned lane, LaunchFn&& on_launch) {
    unsigned need = __ballot_sync(kFull, !alive);
    while (need != 0u && !dry) {
        if (wbase >= wend) {
            unsigned t0 = 0u;
            if (lane == 0u) t0 = atomicAdd(A.ticket, (unsigned)kTicketBatch);
            t0 = __shfl_sync(kFull, t0, 0);
            if (t0 >= A.n) {
                dry = true;
                break;
            }
            wbase = t0;
            wend = min(t0 + (unsigned)kTicketBatch, A.n);
        }
        const unsigned rank = __popc(need & ((1u << lane) - 1u));
        const unsigned avail = wend - wbase;
        if (!alive && rank < avail) {
            const uint32_t pid = wbase + rank;
            if (A.skip && A.skip[A.out_base + pid]) {
                if (A.hash) A.hash[A.out_base + pid] = 0u;
            } else {
                on_launch(pid);
                alive = true;
            }
        }
        wbase += min((unsigned)__popc(need), avail);
        need = __ballot_sync(kFull, !alive);
    }
}

__device__ __forceinline__ void flush_tally(const TransportArgs& A, const Tally& t, unsigned lane) {
    double v[11];
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = warp_sum((double)t.esc[q]);
    v[6] = warp_sum((double)t.absorbed);
    v[7] = warp_sum((double)t.killed);
    v[8] = warp_sum((double)t.gained);
    v[9] = warp_sum((double)t.forced);
    v[10] = warp_sum((double)t.launched);
    const unsigned long long ev = warp_sumu(t.events), sg = warp_sumu(t.segments);
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

// K1: forward transport. EST = 0 voxelised local estimate, 1 classic local estimate.
template <int DT, int EST>
__global__ void __launch_bounds__(kTB) k_transport(const TransportArgs A) {
    const unsigned lane = threadIdx.x & 31u;
    Photon ph;
    Tally t;
    tally_zero(t);
    bool alive = false, dry = false;
    uint32_t wbase = 0u, wend = 0u;
    for (;;) {
        refill(A, alive, dry, wbase, wend, lane, [&](uint32_t pid) {
            launch_photon(A, ph, pid);
            t.launched += A.I0;
            t.traced += 1u;
        });
        if (!__any_sync(kFull, alive)) break;
        if (!alive) continue;
        const int f = flight<DT>(A, ph, t.segments, t.scatters, 0.f);
        if (f >= 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q)
                if (q == f) t.esc[q] += ph.I;
            if (f == kWalkOverflow) t.lost += 1u;
            else t.escaped += 1u;
            finish_photon(A, ph, 1);
            alive = false;
            continue;
        }
        ph.s += 1u;
        const int k = lin_index(A.g, ph.ix, ph.iy, ph.iz);
        ph.hash = (ph.hash ^ (uint32_t)k) * kFnvPrime;
        t.events += 1ull;
        const float w = A.albedo * ph.I;
        if (EST == 0)
            le_voxel(A, ph, w, k);
        else
            le_classic<DT>(A, ph, w);
        const int term = after_event(A, ph, t);
        if (term) {
            finish_photon(A, ph, term);
            alive = false;
        }
    }
    flush_tally(A, t, lane);
}

// K6: replay adjoint. Pass 1 replays the photon and sums W = sum_s w_s; pass 2 replays it
// again and, with S_j = W - sum_{s<j} w_s (FP64), scatters the score of every flight that ends
// in an event. Both passes run the same flight / event code, so they see the same path.
template <int DT>
__global__ void __launch_bounds__(kTB) k_replay(const TransportArgs A) {
    const unsigned lane = threadIdx.x & 31u;
    Photon ph;
    Tally t;
    tally_zero(t);
    bool alive = false, dry = false;
    uint32_t wbase = 0u, wend = 0u;
    int phase = 1;
    double W = 0.0, S = 0.0;
    uint32_t nev = 0u;
    for (;;) {
        refill(A, alive, dry, wbase, wend, lane, [&](uint32_t pid) {
            launch_photon(A, ph, pid);
            phase = 1;
            W = 0.0;
            S = 0.0;
            nev = 0u;
        });
        if (!__any_sync(kFull, alive)) break;
        if (!alive) continue;
        const int f = flight<DT>(A, ph, t.segments, t.scatters, phase == 2 ? (float)S : 0.f);
        bool ended = false;
        if (f >= 0) {
            ended = true;
        } else {
            ph.s += 1u;
            t.events += 1ull;
            const int k = lin_index(A.g, ph.ix, ph.iy, ph.iz);
            const float w = le_adjoint(A, ph, A.albedo * ph.I, k);
            if (phase == 1)
                W += (double)w;
            else
                S -= (double)w;
            if (phase == 2 && ph.s == nev) {
                alive = false;
                continue;
            }
            ended = after_event(A, ph, t) != 0;
        }
        if (ended) {
            if (phase == 1 && W != 0.0 && ph.s > 0u) {
                nev = ph.s;
                const uint32_t pid = ph.idx - A.out_base;
                launch_photon(A, ph, pid);
                phase = 2;
                S = W;
            } else {
                alive = false;
            }
        }
    }
    const unsigned long long ev = warp_sumu(t.events), sg = warp_sumu(t.segments), sc = warp_sumu(t.scatters);
    if (lane == 0u) {
        atomicAdd(A.stats + MST_ST_REPLAY_EVENTS, (double)ev);
        atomicAdd(A.stats + MST_ST_REPLAY_SEGMENTS, (double)sg);
        atomicAdd(A.stats + MST_ST_REPLAY_SCATTERS, (double)sc);
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

__global__ void k_fold_grad(float* __restrict__ gacc, double* __restrict__ g64, int nvox) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nvox; k += gridDim.x * blockDim.x) {
        const float v = gacc[k];
        if (v != 0.f) {
            g64[k] += (double)v;
            gacc[k] = 0.f;
        }
    }
}

template <typename K>
int occupancy(K kern) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kTB, 0) != cudaSuccess || n < 1) n = 1;
    return n;
}

}  // namespace

int transport_blocks_per_sm(int dtype, int estimator, bool replay) {
    static int cache[3][3] = {{0}};
    const int col = replay ? 2 : estimator;
    if (cache[dtype][col]) return cache[dtype][col];
    int n = 1;
#define MST_OCC(DT)                                                   \
    if (dtype == DT) {                                                \
        if (replay) n = occupancy(k_replay<DT>);                      \
        else if (estimator == 0) n = occupancy(k_transport<DT, 0>);   \
        else n = occupancy(k_transport<DT, 1>);                       \
    }
    MST_OCC(0) MST_OCC(1) MST_OCC(2)
#undef MST_OCC
    cache[dtype][col] = n;
    return n;
}

cudaError_t launch_transport(const mst_grid* g, const TransportArgs& a, int dtype, int estimator, int blocks,
                             cudaStream_t st) {
    (void)g;
#define MST_TR(DT)                                                                   \
    if (dtype == DT) {                                                               \
        if (estimator == 0) k_transport<DT, 0><<<blocks, kTB, 0, st>>>(a);           \
        else k_transport<DT, 1><<<blocks, kTB, 0, st>>>(a);                          \
    }
    MST_TR(0) MST_TR(1) MST_TR(2)
#undef MST_TR
    return cudaGetLastError();
}

cudaError_t launch_replay(const mst_grid* g, const TransportArgs& a, int dtype, int blocks, cudaStream_t st) {
    (void)g;
    if (dtype == 0) k_replay<0><<<blocks, kTB, 0, st>>>(a);
    else if (dtype == 1) k_replay<1><<<blocks, kTB, 0, st>>>(a);
    else k_replay<2><<<blocks, kTB, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fold_L(const mst_grid* g, cudaStream_t st) {
    const int nb = (g->geo.nvox + 255) / 256;
    k_fold_L<<<nb < 4096 ? nb : 4096, 256, 0, st>>>(g->Lacc, g->L64, g->geo.nvox, g->n_cams, g->cp);
    return cudaGetLastError();
}

cudaError_t launch_fold_grad(const mst_grid* g, cudaStream_t st) {
    const int nb = (g->geo.nvox + 255) / 256;
    k_fold_grad<<<nb < 4096 ? nb : 4096, 256, 0, st>>>(g->gacc, g->g64, g->geo.nvox);
    return cudaGetLastError();
}

}  // namespace mst

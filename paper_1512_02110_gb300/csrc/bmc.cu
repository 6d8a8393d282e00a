// Backward Monte Carlo with the sun local estimate (Eq. ble): paths start at a camera, fly
// through the staged extinction grid by the voxel walk of the forward transport, and at every
// scattering event add the sun's single-scattered radiance toward the camera. The paper uses it
// to check the in-situ forward model (Sec. 3); here it renders whole images, one path per
// thread, every pixel on its own Philox stream (counter word 3 = 1 + global pixel index).
#include <cmath>

#include "mst_internal.h"

namespace mst {
namespace {

constexpr int kTB = 256;
constexpr int kBmcCollided = -2;

struct BmcArgs {
    Geo g;
    CamSet cams;
    HG hg;
    const void* beta;       // staged extinction [nvox]
    const float* omega;     // [total pix] pixel solid angles
    float3 to_sun;          // unit vector toward the sun
    float albedo, F;        // single-scattering albedo, sun irradiance
    float rr_below, rr_survival, inv_rr_survival;
    uint2 key;
    int max_order, max_events;
    uint32_t n;             // paths per pixel
    uint64_t total;         // total pixels x n
    double* sum;            // [total pix] sum of path values
    double* sum2;           // [total pix] sum of squared path values
    double* stats;          // [MST_NSTATS]
};

// One free flight from the walk's current point with optical depth tau: returns kBmcCollided
// with the collision point (voxel + offset) or the exit face.
template <int DT>
__device__ __forceinline__ int bmc_flight(const BmcArgs& A, Walk& w, float tau, float3& p, int& ix, int& iy, int& iz,
                                          unsigned& nseg) {
    for (;;) {
        const float b = BetaFetch<DT>::get(A.beta, w.lin);
        float seg;
        const int a = walk_axis(w, seg);
        ++nseg;
        const float bs = b * seg;
        if (tau <= bs) {
            p = walk_local(w, A.g, tau / b);
            ix = w.ix;
            iy = w.iy;
            iz = w.iz;
            return kBmcCollided;
        }
        tau -= bs;
        const int r = walk_step(w, A.g, a, seg);
        if (r >= 0) return r;
    }
}

// Optical depth from the point to the grid boundary along the sun-ward ray, and the exit face.
template <int DT>
__device__ __forceinline__ double sun_depth(const BmcArgs& A, float3 p, int ix, int iy, int iz, int& face,
                                            unsigned& nseg) {
    Walk w;
    walk_init(w, A.g, p, A.to_sun, ix, iy, iz);
    double tau = 0.0;
    for (;;) {
        const float b = BetaFetch<DT>::get(A.beta, w.lin);
        float seg;
        const int a = walk_axis(w, seg);
        ++nseg;
        tau += (double)(b * seg);
        const int r = walk_step(w, A.g, a, seg);
        if (r >= 0) {
            face = r;
            return tau;
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(kTB) k_bmc(const BmcArgs A) {
    unsigned paths = 0u, events = 0u, nseg = 0u;
    const uint64_t stride = (uint64_t)gridDim.x * kTB;
    for (uint64_t t = (uint64_t)blockIdx.x * kTB + threadIdx.x; t < A.total; t += stride) {
        const uint32_t gp = (uint32_t)(t / A.n), q = (uint32_t)(t - (uint64_t)gp * A.n);
        const int c = cam_of_pixel(A.cams, (int)gp);
        const Cam& cm = A.cams.c[c];
        const int li = (int)gp - cm.pix_off, i = li % cm.w, j = li / cm.w;
        float4 u = draws(A.key, q, 0u, 1u + gp);
        const float px = (float)i + u.x, py = (float)j + u.y;
        const float xx = (2.f * px / (float)cm.w - 1.f) * cm.tx, yy = (2.f * py / (float)cm.h - 1.f) * cm.ty;
        const float cosv = rsqrtf(1.f + xx * xx + yy * yy);
        const float apix = (2.f * cm.tx / (float)cm.w) * (2.f * cm.ty / (float)cm.h);
        const double wpix = (double)(cosv * cosv * cosv) * (double)apix / (double)A.omega[gp];
        float3 d = pixel_dir(cm, px, py);
        float3 p;
        int ix, iy, iz;
        double contrib = 0.0;
        ++paths;
        if (ray_start(A.g, cm, d, p, ix, iy, iz)) {
            float I = 1.f, tau = -logf(1.f - u.z);
            for (uint32_t ev = 1;; ++ev) {
                Walk w;
                walk_init(w, A.g, p, d, ix, iy, iz);
                if (bmc_flight<DT>(A, w, tau, p, ix, iy, iz, nseg) != kBmcCollided) break;
                ++events;
                int face = -1;
                const double ts = sun_depth<DT>(A, p, ix, iy, iz, face, nseg);
                if (face == 5) {  // the sun-ward ray leaves through the top face: sunlit
                    const float mu = d.x * A.to_sun.x + d.y * A.to_sun.y + d.z * A.to_sun.z;
                    contrib += (double)(A.albedo * I * hg_phase(A.hg, mu)) * exp(-ts) * (double)A.F;
                }
                I *= A.albedo;
                if (I == 0.f) break;
                if (A.max_order > 0 && (int)ev >= A.max_order) break;
                if ((int)ev >= A.max_events) break;
                u = draws(A.key, q, ev, 1u + gp);
                if (I < A.rr_below) {
                    if (u.z < A.rr_survival) I *= A.inv_rr_survival;
                    else break;
                }
                float ct, st;
                hg_sample(A.hg, u.x, ct, st);
                d = rotate_dir(d, ct, st, u.y);
                tau = -logf(1.f - u.w);
            }
        }
        const double v = contrib * wpix;
        if (v != 0.0) {
            atomicAdd(A.sum + gp, v);
            atomicAdd(A.sum2 + gp, v * v);
        }
    }
    const unsigned long long np = warp_sumu(paths), ne = warp_sumu(events), ns = warp_sumu(nseg);
    if ((threadIdx.x & 31u) == 0u) {
        atomicAdd(A.stats + MST_ST_BMC_PATHS, (double)np);
        atomicAdd(A.stats + MST_ST_BMC_EVENTS, (double)ne);
        atomicAdd(A.stats + MST_ST_BMC_SEGMENTS, (double)ns);
    }
}

// Pixel means and the variance of each mean from the path sums.
__global__ void k_bmc_finish(double* __restrict__ mean, double* __restrict__ sum2, double* __restrict__ var,
                             int npix, uint32_t n) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npix; k += gridDim.x * blockDim.x) {
        const double m = mean[k] / n;
        mean[k] = m;
        if (var) var[k] = n > 1 ? (sum2[k] / n - m * m) / (double)(n - 1) : 0.0;
    }
}

}  // namespace

cudaError_t launch_bmc(const mst_grid* g, const mst_params* p, uint32_t n, double* sum, double* sum2, double* var,
                       cudaStream_t st) {
    BmcArgs a;
    a.g = g->geo;
    a.cams = g->cams;
    const double gg = p->g;
    a.hg.g = (float)gg;
    a.hg.k1 = (float)((1.0 - gg * gg) / (4.0 * M_PI));
    a.hg.a = (float)(1.0 + gg * gg);
    a.hg.b = (float)(2.0 * gg);
    a.hg.omg2 = (float)(1.0 - gg * gg);
    a.hg.omg = (float)(1.0 - gg);
    a.hg.opg = (float)(1.0 + gg);
    a.hg.tg = (float)(2.0 * gg);
    a.hg.iso = std::fabs(gg) < 1e-6;
    a.beta = g->ext;
    a.omega = g->omega;
    const double th = p->sun_zenith_rad, ph = p->sun_azimuth_rad;
    a.to_sun = make_float3((float)(std::sin(th) * std::cos(ph)), (float)(std::sin(th) * std::sin(ph)), (float)std::cos(th));
    a.albedo = (float)p->albedo;
    a.F = (float)p->sun_irradiance;
    a.rr_below = (float)p->rr_threshold;
    a.rr_survival = (float)p->rr_survival;
    a.inv_rr_survival = (float)(1.0 / p->rr_survival);
    a.key = make_uint2((uint32_t)p->seed, (uint32_t)(p->seed >> 32));
    a.max_order = p->max_order;
    a.max_events = p->max_events;
    a.n = n;
    a.total = (uint64_t)g->total_pix * n;
    a.sum = sum;
    a.sum2 = sum2;
    a.stats = g->stats;
    const int blocks = g->sm_count * 8;
    if (p->grid_dtype == 0) k_bmc<0><<<blocks, kTB, 0, st>>>(a);
    else if (p->grid_dtype == 1) k_bmc<1><<<blocks, kTB, 0, st>>>(a);
    else k_bmc<2><<<blocks, kTB, 0, st>>>(a);
    const int nb = (g->total_pix + kTB - 1) / kTB;
    k_bmc_finish<<<nb < 4096 ? nb : 4096, kTB, 0, st>>>(sum, sum2, var, g->total_pix, n);
    return cudaGetLastError();
}

}  // namespace mst

// Deterministic ray kernels of the voxelised model: grid staging, LOS transmittance
// (Eq. taoKtoc-Tck), pixel-ray image formation (Eq. Icpixel) with the loss epilogue
// (Eq. Cost), back-projection Pi^T, the LOS adjoint W^T, sub-pixel ray counts (Sec. 6),
// the gradient combinations of Eq. Jaco1-DivTc and the Laplacian regulariser.
//
// Geometry is never stored: every Pi_c and W_c product re-walks its rays through the grid.
// LOS threads run x-fastest over voxels of one camera, so a warp walks 32 nearly parallel
// rays toward the same X_c.
#include <cmath>

#include "mst_internal.h"

namespace mst {
namespace {

constexpr int kTB = 256;

// The extinction grid in the compute dtype, in the linear voxel order of the input.
template <int DT>
__global__ void k_stage(const float* __restrict__ beta, const float* __restrict__ air, void* __restrict__ ext,
                        float* __restrict__ tot, int nvox) {
    typedef typename BetaFetch<DT>::T T;
    T* out = static_cast<T*>(ext);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nvox; k += gridDim.x * blockDim.x) {
        const float b = air ? beta[k] + air[k] : beta[k];  // Sec. 2: beta = beta_aerosol + beta_air
        out[k] = BetaFetch<DT>::make(b);
        if (tot) tot[k] = b;  // two species: the FP32 total for the surrogate's j = L / beta
    }
}

// The grid of the photon flights: the same values on [nz + 4][ny + 4][nx + 4] with a halo of
// +inf extinction, where a flight stops (a free path never outlasts infinite optical depth).
template <int DT>
__global__ void k_stage_pad(const float* __restrict__ beta, const float* __restrict__ air, void* __restrict__ ext,
                            const Geo g) {
    typedef typename BetaFetch<DT>::T T;
    T* out = static_cast<T*>(ext);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.npad; q += gridDim.x * blockDim.x) {
        const int ix = q % g.p0 - kHalo, iy = (q / g.p0) % (g.ny + 2 * kHalo) - kHalo, iz = q / g.p01 - kHalo;
        float b = CUDART_INF_F;
        if (ix >= 0 && ix < g.nx && iy >= 0 && iy < g.ny && iz >= 0 && iz < g.nz) {
            const int k = lin_index(g, ix, iy, iz);
            b = air ? beta[k] + air[k] : beta[k];
        }
        out[q] = BetaFetch<DT>::make(b);
    }
}

// beta_ref + beta_air in FP32 (the surrogate's reference total)
__global__ void k_add_air(const float* __restrict__ beta, const float* __restrict__ air, float* __restrict__ out,
                          int nvox) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nvox; k += gridDim.x * blockDim.x) out[k] = beta[k] + air[k];
}

__device__ __forceinline__ void flush_count(double* stats, int slot, unsigned long long n) {
    n = warp_sumu(n);
    if ((threadIdx.x & 31u) == 0u && n) atomicAdd(stats + slot, (double)n);
}

// K2: tau_c(k) along the LOS from the centre of voxel k to X_c; T = exp(-tau). With L given,
// also R_c(k) = L_c(k) T_c(k) (Eq. Rck), where L = Lsrc * beta / beta_ref when beta_ref is
// given (the j-fixed surrogate, L = j beta with j = L_ref / beta_ref).
template <int DT>
__global__ void __launch_bounds__(kTB) k_los(const Geo g, const CamSet cs, const void* __restrict__ ext,
                                             const double* __restrict__ Lsrc, const float* __restrict__ beta_ref,
                                             const float* __restrict__ beta, float* __restrict__ T_out,
                                             float* __restrict__ R_out, double* stats) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)cs.n * g.nvox;
    unsigned long long nseg = 0;
    if (idx < total) {
        const int c = (int)(idx / g.nvox), k = (int)(idx - (long long)c * g.nvox);
        const int ix = k % g.nx, iy = (k / g.nx) % g.ny, iz = k / (g.nx * g.ny);
        double tau = 0.0;  // FP64 sum: ~1e-7 relative for optical depths up to ~100
        walk_to_camera(g, cs.c[c], ix, iy, iz, make_float3(0.5f * g.hx, 0.5f * g.hy, 0.5f * g.hz),
                       [&](const Walk& w, float len) { tau += (double)(BetaFetch<DT>::get(ext, w.lin) * len); },
                       nseg);
        const float T = (float)exp(-tau);
        if (T_out) T_out[idx] = T;
        if (R_out) {
            double L = Lsrc[idx];
            if (beta_ref) {
                const float br = beta_ref[k];
                L = br > 0.f ? L * (double)beta[k] / (double)br : 0.0;
            }
            R_out[idx] = (float)(L * (double)T);
        }
    }
    if (stats) flush_count(stats, MST_ST_LOS_SEGMENTS, nseg);
}

// K3: i_c(p) = 1/(N_rays V) sum_rho sum_k l(k) R_c(k) (Eq. Icpixel), FP64 per pixel. With
// measurements, also r = M (i - i_meas), resid = 2 r = dE/di, and E += r^2 (Eq. Cost).
__global__ void __launch_bounds__(kTB) k_images(const Geo g, const CamSet cs, const Halton hs, float inv_nv,
                                                const float* __restrict__ R, double* __restrict__ images,
                                                const double* __restrict__ meas, const uint8_t* __restrict__ mask,
                                                double* __restrict__ resid, double* loss, int total_pix,
                                                double* stats) {
    const int gp = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nseg = 0;
    double r2 = 0.0;
    if (gp < total_pix) {
        const int c = cam_of_pixel(cs, gp);
        const Cam& cm = cs.c[c];
        const int p = gp - cm.pix_off, i = p % cm.w, j = p / cm.w;
        const float* Rc = R + (size_t)c * g.nvox;
        double acc = 0.0;
        for (int rho = 0; rho < hs.n; ++rho) {
            const float3 d = pixel_dir(cm, (float)i + hs.a[rho], (float)j + hs.b[rho]);
            walk_from_camera(g, cm, d, [&](const Walk& w, float len) { acc += (double)(len * __ldg(Rc + w.lin)); },
                             nseg);
        }
        const double img = acc * (double)inv_nv;
        if (images) images[gp] = img;
        if (meas) {
            const double r = (mask && !mask[gp]) ? 0.0 : img - meas[gp];
            resid[gp] = 2.0 * r;
            r2 = r * r;
        }
    }
    if (meas) {
        r2 = warp_sum(r2);
        if ((threadIdx.x & 31u) == 0u && r2 != 0.0) atomicAdd(loss, r2);
    }
    if (stats) flush_count(stats, MST_ST_PIXEL_SEGMENTS, nseg);
}

// K4: b_c(k) = sum_p Pi_c(p, k) resid(p)  (Pi^T, Eq. PIc transposed)
__global__ void __launch_bounds__(kTB) k_backproject(const Geo g, const CamSet cs, const Halton hs, float inv_nv,
                                                     const double* __restrict__ resid, float* __restrict__ bacc,
                                                     int total_pix, double* stats) {
    const int gp = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nseg = 0;
    if (gp < total_pix) {
        const float wgt = (float)(resid[gp] * (double)inv_nv);
        if (wgt != 0.f) {
            const int c = cam_of_pixel(cs, gp);
            const Cam& cm = cs.c[c];
            const int p = gp - cm.pix_off, i = p % cm.w, j = p / cm.w;
            float* bc = bacc + (size_t)c * g.nvox;
            for (int rho = 0; rho < hs.n; ++rho) {
                const float3 d = pixel_dir(cm, (float)i + hs.a[rho], (float)j + hs.b[rho]);
                walk_from_camera(g, cm, d, [&](const Walk& w, float len) {
                    if (len > 0.f) atomicAdd(bc + w.lin, wgt * len);
                }, nseg);
            }
        }
    }
    if (stats) flush_count(stats, MST_ST_BACKPROJ_SEGMENTS, nseg);
}

// K5: gT_c(m) = sum_k W_c(k, m) s_c(k), s = R b = L T b (Eq. DivTc transposed)
__global__ void __launch_bounds__(kTB) k_los_adjoint(const Geo g, const CamSet cs, const float* __restrict__ R,
                                                     const float* __restrict__ bacc, float* __restrict__ gT,
                                                     double* stats) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)cs.n * g.nvox;
    unsigned long long nseg = 0;
    if (idx < total) {
        const float s = R[idx] * bacc[idx];
        if (s != 0.f) {
            const int c = (int)(idx / g.nvox), k = (int)(idx - (long long)c * g.nvox);
            const int ix = k % g.nx, iy = (k / g.nx) % g.ny, iz = k / (g.nx * g.ny);
            float* gc = gT + (size_t)c * g.nvox;
            walk_to_camera(g, cs.c[c], ix, iy, iz, make_float3(0.5f * g.hx, 0.5f * g.hy, 0.5f * g.hz),
                           [&](const Walk& w, float len) {
                               if (len > 0.f) atomicAdd(gc + w.lin, s * len);
                           },
                           nseg);
        }
    }
    if (stats) flush_count(stats, MST_ST_LOSADJ_SEGMENTS, nseg);
}

// Q_c(k): number of sub-pixel rays through voxel k; a ray counts when its chord is at least
// 1e-4 of the smallest voxel edge (grazing rays with chords ~ 0 are not counted)
__global__ void __launch_bounds__(kTB) k_ray_counts(const Geo g, const CamSet cs, const Halton hs, float* __restrict__ Q,
                                                    int total_pix) {
    const float eps = 1e-4f * fminf(g.hx, fminf(g.hy, g.hz));
    const int gp = blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= total_pix) return;
    const int c = cam_of_pixel(cs, gp);
    const Cam& cm = cs.c[c];
    const int p = gp - cm.pix_off, i = p % cm.w, j = p / cm.w;
    float* qc = Q + (size_t)c * g.nvox;
    unsigned long long nseg = 0;
    for (int rho = 0; rho < hs.n; ++rho) {
        const float3 d = pixel_dir(cm, (float)i + hs.a[rho], (float)j + hs.b[rho]);
        walk_from_camera(g, cm, d, [&](const Walk& w, float len) {
            if (len >= eps) atomicAdd(qc + w.lin, 1.f);
        }, nseg);
    }
}

// conditioning weight from counts: mode 1 -> 1 / max(1, Q), mode 2 -> Q
__global__ void k_qweights(float* Q, long long n, int mode) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Q[i] = mode == 1 ? 1.f / fmaxf(1.f, Q[i]) : Q[i];
}

// a_c(k) = T_c(k) b_c(k) in the [nvox][cp] layout gathered at photon events
__global__ void k_adjoint_tiles(const float* __restrict__ T, const float* __restrict__ bacc, float* __restrict__ adj,
                                int nvox, int C, int cp) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nvox; k += gridDim.x * blockDim.x)
        for (int c = 0; c < cp; ++c)
            adj[(size_t)k * cp + c] = c < C ? T[(size_t)c * nvox + k] * bacc[(size_t)c * nvox + k] : 0.f;
}

// surrogate: grad(m) = sum_c Q_c(m) [ j_c(m) T_c(m) b_c(m) - gT_c(m) ], j = Lsrc / beta_ref
__global__ void k_combine_surrogate(const double* __restrict__ Lsrc, const float* __restrict__ beta_ref,
                                    const float* __restrict__ T, const float* __restrict__ bacc,
                                    const float* __restrict__ gT, const float* __restrict__ Qw,
                                    double* __restrict__ grad, int nvox, int C) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nvox; k += gridDim.x * blockDim.x) {
        const float br = beta_ref[k];
        double acc = 0.0;
        for (int c = 0; c < C; ++c) {
            const size_t i = (size_t)c * nvox + k;
            const double j = br > 0.f ? Lsrc[i] / (double)br : 0.0;
            const double q = Qw ? (double)Qw[i] : 1.0;
            acc += q * (j * (double)T[i] * (double)bacc[i] - (double)gT[i]);
        }
        grad[k] = acc;
    }
}

// full: grad(m) = gL(m) - sum_c gT_c(m)
__global__ void k_combine_full(const float* __restrict__ gT, const double* __restrict__ gL, double* __restrict__ grad,
                               int nvox, int C) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nvox; k += gridDim.x * blockDim.x) {
        double acc = gL[k];
        if (gT)  // voxel estimator: the LOS term; the classic estimator has none
            for (int c = 0; c < C; ++c) acc -= (double)gT[(size_t)c * nvox + k];
        grad[k] = acc;
    }
}

// Loss of the classic images (Eq. Cost): r = M (i - i_meas), E += sum r^2, resid = dE/di = 2 r.
__global__ void k_classic_resid(const double* __restrict__ img, const double* __restrict__ meas,
                                const uint8_t* __restrict__ mask, double* __restrict__ resid, double* loss, int npix) {
    double e = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        const double r = (mask && !mask[p]) ? 0.0 : img[p] - meas[p];
        resid[p] = 2.0 * r;
        e += r * r;
    }
    e = warp_sum(e);
    if ((threadIdx.x & 31u) == 0u && e != 0.0) atomicAdd(loss, e);
}

// Laplacian of a dense field: out(k) = sum over in-grid 6-neighbours n of (x(n) - x(k))
template <typename TIn>
__device__ __forceinline__ double lap_at(const Geo& g, const TIn* x, int k) {
    const int ix = k % g.nx, iy = (k / g.nx) % g.ny, iz = k / (g.nx * g.ny);
    const double xk = (double)x[k];
    double acc = 0.0;
    if (ix > 0) acc += (double)x[k - 1] - xk;
    if (ix < g.nx - 1) acc += (double)x[k + 1] - xk;
    if (iy > 0) acc += (double)x[k - g.nx] - xk;
    if (iy < g.ny - 1) acc += (double)x[k + g.nx] - xk;
    if (iz > 0) acc += (double)x[k - g.nx * g.ny] - xk;
    if (iz < g.nz - 1) acc += (double)x[k + g.nx * g.ny] - xk;
    return acc;
}

// Psi = |W Lap beta|^2 (W diagonal by altitude: wz[iz], or 1 when wz is NULL); lap <- W^T W Lap beta
__global__ void k_lap1(const Geo g, const float* __restrict__ beta, const double* __restrict__ wz,
                       double* __restrict__ lap, double* psi) {
    double s = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.nvox; k += gridDim.x * blockDim.x) {
        const double w = wz ? wz[k / (g.nx * g.ny)] : 1.0;
        const double v = w * lap_at(g, beta, k);
        lap[k] = w * v;
        s += v * v;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31u) == 0u && s != 0.0) atomicAdd(psi, s);
}

__global__ void k_lap2(const Geo g, const double* __restrict__ lap, double eta, double* __restrict__ grad) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.nvox; k += gridDim.x * blockDim.x)
        grad[k] += eta * 2.0 * lap_at(g, lap, k);
}

__global__ void k_add_scaled(double* dst, const double* src, double eta) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst += eta * (*src);
}

inline int nblocks(long long n, int tb = kTB, int cap = 1 << 20) {
    const long long b = (n + tb - 1) / tb;
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

cudaError_t launch_stage(const mst_grid* g, const float* beta, const float* air, int dtype, cudaStream_t st) {
    const int nvox = g->geo.nvox;
    const int nb = nblocks(nvox, kTB, 8192);
    float* tot = air ? g->btot : nullptr;
    if (dtype == 0) k_stage<0><<<nb, kTB, 0, st>>>(beta, air, g->ext, tot, nvox);
    else if (dtype == 1) k_stage<1><<<nb, kTB, 0, st>>>(beta, air, g->ext, tot, nvox);
    else k_stage<2><<<nb, kTB, 0, st>>>(beta, air, g->ext, tot, nvox);
    if (g->ext_pad) {
        const int np = nblocks(g->geo.npad, kTB, 4096);
        if (dtype == 0) k_stage_pad<0><<<np, kTB, 0, st>>>(beta, air, g->ext_pad, g->geo);
        else if (dtype == 1) k_stage_pad<1><<<np, kTB, 0, st>>>(beta, air, g->ext_pad, g->geo);
        else k_stage_pad<2><<<np, kTB, 0, st>>>(beta, air, g->ext_pad, g->geo);
    }
    return cudaGetLastError();
}

cudaError_t launch_add_air(const mst_grid* g, const float* beta, const float* air, float* out, cudaStream_t st) {
    k_add_air<<<nblocks(g->geo.nvox, kTB, 4096), kTB, 0, st>>>(beta, air, out, g->geo.nvox);
    return cudaGetLastError();
}

cudaError_t launch_los(const mst_grid* g, int dtype, const double* L, const double* /*jfix*/, const float* beta_ref,
                       const float* beta, float* T_out, float* R_out, cudaStream_t st) {
    const long long total = (long long)g->n_cams * g->geo.nvox;
    const int nb = nblocks(total);
    if (dtype == 0) k_los<0><<<nb, kTB, 0, st>>>(g->geo, g->cams, g->ext, L, beta_ref, beta, T_out, R_out, g->stats);
    else if (dtype == 1) k_los<1><<<nb, kTB, 0, st>>>(g->geo, g->cams, g->ext, L, beta_ref, beta, T_out, R_out, g->stats);
    else k_los<2><<<nb, kTB, 0, st>>>(g->geo, g->cams, g->ext, L, beta_ref, beta, T_out, R_out, g->stats);
    return cudaGetLastError();
}

cudaError_t launch_images(const mst_grid* g, const float* R, double* images, const double* meas, const uint8_t* mask,
                          double* resid, double* loss, cudaStream_t st) {
    const float inv_nv = (float)(1.0 / (g->n_rays * g->voxel_volume));
    k_images<<<nblocks(g->total_pix), kTB, 0, st>>>(g->geo, g->cams, g->halton, inv_nv, R, images, meas, mask, resid,
                                                     loss, g->total_pix, g->stats);
    return cudaGetLastError();
}

cudaError_t launch_backproject(const mst_grid* g, const double* resid, float* bacc, cudaStream_t st) {
    const float inv_nv = (float)(1.0 / (g->n_rays * g->voxel_volume));
    k_backproject<<<nblocks(g->total_pix), kTB, 0, st>>>(g->geo, g->cams, g->halton, inv_nv, resid, bacc, g->total_pix,
                                                          g->stats);
    return cudaGetLastError();
}

cudaError_t launch_los_adjoint(const mst_grid* g, const float* R, const float* bacc, float* gT, cudaStream_t st) {
    const long long total = (long long)g->n_cams * g->geo.nvox;
    k_los_adjoint<<<nblocks(total), kTB, 0, st>>>(g->geo, g->cams, R, bacc, gT, g->stats);
    return cudaGetLastError();
}

cudaError_t launch_ray_counts(const mst_grid* g, float* Q, int mode, cudaStream_t st) {
    const long long n = (long long)g->n_cams * g->geo.nvox;
    cudaError_t e = cudaMemsetAsync(Q, 0, sizeof(float) * n, st);
    if (e != cudaSuccess) return e;
    k_ray_counts<<<nblocks(g->total_pix), kTB, 0, st>>>(g->geo, g->cams, g->halton, Q, g->total_pix);
    if (mode == 1 || mode == 2) k_qweights<<<nblocks(n, kTB, 4096), kTB, 0, st>>>(Q, n, mode);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_tiles(const mst_grid* g, const float* T, const float* bacc, float* adj, cudaStream_t st) {
    k_adjoint_tiles<<<nblocks(g->geo.nvox, kTB, 4096), kTB, 0, st>>>(T, bacc, adj, g->geo.nvox, g->n_cams, g->cp);
    return cudaGetLastError();
}

cudaError_t launch_combine_surrogate(const mst_grid* g, const double* Lsrc, const double* /*jfix*/,
                                     const float* beta_ref, const float* /*beta*/, const float* T, const float* bacc,
                                     const float* gT, const float* Qw, double* grad, cudaStream_t st) {
    k_combine_surrogate<<<nblocks(g->geo.nvox, kTB, 4096), kTB, 0, st>>>(Lsrc, beta_ref, T, bacc, gT, Qw, grad,
                                                                         g->geo.nvox, g->n_cams);
    return cudaGetLastError();
}

cudaError_t launch_combine_full(const mst_grid* g, const float* gT, const double* gL, double* grad, cudaStream_t st) {
    k_combine_full<<<nblocks(g->geo.nvox, kTB, 4096), kTB, 0, st>>>(gT, gL, grad, g->geo.nvox, g->n_cams);
    return cudaGetLastError();
}

cudaError_t launch_classic_residual(const mst_grid* g, const double* img, const double* meas, const uint8_t* mask,
                                    double* resid, double* loss, cudaStream_t st) {
    k_classic_resid<<<nblocks(g->total_pix, kTB, 4096), kTB, 0, st>>>(img, meas, mask, resid, loss, g->total_pix);
    return cudaGetLastError();
}

// Sun mask M_c of Eq. Cost: 0 where the pixel's centre ray is within `radius` of the direction
// to the sun (cos of the angle above cos(radius), evaluated in FP64), 1 elsewhere.
__global__ void k_sun_mask(const CamSet cs, double3 to_sun, double cos_r, uint8_t* __restrict__ mask, int npix) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        const int c = cam_of_pixel(cs, p);
        const Cam& cm = cs.c[c];
        const int li = p - cm.pix_off, i = li % cm.w, j = li / cm.w;
        const double x = (2.0 * (i + 0.5) / cm.w - 1.0) * (double)cm.tx;
        const double y = (2.0 * (j + 0.5) / cm.h - 1.0) * (double)cm.ty;
        const double dx = cm.fx + x * cm.rx + y * cm.ux, dy = cm.fy + x * cm.ry + y * cm.uy;
        const double dz = cm.fz + x * cm.rz + y * cm.uz;
        const double cosang = (dx * to_sun.x + dy * to_sun.y + dz * to_sun.z) / sqrt(dx * dx + dy * dy + dz * dz);
        mask[p] = cosang > cos_r ? 0 : 1;
    }
}

cudaError_t launch_sun_mask(const mst_grid* g, double zenith, double azimuth, double radius, uint8_t* mask,
                            cudaStream_t st) {
    const double3 s = make_double3(std::sin(zenith) * std::cos(azimuth), std::sin(zenith) * std::sin(azimuth),
                                   std::cos(zenith));
    k_sun_mask<<<nblocks(g->total_pix, kTB, 4096), kTB, 0, st>>>(g->cams, s, std::cos(radius), mask, g->total_pix);
    return cudaGetLastError();
}

// Eq. channelBeta: the aerosol of channel mu, sigma~_mu times the reference field (FP64 product,
// rounded to FP32 like every beta the library reads).
__global__ void k_channel_beta(const float* __restrict__ ref, double sigma, float* __restrict__ out, int nvox) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nvox; k += gridDim.x * blockDim.x)
        out[k] = (float)(sigma * (double)ref[k]);
}

// Eq. divCost1 and Eq. Cost over channels: grad += sigma~_mu dE_mu/dbeta_mu, loss += E_mu.
__global__ void k_channel_add(double* __restrict__ grad, double sigma, const double* __restrict__ gmu, int nvox,
                              double* loss, const double* loss_mu) {
    const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int k = k0; k < nvox; k += gridDim.x * blockDim.x) grad[k] += sigma * gmu[k];
    if (k0 == 0) *loss += *loss_mu;
}

cudaError_t launch_channel_beta(const mst_grid* g, const float* ref, double sigma, float* out, cudaStream_t st) {
    k_channel_beta<<<nblocks(g->geo.nvox, kTB, 4096), kTB, 0, st>>>(ref, sigma, out, g->geo.nvox);
    return cudaGetLastError();
}

cudaError_t launch_channel_add(const mst_grid* g, double* grad, double sigma, const double* gmu, double* loss,
                               const double* loss_mu, cudaStream_t st) {
    k_channel_add<<<nblocks(g->geo.nvox, kTB, 4096), kTB, 0, st>>>(grad, sigma, gmu, g->geo.nvox, loss, loss_mu);
    return cudaGetLastError();
}

cudaError_t launch_regularizer(const mst_grid* g, const float* beta, double eta, double* lap, double* psi, double* loss,
                               double* grad, cudaStream_t st) {
    const int nb = nblocks(g->geo.nvox, kTB, 4096);
    cudaError_t e = cudaMemsetAsync(psi, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_lap1<<<nb, kTB, 0, st>>>(g->geo, beta, g->reg_wz, lap, psi);
    if (grad) k_lap2<<<nb, kTB, 0, st>>>(g->geo, lap, eta, grad);
    if (loss) k_add_scaled<<<1, 32, 0, st>>>(loss, psi, eta);
    return cudaGetLastError();
}

}  // namespace mst

/*
 * mst.h - C ABI of the GB300 library for in-situ multi-scattering tomography
 * (Holodovsky, Schechner, Levin, Levis, Aides, "In-situ multi-scattering tomography", 2015).
 *
 * The library renders the paper's voxelised forward Monte-Carlo model and its per-voxel
 * gradient on one CUDA GPU (sm_103a). All arrays passed in or out are device pointers unless
 * a name ends in _host. Nothing here allocates or frees caller memory.
 *
 * Units: lengths in metres, extinction beta in 1/m, angles in radians.
 *
 * Layouts:
 *   voxel k = ix + nx*(iy + ny*iz), x fastest; voxel (ix,iy,iz) covers
 *     [origin + i*h, origin + (i+1)*h) on each axis; z is up; the top face is the top of the
 *     atmosphere where sunlight enters (Sec. 2.1.2, step i).
 *   per-camera fields [C][nvox]; images [sum_c W_c*H_c], camera c's block at offset
 *     sum_{c'<c} W_c' H_c', pixel (i, j) of a block at j*W + i (i = column along `right`,
 *     j = row along `up`).
 *
 * Asynchrony: every call that takes a stream only enqueues work on that stream (cudaStream_t,
 * NULL = legacy default stream) and returns. Errors raised by kernels show up at mst_sync or
 * at the next call. One handle owns scratch buffers, so calls on the same handle must be
 * ordered (same stream, or synchronised by the caller).
 *
 * Return codes: MST_OK (0) or a negative MST_ERR_*; mst_last_error(handle) describes the last
 * failure on that handle.
 */
#ifndef MST_H
#define MST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MST_OK 0
#define MST_ERR_INVALID_ARG (-1) /* rejected before any launch; nothing was enqueued */
#define MST_ERR_CUDA (-2)        /* a CUDA call or kernel failed */
#define MST_ERR_OOM (-3)         /* device allocation failed in mst_create_grid */
#define MST_ERR_NO_DEVICE (-4)   /* no usable CUDA device */
#define MST_ERR_UNSUPPORTED (-5) /* combination of options not implemented */
#define MST_ERR_TOO_LARGE (-6)   /* grid exceeds the fixed scratch of mst_transmittance_noalloc */

#define MST_MAX_CAMERAS 64
#define MST_MAX_SUBPIXEL_RAYS 64
#define MST_NSTATS 32
#define MST_NOALLOC_MAX_VOXELS (1 << 21) /* largest grid (nx ny nz) of mst_transmittance_noalloc */

/* local estimate used by the forward render */
enum { MST_EST_VOXEL = 0, MST_EST_CLASSIC = 1 };
/* storage type of the staged extinction grid (arithmetic is always FP32) */
enum { MST_GRID_F32 = 0, MST_GRID_F16 = 1, MST_GRID_BF16 = 2 };
/* gradient of mst_render_grad */
enum { MST_GRAD_SURROGATE = 0, MST_GRAD_FULL = 1 };
/* diagonal conditioning Q_c of the surrogate gradient (Sec. 6) */
enum { MST_COND_NONE = 0, MST_COND_INV_COUNT = 1, MST_COND_COUNT = 2 };

/* indices into the statistics block (mst_get_stats) */
enum {
    MST_ST_ESC_XM = 0, MST_ST_ESC_XP, MST_ST_ESC_YM, MST_ST_ESC_YP, MST_ST_ESC_ZM, MST_ST_ESC_ZP,
    MST_ST_ABSORBED = 6, MST_ST_RR_KILLED = 7, MST_ST_RR_GAINED = 8, MST_ST_FORCED = 9,
    MST_ST_EVENTS = 10, MST_ST_SEGMENTS = 11, MST_ST_CAPPED = 12, MST_ST_ESCAPED_N = 13,
    MST_ST_LAUNCHED = 14, MST_ST_TRACED = 15,
    MST_ST_REPLAY_SEGMENTS = 16, MST_ST_REPLAY_EVENTS = 17, MST_ST_LOS_SEGMENTS = 18,
    MST_ST_PIXEL_SEGMENTS = 19, MST_ST_BACKPROJ_SEGMENTS = 20, MST_ST_LOSADJ_SEGMENTS = 21,
    MST_ST_REPLAY_SCATTERS = 22,
    MST_ST_LOST = 23, /* walks abandoned (non-finite direction), or replay flights that missed their stored
                         event's voxel; 0 in valid use */
    MST_ST_EVENTS_STORED = 24, /* full gradient: events the forward stored for the adjoint (0: replayed instead) */
    MST_ST_BMC_PATHS = 25, MST_ST_BMC_EVENTS = 26, MST_ST_BMC_SEGMENTS = 27, /* mst_render_bmc: flight + sun-ray voxels */
    MST_ST_AIR_EVENTS = 28, /* two-species medium (mst_set_air): forward events whose particle was air */
    MST_ST_SHADOW_RAYS = 29, MST_ST_SHADOW_SEGMENTS = 30 /* classic estimator (Eq. fle): shadow rays walked by the
                                                            call's transport passes, and their voxel segments (the
                                                            scatter walk of replay pass 2 counted again) */
};

/* phases timed by the profiler (mst_get_phase_times) */
enum {
    MST_PH_STAGE = 0, MST_PH_TRANSPORT = 1, MST_PH_FOLD = 2, MST_PH_LOS = 3, MST_PH_IMAGES = 4,
    MST_PH_BACKPROJECT = 5, MST_PH_LOS_ADJOINT = 6, MST_PH_REPLAY = 7, MST_PH_COMBINE = 8, MST_PH_REPLAY2 = 9,
    MST_PH_REPLAY_LIST = 10, MST_PH_EVENT_ADJOINT = 11, MST_PH_BMC = 12,
    MST_NPHASES = 13 /* MST_PH_REPLAY: replay pass 1 (W per photon); MST_PH_EVENT_ADJOINT: W per photon from
                        the events the forward stored (instead of pass 1); MST_PH_REPLAY_LIST: the list of
                        photons with W != 0 that pass 2 walks; MST_PH_REPLAY2: pass 2 (scatter) */
};

typedef struct mst_grid mst_grid; /* opaque; owned by the library */

/* Voxel grid of cuboid voxels (Sec. 3: beta, albedo and g constant per voxel). */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double origin[3];
} mst_grid_desc;

/* Pinhole camera c with centre of projection X_c = pos (Sec. 2.1). rot holds the
 * world-from-camera axes right, up, forward as three consecutive 3-vectors, orthonormal to
 * 1e-3 (mst_create_grid rejects other bases). The ray through
 * image-plane point (px, py), px in [0, W], py in [0, H], has direction
 * normalize(forward + x right + y up), x = (2 px/W - 1) tan(fov_x/2),
 * y = (2 py/H - 1) tan(fov_x/2) H/W. */
typedef struct {
    double pos[3];
    double rot[9];
    int width, height;
    double fov_x_rad;
} mst_camera;

/* Parameters of one render (Sec. 2.1.2, Sec. 3.2, Sec. 5-6). */
typedef struct {
    double albedo;          /* single-scattering albedo, in [0, 1] */
    double g;               /* Henyey-Greenstein anisotropy, in (-1, 1) (Eq. Phg) */
    double sun_zenith_rad;  /* direction TO the sun: zenith angle ...                        */
    double sun_azimuth_rad; /* ... and azimuth from +x; photons travel along the opposite     */
    double sun_irradiance;  /* F: irradiance on a surface normal to the sun (images in F units) */
    double rr_threshold;    /* Russian roulette below rr_threshold * I0 (0 disables)          */
    double rr_survival;     /* survival probability of the roulette, in (0, 1]                */
    uint64_t n_photons;     /* photons traced by this call (>= 1)                             */
    uint64_t photon_offset; /* global id of the first photon (sharding)                      */
    uint64_t n_photons_total; /* normaliser N in I0 = F cos(theta0) Lx Ly / N; 0 = n_photons  */
    uint64_t seed;          /* Philox key                                                      */
    int max_order;          /* stop after this many scattering events (0 = no limit)          */
    int max_events;         /* hard cap on events per photon, counted in MST_ST_CAPPED        */
    int estimator;          /* MST_EST_VOXEL (the paper's method) or MST_EST_CLASSIC (Eq. fle) */
    int grid_dtype;         /* MST_GRID_F32 / F16 / BF16 storage of the staged beta            */
    int grad_mode;          /* MST_GRAD_SURROGATE or MST_GRAD_FULL                             */
    int conditioning;       /* MST_COND_*: applies to MST_GRAD_SURROGATE only                  */
    double reg_eta;         /* weight eta of the Laplacian regulariser (Eq. Cost, Sec. 6)      */
} mst_params;

/* Fills defaults: albedo 0.99, g 0.85, sun at zenith, F = 1, roulette 0.01 / 0.1,
 * 1e6 photons, seed 3, max_events 100000, voxel estimator, FP32 grid, surrogate gradient,
 * no conditioning, eta 0. */
void mst_default_params(mst_params *p);

/* Geometry pre-calculation (Sec. 3, step i). Copies the grid and cameras into a new handle
 * on the current CUDA device and allocates its scratch buffers. Grid limits: nx, ny <= 2048,
 * nz <= 1024, nx*ny*nz <= 2^30. n_subpixel_rays = N_rays of
 * Eq. PIc (1..MST_MAX_SUBPIXEL_RAYS); the sub-pixel points are the 2-D Halton points (bases 2
 * and 3, indices 1..N_rays). Requires 1 <= n_cams <= MST_MAX_CAMERAS, positive sizes.
 * On failure *out is NULL. */
int mst_create_grid(const mst_grid_desc *grid, int n_cams, const mst_camera *cams, int n_subpixel_rays,
                    mst_grid **out);

/* Releases the handle and everything it owns. NULL-safe. Synchronises the device first. */
void mst_destroy(mst_grid *g);

/* Forward render (Sec. 2.1.2 steps i-vi; Eq. Lcupdate; Eq. taoKtoc-Tck; Eq. Icpixel).
 *   beta_dev   [nvox] float, >= 0, read only.
 *   images_dev [sum W*H] double or NULL: voxel estimator -> i_c = Pi_c (L_c . T_c);
 *              classic estimator -> the local-estimate images of Eq. fle.
 *   L_dev      [C][nvox] double or NULL: L_c(k) of Eq. Lcupdate (voxel estimator only).
 * Photon p (global id photon_offset + p) draws from Philox-4x32-10 with key = seed and
 * counter (id lo, id hi, event, 0). */
int mst_render(mst_grid *g, const float *beta_dev, const mst_params *p, double *images_dev, double *L_dev,
               void *stream);

/* Forward render plus the masked L2 loss of Eq. Cost and its gradient dE/dbeta.
 *   images_meas_dev [sum W*H] double: measured images.
 *   mask_dev        [sum W*H] uint8 or NULL (all ones): the sun mask M_c.
 *   images_dev      [sum W*H] double or NULL: rendered images.
 *   grad_dev        [nvox] double: written (not accumulated).
 *   loss_dev        [1] double or NULL: E = sum M (i - i_meas)^2 + eta Psi.
 * MST_GRAD_SURROGATE: the paper's gradient with j = L/beta held fixed (Eq. divCost1 with
 * Eq. Jaco1, Eq. TcofJaco1, Eq. DivTc) and conditioning Q_c.
 * MST_GRAD_FULL: the full gradient of Eq. DirectJacob applied to the residual, where
 * dL/dbeta is estimated by the score of the free-flight density (Eq. beer-lambert,
 * Eq. MCextinct) over paths replayed from their Philox keys. W = sum_s w_s per photon and the
 * w_s come from the events the forward render stored (44 B per event, within the handle's
 * budget, see mst_set_replay_memory), or, when they do not fit, from a first replay of every
 * path; a last replay scatters the score. Results agree either way. With MST_EST_CLASSIC the
 * images are Eq. fle's, w_s weights each camera's classic contribution by its pixel's dE/di,
 * and each contribution's shadow ray adds its own term (no events are stored). The surrogate
 * gradient needs the voxel estimator. */
int mst_render_grad(mst_grid *g, const float *beta_dev, const mst_params *p, const double *images_meas_dev,
                    const uint8_t *mask_dev, double *images_dev, double *grad_dev, double *loss_dev, void *stream);

/* Sun mask M_c of Eq. Cost (Sec. 5: pixels around the sun are left out of the loss):
 * mask_dev[p] = 0 for the pixels whose centre ray (image point (i + 1/2, j + 1/2)) makes an
 * angle below radius_rad with the direction to the sun (sun_zenith_rad, sun_azimuth_rad as in
 * mst_params), 1 for the others; the result is the mask_dev argument of mst_render_grad.
 *   mask_dev [sum W*H] uint8, written. radius_rad in [0, pi]; 0 masks nothing.
 * The camera axes are held in FP32, so a pixel within ~1e-6 rad of the edge may fall either way.
 * Returns MST_ERR_INVALID_ARG for a radius outside [0, pi] or non-finite sun angles. */
int mst_sun_mask(mst_grid *g, double sun_zenith_rad, double sun_azimuth_rad, double radius_rad, uint8_t *mask_dev,
                 void *stream);

/* LOS transmittance T_c(k) = exp(-tau_c(k)), tau_c = W_c beta, from the centre of voxel k to
 * X_c (Eq. taoKtoc, Eq. Dvc, Eq. bTck, Eq. Tck). T_dev [C][nvox] float. grid_dtype as above. */
int mst_transmittance(mst_grid *g, const float *beta_dev, int grid_dtype, float *T_dev, void *stream);

/* Image formation from a given L (Eq. Rc, Eq. IcPJbetaT, Eq. Icpixel):
 * i_c(p) = 1/(N_rays V) sum_rho sum_k l^rho_{c,p}(k) L_c(k) T_c(k), T from beta_dev.
 * L_dev [C][nvox] double, images_dev [sum W*H] double. */
int mst_form_images(mst_grid *g, const float *beta_dev, int grid_dtype, const double *L_dev, double *images_dev,
                    void *stream);

/* Surrogate gradient with j = L_ref/beta_ref held fixed (Sec. 5.2; Eq. minobjectiveBetaQplus1,
 * Eq. Jaco1-DivTc; j = 0 where beta_ref = 0): images i_c = Pi_c(j . beta . T_c(beta)), loss
 * and dE/dbeta at beta_dev, with p->conditioning and p->reg_eta. Only p->conditioning,
 * p->reg_eta and p->grid_dtype are read. No photons are traced: this is the inner step of
 * the N_GD loop of Eq. GD. L_ref_dev [C][nvox] double, beta_ref_dev [nvox] float. */
int mst_surrogate_grad(mst_grid *g, const float *beta_dev, const double *L_ref_dev, const float *beta_ref_dev,
                       const mst_params *p, const double *images_meas_dev, const uint8_t *mask_dev,
                       double *images_dev, double *grad_dev, double *loss_dev, void *stream);

/* Q_c(k): number of sub-pixel rays through voxel k (Sec. 6); a ray counts when its chord in
 * the voxel is at least 1e-4 of the smallest voxel edge.
 * Q_dev [C][nvox] float. */
int mst_ray_counts(mst_grid *g, float *Q_dev, void *stream);

/* Laplacian regulariser Psi = ||W Lap beta||^2 with the 6-neighbour graph Laplacian and W
 * diagonal by altitude (Sec. 6; W = I unless mst_set_reg_weights gave weights), gradient
 * 2 Lap^T W^T W Lap beta. psi_dev [1] double or NULL; grad_dev [nvox] double or NULL,
 * receives += eta dPsi. */
int mst_regularizer(mst_grid *g, const float *beta_dev, double eta, double *psi_dev, double *grad_dev,
                    void *stream);

/* Altitude weights of the regulariser (Sec. 6): W_kk = wz_host[iz] for voxel k in layer iz.
 * wz_host [nz] double, copied; NULL restores W = I. Used by mst_regularizer and by the eta
 * term of mst_render_grad and mst_surrogate_grad. Synchronises the device. */
int mst_set_reg_weights(mst_grid *g, const double *wz_host);

/* Backward Monte Carlo with the sun local estimate (Eq. ble; Sec. 3, the paper's check of the
 * in-situ forward model): for every pixel, n_per_pixel paths start at the camera through uniform
 * points of the pixel (weight cos^3 A_pix / Omega_p, so the mean is the pixel's solid-angle
 * average radiance), fly by the same voxel walk as the forward transport, and at each
 * scattering event add albedo I P_HG(d . s_sun) exp(-tau) F, where tau is the optical depth
 * along the sun-ward ray and the event counts as sunlit only if that ray leaves through the top
 * face (the forward model's illumination); then albedo, roulette and HG sampling as in
 * mst_render. Sample q of global pixel p draws Philox counters (q, event, 1 + p) under p->seed.
 *   images_dev [sum W*H] double: pixel means, in the units of mst_render's images.
 *   var_dev    [sum W*H] double or NULL: variance of each pixel's mean (n_per_pixel >= 2).
 * Reads albedo, g, the sun angles and irradiance, rr_threshold (absolute: a path starts with
 * weight 1), rr_survival, max_order, max_events, seed and grid_dtype. n_per_pixel >= 1; the
 * handle's per-pixel FP64 scratch is reused. */
int mst_render_bmc(mst_grid *g, const float *beta_dev, const mst_params *p, uint32_t n_per_pixel, double *images_dev,
                   double *var_dev, void *stream);

/* Two-species medium (Sec. 2; Sec. 2.1.2 steps iv-vi): air molecules beside the aerosol field
 * that beta describes. The extinction the photons see is beta + beta_air; at each scattering
 * event the particle is air with probability beta_air / (beta + beta_air) in the event's voxel
 * (Philox counter (id lo, id hi, event, 0xFFFFFFFF), first uniform u: air when
 * u (beta + beta_air) < beta_air, evaluated in FP64), and the event takes that particle's albedo
 * (albedo_air for air, params.albedo for aerosol) and phase function: Rayleigh (Eq. Pray),
 * sampled by Eq. thetaREY, for air; Henyey-Greenstein (Eq. Phg) for aerosol.
 *   beta_air_dev [nvox] float, >= 0, on the handle's device, or NULL for one species. Borrowed:
 *                the caller keeps it alive and unchanged until it is replaced or the handle
 *                is destroyed; it is read by every later call.
 *   albedo_air   in [0, 1] (1: air absorbs nothing at visible wavelengths).
 * With air set, mst_render and mst_render_grad render the mixture, and the gradients are
 * dE/dbeta w.r.t. the aerosol field (the air field is known). MST_GRAD_FULL: the free-flight
 * score of every flight plus 1/beta for aerosol events only, and the LOS transmittance through
 * the total extinction. MST_GRAD_SURROGATE and mst_surrogate_grad (whose beta and beta_ref are
 * then aerosol fields too): j = L / (beta + beta_air) held fixed, every term a derivative
 * w.r.t. the total, which equals the derivative w.r.t. the aerosol. The regulariser acts on the
 * aerosol field. mst_render_bmc returns MST_ERR_UNSUPPORTED (one species); mst_transmittance,
 * mst_form_images, mst_ray_counts and mst_regularizer use the field they are given. The first
 * call with a field allocates two [nvox] float buffers on the handle (the FP32 totals); no
 * other device work. Returns MST_ERR_INVALID_ARG for albedo_air outside [0, 1]. */
int mst_set_air(mst_grid *g, const float *beta_air_dev, double albedo_air);

#define MST_MAX_CHANNELS 8

/* One colour channel mu of a multi-channel reconstruction (Sec. 5, Eq. channelBeta). */
typedef struct {
    mst_params params;              /* the channel's render: aerosol albedo and g, sun irradiance F_mu, photons,
                                       seed, estimator, grad_mode, conditioning, grid_dtype; reg_eta is
                                       ignored (the regulariser acts once, on the reference field) */
    const float *beta_air_dev;      /* [nvox] float air extinction in this channel, or NULL (no air) */
    double albedo_air;              /* air albedo in this channel, in [0, 1] */
    double sigma_ratio;             /* sigma~_mu = sigma_aerosol,mu / sigma_aerosol,ref, > 0 */
    const double *images_meas_dev;  /* [sum W*H] measured images of the channel */
    double *images_dev;             /* [sum W*H] rendered images of the channel, or NULL */
} mst_channel;

/* Multi-channel loss and gradient w.r.t. the reference channel's aerosol field
 * (Eq. channelBeta, Eq. Cost, Eq. divCost1). Channel mu renders the two-species medium with
 * aerosol sigma_ratio_mu * beta_aer_dev (rounded to float) and its own air field, as
 * mst_render_grad with mst_set_air would; then
 *   E = sum_mu E_mu + eta Psi(beta_aer),  dE/dbeta_aer = sum_mu sigma_ratio_mu dE_mu/dbeta_mu + eta dPsi,
 * E_mu the masked L2 loss of channel mu (Eq. Cost) and Psi the regulariser of mst_regularizer.
 *   beta_aer_dev [nvox] float >= 0; channels [n_channels] host structs (1..MST_MAX_CHANNELS);
 *   mask_dev [sum W*H] uint8 or NULL, shared by all channels; grad_dev [nvox] double, written;
 *   loss_dev [1] double or NULL.
 * With MST_GRAD_SURROGATE in a channel's params, dE_mu/dbeta_mu is the surrogate of
 * mst_render_grad (Eq. divCost1 with Q_c, j of the channel fixed). The handle's own mst_set_air
 * setting is left as it was. Channels run one after another on the stream; mst_get_stats then
 * holds the last channel's statistics. */
int mst_render_grad_channels(mst_grid *g, const float *beta_aer_dev, int n_channels, const mst_channel *channels,
                             const uint8_t *mask_dev, double eta, double *grad_dev, double *loss_dev, void *stream);

/* Wavefront shape of the persistent transport kernels on this handle: the voxels a flying lane
 * advances per loop trip, and the resident blocks per SM, for the forward render (voxel
 * estimator) and for replay pass 2. 0 keeps the built-in default (12 and 6 voxels; the
 * register budget's occupancy, 3 blocks). The trip is a compile-time constant of the kernels:
 * forward trips 8, 10, 12, 16 and pass-2 trips 4, 6, 8, 10 are built, for the FP32 grid (the
 * FP16 / BF16 grids use the defaults). Results do not depend on the shape beyond the order of
 * floating-point additions: each photon's path is fixed by its Philox key. Blocks per SM in
 * 0..8 (more than the occupancy runs at the occupancy); other trips return MST_ERR_INVALID_ARG. */
int mst_set_wavefront(mst_grid *g, int forward_trip, int forward_blocks_per_sm, int replay_trip,
                      int replay_blocks_per_sm);

/* Autotuner of the wavefront shape. Times full-gradient calls of the voxel estimator on this
 * scene (beta_dev; p's optics, sun, seed and grid_dtype; zero measured images) with n_sample
 * photons for each candidate (forward trips 8, 10, 12, 16 and pass-2 trips 4, 6, 8, 10, each at
 * the register budget's occupancy and one block per SM less), sets the fastest forward and
 * pass-2 shapes on the handle (as mst_set_wavefront) and writes them to
 * choice_host[4] = {forward trip, forward blocks per SM, pass-2 trip, pass-2 blocks per SM}.
 * Synchronises the stream, allocates and frees its own scratch, leaves the handle's statistics
 * those of its last call. n_sample in [2^16, 2^27]; on failure the shape is left unchanged. */
int mst_autotune(mst_grid *g, const float *beta_dev, const mst_params *p, uint64_t n_sample, int *choice_host,
                 void *stream);

/* Device memory the handle may hold for the events a full-gradient forward render stores
 * (60 B per scattering event: voxel, position, incoming direction, weight, photon index, event
 * number, the free path left on entering the voxel, and the event's step for replay pass 2:
 * w_s, voxel, free path), for
 * calls of at most 2^27 photons. Default 32 GiB; 0 stores nothing (W by replay). The buffer
 * is allocated at the first full-gradient call that needs it and grown, within the budget,
 * when a call stored more events than it held, and never so large that less than a sixteenth of
 * the device's memory (at least 4 GiB) stays free; a call whose events do not fit, or whose
 * allocation fails, computes W by replay instead. Takes effect at the next call. */
int mst_set_replay_memory(mst_grid *g, uint64_t bytes);

/* Validation aids for the forward render, kept on the handle until replaced:
 *   photon_hash_dev [n_photons] uint32 or NULL: per-photon path checksum (FNV-1a over the
 *     event voxels, then the event count and the termination code 1 escape, 2 absorbed,
 *     3 roulette, 4 max_order, 5 event cap); 0 for skipped photons.
 *   photon_skip_dev [n_photons] uint8 or NULL: photons with a nonzero entry are not traced.
 * Both are indexed by the call's photon index (0 .. n_photons-1). */
int mst_set_debug(mst_grid *g, uint32_t *photon_hash_dev, const uint8_t *photon_skip_dev);

/* Validation aid for the forward render, kept on the handle until replaced (NULL: off):
 *   photon_point_dev [n_photons][4] float: each traced photon's last event point (its launch
 *     point if it had no event) as the offset inside its voxel (x, y, z in metres, entries 0-2)
 *     and the voxel packed as ix | iy << 11 | iz << 22 (entry 3, the bits of a uint32). With the
 *     path checksum this tells whether FP32 carried the photon along the path of an FP64
 *     reference: positions drift apart along long paths (Sec. 2.1.2 steps ii-iii) even where
 *     the voxels agree. Indexed by the call's photon index; skipped photons are not written. */
int mst_set_debug_points(mst_grid *g, float *photon_point_dev);

/* Copies the statistics of the last render call (MST_NSTATS doubles: escaped weight per face,
 * absorbed, roulette, segment and event counts) to the host. Synchronises the device. */
int mst_get_stats(mst_grid *g, double *stats_host);

/* Enables (1) or disables (0) the phase profiler: every later call records a CUDA event pair on
 * its stream around each kernel launch, grouped by MST_PH_* phase. */
int mst_set_profiling(mst_grid *g, int enable);

/* Per-phase device time of the last call, in ms (ms_host[MST_NPHASES]), and the number of
 * launches per phase (launches_host[MST_NPHASES], may be NULL). Synchronises the device.
 * Returns MST_ERR_INVALID_ARG when profiling is off. */
int mst_get_phase_times(mst_grid *g, double *ms_host, int *launches_host);

/* Waits for the handle's work and reports any asynchronous error. */
int mst_sync(mst_grid *g);

/* Message of the last error on the handle ("" if none); valid until the next call. */
const char *mst_last_error(mst_grid *g);

/* LOS transmittance without a handle and without allocating: for callers that cannot call
 * cudaMalloc (hosts that hand out device memory only from their own arena, plugins that may not
 * allocate after start-up). The paper has no counterpart: it
 * computes the same T_c(k) as mst_transmittance (FP32 grid) for the grid and cameras given.
 *   beta_dev [nvox] float, T_dev [C][nvox] float: the caller's buffers.
 * Scratch: a fixed device array of MST_NOALLOC_MAX_VOXELS floats (8 MiB) inside the library,
 * held by every GPU that loads it until the process exits. Grids of more voxels (nx ny nz) are
 * rejected with MST_ERR_TOO_LARGE before anything is enqueued (e.g. 128^3 fits, 136 x 128 x 128
 * does not).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call outside any stream capture. The address is kept for the life of the
 * process: after a cudaDeviceReset of that device it is stale. Every call shares the one array and
 * overwrites it; calls whose work overlaps on the GPU (other streams, other threads) race,
 * so order them on one stream or synchronise between them. Returns MST_OK, MST_ERR_INVALID_ARG,
 * MST_ERR_TOO_LARGE, MST_ERR_NO_DEVICE or MST_ERR_CUDA. */
int mst_transmittance_noalloc(const mst_grid_desc *grid, int n_cams, const mst_camera *cams, const float *beta_dev,
                              float *T_dev, void *stream);

/* Batched scenes (many independent scenes of uneven size; Sec. 1 photon parallelism across them).
 * A batch owns one CUDA graph holding the mst_render_grad sequences of n distinct handles, each
 * on its own branch, so scenes of uneven size overlap on the GPU and the whole batch is one
 * graph launch. The graph is captured on the first call (work is enqueued on internal
 * streams; the handles' conditioning weights are prepared on `stream` first, and each
 * full-gradient handle's event and per-photon buffers are sized for its photons, so that the
 * graph's forwards store their events as mst_render_grad's do) and replayed while every
 * pointer, parameter and handle buffer is unchanged; any change, including a buffer a direct
 * call on one of the handles reallocated, re-captures it. Results are those of n
 * mst_render_grad calls with the same arguments.
 *   grids: n distinct handles on one device (1 <= n <= MST_MAX_BATCH); the batch does not own
 *          them and must be destroyed before them.
 *   betas[i], params[i], meas[i], masks[i] (masks may be NULL, entries may be NULL),
 *   images[i] (images may be NULL, entries may be NULL), grads[i]: as in mst_render_grad.
 *   losses [n] device doubles. */
#define MST_MAX_BATCH 64
typedef struct mst_batch mst_batch;
int mst_batch_create(int n, mst_grid *const *grids, mst_batch **out);
int mst_batch_render_grad(mst_batch *b, const float *const *betas, const mst_params *params,
                          const double *const *images_meas, const uint8_t *const *masks, double *const *images,
                          double *const *grads, double *losses_dev, void *stream);
const char *mst_batch_last_error(mst_batch *b);

/* Form of the batch's graph (Sec. 1: photons of all scenes are independent work items).
 * MST_BATCH_BRANCHES (the default): one graph branch per scene holding that scene's
 * mst_render_grad sequence; the branches overlap on the GPU.
 * MST_BATCH_PERSISTENT: the photon transport of all scenes runs as single
 * persistent launches (forward, stored-event adjoint, replay passes 1 and 2), every warp taking
 * the scenes one after the other from a device table, with each scene's small kernels (staging,
 * LOS, images, back-projection, folds) on a graph branch of its own between them. It applies
 * when every scene renders the voxel estimator's full gradient on an FP32 grid with one species
 * and its events fit the handle's budget; otherwise the call falls back to the branches. The
 * persistent kernels read each scene's arguments from device memory instead of the parameter
 * bank, which costs them registers: at 16 uneven scenes the branches are the faster form.
 * mst_batch_get_form returns the form of the last captured graph (-1 for NULL). */
enum { MST_BATCH_BRANCHES = 0, MST_BATCH_PERSISTENT = 1 };
int mst_batch_set_form(mst_batch *b, int form);
int mst_batch_get_form(mst_batch *b);

/* Wavefront of the persistent form's launches, as mst_set_wavefront sets it for one handle:
 * forward voxels per trip in {0, 8, 10, 12, 16} (0 or 12: default), pass-2 voxels per trip in
 * {0, 4, 6, 8, 10} (0 or 6: default), blocks per SM (0: the register budget's occupancy). */
int mst_batch_set_wavefront(mst_batch *b, int forward_trip, int forward_blocks, int replay_trip, int replay_blocks);

/* Times batch calls on a sample of the given call (each scene's photons divided by sample_div,
 * no regulariser) for each wavefront candidate, forward shapes first, then pass 2's, and keeps
 * the fastest; choice[4] receives forward trip, forward blocks per SM, pass-2 trip, pass-2 blocks
 * per SM. The handles' record-buffer sizing is restored afterwards. Synchronises the stream. */
int mst_batch_autotune(mst_batch *b, const float *const *betas, const mst_params *params,
                       const double *const *images_meas, int sample_div, int *choice, void *stream);
void mst_batch_destroy(mst_batch *b); /* NULL-safe; synchronises the device first */

/* Library version (integer, increases with the ABI). */
int mst_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MST_H */

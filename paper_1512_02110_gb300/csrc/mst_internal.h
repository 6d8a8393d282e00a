// Host-side handle and kernel argument blocks shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mst.h"
#include "mst_dev.cuh"

namespace mst {

// The transport accumulates into FP32 tiles. While a launch runs, every new ticket batch of a
// warp also folds one slice of the tile into the FP64 result (swap to zero, add in FP64), the
// slices sized so that a sweep over the whole tile takes at most about kFoldSweep photons:
// no FP32 bin sums more than a sweep's contributions, however many photons a launch traces.
constexpr uint64_t kMaxPhotons = 1ull << 34;    // photons per call
constexpr uint64_t kLaunchPhotons = 1ull << 30;  // photons per forward launch (32-bit ticket)
constexpr uint64_t kReplayChunk = 1ull << 24;    // photons per replay pass-1 / pass-2 pair
// Full gradient: the forward stores its events (kEventWords words each, structure of arrays)
// for calls of at most kRecordMaxPhotons photons; W then comes from the stored events and the
// replay is one pass-2 launch over the call's photons.
constexpr uint64_t kRecordMaxPhotons = 1ull << 27;
// packed voxel, offset (3), incoming direction (3), albedo * weight, photon, event number, and the
// free path left when the flight entered the event's voxel
constexpr int kEventWords = 11;
// What replay pass 2 needs of each stored event, in the photon's slot (event order): w_s, the
// event's packed voxel and the free path left on entering it. Pass 2 then walks each flight to
// that voxel without loading the extinction of the voxels before it.
struct EventStep {
    float w;
    uint32_t vox;
    float tau_in;
    uint32_t pad;
};
constexpr int kEventBytes = kEventWords * 4 + (int)sizeof(EventStep);  // the record and its slot
constexpr unsigned kEventChunk = 256;  // record slots a warp of the forward reserves at a time
constexpr int kTransportWarps = 8;     // warps per transport block (256 threads)
constexpr uint32_t kEndChunk = 0xFFFFFFFFu;  // end of a warp's chunk list
constexpr int kMaxWarpsPerSm = 64;     // warp_head entries per SM (the forward runs 24)
constexpr uint64_t kDefaultRecordBytes = 32ull << 30;
constexpr uint64_t kFoldSweep = 1ull << 21;
constexpr int kTicketBatch = 64;  // photon ids a warp takes from the global ticket at a time
constexpr int kMaxTickets = (int)(2 * (kMaxPhotons / kReplayChunk));
constexpr int kScoreBins = 64;  // replay pass-2 list bins over the pass-1 event count (multiple of 32)

// A photon that replay pass 2 must walk: index in the chunk, event count and W of pass 1.
struct ScoreRec {
    uint32_t pid;
    uint32_t nev;
    double W;
};

struct TransportArgs {
    Geo g;
    CamSet cams;
    HG hg;
    const void* beta;          // staged extinction [nvox] in the compute dtype (camera and shadow rays)
    const void* beta_pad;      // the same on the padded grid of the flights (halo +inf)
    const float* beta_air;     // two species: air extinction [nvox] (NULL: one species)
    const float* beta_aer;     // two species: aerosol extinction [nvox], the unknown
    float3 sun;                // photon direction at launch
    float albedo, I0, rr_below, rr_survival, inv_rr_survival;
    float albedo_air;          // single-scattering albedo of air (two species)
    uint2 key;
    uint64_t first_id;         // global id of chunk photon 0
    uint32_t n;                // photons in this chunk
    uint32_t out_base;         // call-relative index of chunk photon 0 (hash / skip arrays)
    int max_order, max_events;
    int cp;                    // padded camera stride of the [nvox][cp] tiles (multiple of 4)
    float* Lacc;               // [nvox][cp] FP32 accumulator (voxel estimator)
    double* cimg;              // classic images (classic estimator)
    const float* omega;        // [total pix] pixel solid angles (classic estimator)
    const double* cres;        // [total pix] dE/di of the classic images (classic-estimator gradient)
    const float* adj;          // [nvox][cp] a_c(k) = T_c(k) b_c(k) (replay)
    float* gacc;               // [npad] FP32 gradient accumulator on the padded grid (replay)
    double* wbuf;              // [photons of the chunk] W per photon (replay pass 1, stored-event adjoint)
    uint32_t* nevbuf;          // [photons of the chunk] events per photon (replay pass 1, or the forward
                               // when it stores events)
    uint32_t* evrec;           // stored events [kEventWords][ev_cap] (forward), or NULL
    unsigned long long ev_cap;     // capacity of evrec in events (0: no events stored)
    unsigned long long* ev_count;  // events offered for storage; > ev_cap: they did not fit
    EventStep* wseq;           // [ev_cap] the stored events' steps, photon after photon (event order)
    uint32_t* ch_next;         // [ev_cap / kEventChunk] next chunk of the same forward warp (kEndChunk: none)
    uint32_t* warp_head;       // [warps of the forward launch] each warp's first chunk (kEndChunk: none)
    uint32_t n_warps;          // warps of the forward launch that stored the events
    const uint32_t* evoff;     // [photons of the call] each photon's first slot in wseq
    const ScoreRec* plist;     // [kReplayChunk] photons with W != 0 (replay pass 2)
    const unsigned int* plist_n;  // entries in plist
    double* L64;               // [C][nvox] FP64 result the L tile folds into
    double* g64;               // [nvox] FP64 result the gradient tile folds into
    uint64_t fold_bins;        // bins of the tile this launch folds while it runs (0: none)
    uint32_t fold_slice;       // bins per slice (one slice per ticket batch)
    uint32_t fold_nslices;     // slices per sweep
    double* stats;             // [MST_NSTATS]
    uint32_t* hash;            // per-photon checksum or NULL
    float4* point;             // per-photon last event point (offset, packed voxel) or NULL
    const uint8_t* skip;       // per-photon skip mask or NULL
    unsigned int* ticket;      // per-chunk photon ticket
};

}  // namespace mst

struct mst_grid {
    int device = 0;
    int sm_count = 0;
    mst::Geo geo{};
    mst::CamSet cams{};
    mst::Halton halton{};
    int n_cams = 0, cp = 0, total_pix = 0, n_rays = 0;
    double origin[3] = {0, 0, 0};
    double voxel_volume = 0;

    // device buffers owned by the handle
    void* ext = nullptr;          // staged extinction [nvox], up to 4 bytes per voxel
    void* ext_pad = nullptr;      // staged extinction on the padded grid [npad] (photon flights)
    float* Lacc = nullptr;        // [nvox][cp]
    double* L64 = nullptr;        // [C][nvox]
    float* T = nullptr;           // [C][nvox]
    float* R = nullptr;           // [C][nvox]  L_c T_c
    float* bacc = nullptr;        // [C][nvox]  Pi_c^T (2 r_c)
    float* gT = nullptr;          // [C][nvox]  W_c^T (L T b)
    float* adj = nullptr;         // [nvox][cp] T_c b_c
    float* gacc = nullptr;        // [npad] gradient tile on the padded grid
    double* wbuf = nullptr;       // [replay_cap], allocated by the first full-gradient call
    uint32_t* nevbuf = nullptr;   // [replay_cap]
    mst::ScoreRec* plist = nullptr;     // [replay_cap]
    uint32_t* evoff = nullptr;          // [replay_cap] first step slot of each photon (stored events)
    uint64_t replay_cap = 0;            // photons the four buffers above hold
    uint32_t* evrec = nullptr;          // [kEventWords][ev_cap] stored events (full gradient)
    mst::EventStep* wseq = nullptr;     // [ev_cap] their steps (w_s, voxel, free path), grouped by photon
    unsigned long long ev_cap = 0;
    unsigned long long* ev_count = nullptr;  // device counter of the last recording forward
    unsigned long long* ev_seen = nullptr;   // pinned host copy of it, read at the next call
    cudaEvent_t ev_seen_ready = nullptr;     // recorded after that copy
    bool ev_seen_pending = false;
    bool ev_counted = false;                 // a count of this handle's stored events has arrived
    unsigned long long ev_last = 0;          // events offered by the last storing call whose count arrived
    bool capturing = false;                  // inside a stream capture: no allocation, no event query
    bool batch_stored = false;               // the batch allocated this handle's event buffers before capture
    int wf_trip[7] = {0, 0, 0, 0, 0, 0, 0};    // per kernel mode: voxels per trip (0: kernel default) ...
    int wf_blocks[7] = {0, 0, 0, 0, 0, 0, 0};  // ... and blocks per SM (0: the register budget's occupancy)
    uint64_t rec_budget = mst::kDefaultRecordBytes;
    unsigned int* score_cnt = nullptr;  // [2 kScoreBins + 1] list bin counts, bin fill, list length
    double* g64 = nullptr;        // [nvox]
    double* resid = nullptr;      // [total_pix] 2 M (i - i_meas)
    double* cimg = nullptr;       // [total_pix] classic images of a gradient call
    double* lap = nullptr;        // [nvox] W^T W Lap beta
    double* reg_wz = nullptr;     // [nz] altitude weights W of the regulariser, NULL: W = I
    const float* air = nullptr;   // [nvox] air extinction (borrowed, mst_set_air), NULL: one species
    double albedo_air = 1.0;      // single-scattering albedo of air
    const float* beta_in = nullptr;  // the running call's beta (the aerosol field with air)
    uint32_t* ch_next = nullptr;  // [ev_cap / kEventChunk] chunk lists of the stored events
    uint32_t* warp_head = nullptr;  // [sm_count * kMaxWarpsPerSm] first chunk of each forward warp
    uint32_t ev_warps = 0;        // warps of the last storing forward launch
    float* btot = nullptr;        // [nvox] two species: beta + beta_air in FP32, written by the staging
    float* btot_ref = nullptr;    // [nvox] two species: beta_ref + beta_air (mst_surrogate_grad)
    float* ch_beta = nullptr;     // [nvox] mst_render_grad_channels: the channel's aerosol field
    double* ch_grad = nullptr;    // [nvox] mst_render_grad_channels: the channel's gradient
    float* omega = nullptr;       // [total_pix]
    float* Qw = nullptr;          // [C][nvox] conditioning weights for qw_mode
    int qw_mode = -1;
    double* stats = nullptr;      // [MST_NSTATS]
    unsigned int* tickets = nullptr;  // [kMaxTickets]

    // phase profiler: event pairs recorded on the call's stream
    struct ProfRec {
        int phase;
        cudaEvent_t a, b;
    };
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_next = 0;
    std::vector<ProfRec> prof_recs;

    uint32_t* dbg_hash = nullptr;
    const uint8_t* dbg_skip = nullptr;
    float4* dbg_point = nullptr;
    std::string err;
};

namespace mst {

// launchers (all enqueue on `st`; return cudaGetLastError())
cudaError_t launch_stage(const mst_grid* g, const float* beta, const float* air, int dtype, cudaStream_t st);
cudaError_t launch_sun_mask(const mst_grid* g, double zenith, double azimuth, double radius, uint8_t* mask,
                            cudaStream_t st);
cudaError_t launch_add_air(const mst_grid* g, const float* beta, const float* air, float* out, cudaStream_t st);
cudaError_t launch_channel_beta(const mst_grid* g, const float* ref, double sigma, float* out, cudaStream_t st);
cudaError_t launch_channel_add(const mst_grid* g, double* grad, double sigma, const double* gmu, double* loss,
                               const double* loss_mu, cudaStream_t st);
// transport kernel modes: 0 forward voxel LE, 1 forward classic LE, 3 replay pass 1, 2 replay pass 2,
// 4 replay pass 2 reading w_s from the stored events, 5 / 6 passes 1 / 2 of the classic-estimator
// gradient
cudaError_t launch_transport(const mst_grid* g, const TransportArgs& a, int dtype, int mode, int blocks,
                             cudaStream_t st);
cudaError_t launch_fold_L(const mst_grid* g, cudaStream_t st);
cudaError_t launch_fold_grad(const mst_grid* g, cudaStream_t st);
cudaError_t launch_score_list(const mst_grid* g, uint32_t n, cudaStream_t st);
// W per photon from the stored events (returns at once when they did not fit)
cudaError_t launch_event_adjoint(const mst_grid* g, const TransportArgs& a, int dtype, cudaStream_t st);
// backward MC images (Eq. ble): n paths per pixel, sums into sum / sum2, then sum <- means and
// var <- variances of the means (var may be NULL)
cudaError_t launch_bmc(const mst_grid* g, const mst_params* p, uint32_t n, double* sum, double* sum2, double* var,
                       cudaStream_t st);
// evoff = exclusive prefix sum of the n photons' event counts (nevbuf)
cudaError_t launch_event_offsets(const mst_grid* g, uint32_t n, cudaStream_t st);
cudaError_t launch_los(const mst_grid* g, int dtype, const double* L, const double* jfix, const float* beta_ref,
                       const float* beta, float* T_out, float* R_out, cudaStream_t st);
cudaError_t launch_images(const mst_grid* g, const float* R, double* images, const double* meas, const uint8_t* mask,
                          double* resid, double* loss, cudaStream_t st);
cudaError_t launch_backproject(const mst_grid* g, const double* resid, float* bacc, cudaStream_t st);
cudaError_t launch_los_adjoint(const mst_grid* g, const float* R, const float* bacc, float* gT, cudaStream_t st);
cudaError_t launch_ray_counts(const mst_grid* g, float* Q, int mode, cudaStream_t st);
cudaError_t launch_adjoint_tiles(const mst_grid* g, const float* T, const float* bacc, float* adj, cudaStream_t st);
cudaError_t launch_combine_surrogate(const mst_grid* g, const double* Lsrc, const double* jfix, const float* beta_ref,
                                     const float* beta, const float* T, const float* bacc, const float* gT,
                                     const float* Qw, double* grad, cudaStream_t st);
cudaError_t launch_combine_full(const mst_grid* g, const float* gT, const double* gL, double* grad, cudaStream_t st);
cudaError_t launch_classic_residual(const mst_grid* g, const double* img, const double* meas, const uint8_t* mask,
                                    double* resid, double* loss, cudaStream_t st);
cudaError_t launch_regularizer(const mst_grid* g, const float* beta, double eta, double* lap, double* psi,
                               double* loss, double* grad, cudaStream_t st);
int transport_blocks_per_sm(int dtype, int mode, bool two);
// The batched form (FP32 grid, one species): one persistent launch of transport mode `mode` (0, 3,
// 4 or 2) over n scenes whose arguments sit in the device table, scene after scene in every warp;
// trip as in the handle's wavefront setting (0: the mode's default).
cudaError_t launch_transport_batch(const TransportArgs* table, int n, int mode, int trip, int blocks,
                                   cudaStream_t st);
cudaError_t launch_event_adjoint_batch(const TransportArgs* table, int n, int blocks, cudaStream_t st);
// Resident blocks per SM of the batched kernels of a mode; the first call sets the attributes of
// every batched instantiation (call it before a stream capture).
int transport_batch_blocks_per_sm(int mode);
// blocks of a persistent transport launch of this mode on the handle (its wavefront setting)
inline int transport_blocks(const mst_grid* g, int dtype, int mode) {
    const int occ = transport_blocks_per_sm(dtype, mode, g->air != nullptr);
    const int b = g->wf_blocks[mode];
    return g->sm_count * (b > 0 && b < occ ? b : occ);
}

}  // namespace mst

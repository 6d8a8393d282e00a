// C ABI of the library: argument validation, handle ownership and the order of kernel
// launches for each call. No computation of the method happens on the host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "mst_internal.h"

using namespace mst;

namespace {

constexpr int kVersion = 1;

int fail(mst_grid* g, int code, const std::string& msg) {
    if (g) g->err = msg;
    return code;
}

#define MST_CK(expr)                                                                                   \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return fail(g, MST_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Phase profiler: an event pair on the call's stream around each launch, when enabled.
void prof_reset(mst_grid* g) {
    g->ev_next = 0;
    g->prof_recs.clear();
}

cudaEvent_t prof_event(mst_grid* g) {
    if (g->ev_next == g->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g->ev_pool.push_back(e);
    }
    return g->ev_pool[g->ev_next++];
}

// NVTX range names of the phases (MST_PH_*), for profilers that attach (ncu --nvtx)
const char* const kPhaseNames[MST_NPHASES] = {"mst:stage",   "mst:transport", "mst:fold",     "mst:los",
                                              "mst:images",  "mst:backproject", "mst:los_adjoint",
                                              "mst:replay",  "mst:combine",   "mst:replay2",  "mst:replay_list",
                                              "mst:event_adjoint", "mst:bmc"};

struct Phase {
    mst_grid* g;
    int phase;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    Phase(mst_grid* g_, int ph, cudaStream_t s) : g(g_), phase(ph), st(s) {
        nvtxRangePushA(kPhaseNames[ph]);
        if (g->prof && (a = prof_event(g)) != nullptr) cudaEventRecord(a, st);
    }
    ~Phase() {
        nvtxRangePop();
        if (!a) return;
        cudaEvent_t b = prof_event(g);
        if (!b) return;
        cudaEventRecord(b, st);
        g->prof_recs.push_back({phase, a, b});
    }
};

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

int check_params(mst_grid* g, const mst_params* p, bool photons) {
    if (!p) return fail(g, MST_ERR_INVALID_ARG, "params is NULL");
    if (!(p->albedo >= 0.0 && p->albedo <= 1.0)) return fail(g, MST_ERR_INVALID_ARG, "albedo must be in [0, 1]");
    if (!(p->g > -1.0 && p->g < 1.0)) return fail(g, MST_ERR_INVALID_ARG, "g must be in (-1, 1)");
    if (!(p->sun_zenith_rad >= 0.0 && p->sun_zenith_rad < 0.5 * M_PI))
        return fail(g, MST_ERR_INVALID_ARG, "sun zenith must be in [0, pi/2)");
    if (!std::isfinite(p->sun_azimuth_rad)) return fail(g, MST_ERR_INVALID_ARG, "sun azimuth must be finite");
    if (!(p->sun_irradiance >= 0.0 && std::isfinite(p->sun_irradiance)))
        return fail(g, MST_ERR_INVALID_ARG, "sun irradiance must be finite and >= 0");
    if (!(p->rr_threshold >= 0.0 && std::isfinite(p->rr_threshold)))
        return fail(g, MST_ERR_INVALID_ARG, "rr_threshold must be >= 0");
    if (!(p->rr_survival > 0.0 && p->rr_survival <= 1.0))
        return fail(g, MST_ERR_INVALID_ARG, "rr_survival must be in (0, 1]");
    if (p->grid_dtype < 0 || p->grid_dtype > 2) return fail(g, MST_ERR_INVALID_ARG, "unknown grid_dtype");
    if (p->estimator < 0 || p->estimator > 1) return fail(g, MST_ERR_INVALID_ARG, "unknown estimator");
    if (p->grad_mode < 0 || p->grad_mode > 1) return fail(g, MST_ERR_INVALID_ARG, "unknown grad_mode");
    if (p->conditioning < 0 || p->conditioning > 2) return fail(g, MST_ERR_INVALID_ARG, "unknown conditioning");
    if (!std::isfinite(p->reg_eta)) return fail(g, MST_ERR_INVALID_ARG, "reg_eta must be finite");
    if (photons) {
        if (p->n_photons == 0) return fail(g, MST_ERR_INVALID_ARG, "n_photons must be >= 1");
        if (p->n_photons > kMaxPhotons)
            return fail(g, MST_ERR_INVALID_ARG, "n_photons above the per-call limit (split the call)");
        if (p->max_events < 1) return fail(g, MST_ERR_INVALID_ARG, "max_events must be >= 1");
        if (p->max_order < 0) return fail(g, MST_ERR_INVALID_ARG, "max_order must be >= 0");
        if (p->n_photons_total != 0 && p->n_photons_total < p->n_photons)
            return fail(g, MST_ERR_INVALID_ARG, "n_photons_total must be 0 or >= n_photons");
    }
    return MST_OK;
}

TransportArgs transport_args(mst_grid* g, const mst_params* p) {
    TransportArgs a;
    std::memset(&a, 0, sizeof(a));
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
    a.beta_pad = g->ext_pad;
    a.beta_air = g->air;  // two species (Sec. 2): the particle of each event is drawn
    a.beta_aer = g->air ? g->beta_in : nullptr;
    a.albedo_air = (float)g->albedo_air;
    const double th = p->sun_zenith_rad, ph = p->sun_azimuth_rad;
    a.sun = make_float3((float)(-std::sin(th) * std::cos(ph)), (float)(-std::sin(th) * std::sin(ph)),
                        (float)(-std::cos(th)));
    const double N = (double)(p->n_photons_total ? p->n_photons_total : p->n_photons);
    const double I0 = p->sun_irradiance * std::cos(th) * (double)g->geo.ex * (double)g->geo.ey / N;
    a.albedo = (float)p->albedo;
    a.I0 = (float)I0;
    a.rr_below = (float)(p->rr_threshold * I0);
    a.rr_survival = (float)p->rr_survival;
    a.inv_rr_survival = (float)(1.0 / p->rr_survival);
    a.key = make_uint2((uint32_t)p->seed, (uint32_t)(p->seed >> 32));
    a.max_order = p->max_order;
    a.max_events = p->max_events;
    a.cp = g->cp;
    a.Lacc = g->Lacc;
    a.omega = g->omega;
    a.adj = g->adj;
    a.gacc = g->gacc;
    a.wbuf = g->wbuf;
    a.nevbuf = g->nevbuf;
    a.plist = g->plist;
    a.plist_n = g->score_cnt + 2 * kScoreBins;
    a.L64 = g->L64;
    a.g64 = g->g64;
    a.stats = g->stats;
    a.hash = g->dbg_hash;
    a.skip = g->dbg_skip;
    a.point = g->dbg_point;
    return a;
}

// Rolling-fold slicing of a tile of `bins` bins (see kFoldSweep): slices of a multiple of 32
// bins, at least 128, such that one sweep takes at most about kFoldSweep photons.
void set_fold(TransportArgs& a, uint64_t bins) {
    const uint64_t batches = kFoldSweep / kTicketBatch;
    uint64_t slice = (bins + batches - 1) / batches;
    slice = std::max<uint64_t>(128, (slice + 31) / 32 * 32);
    a.fold_bins = bins;
    a.fold_slice = (uint32_t)slice;
    a.fold_nslices = (uint32_t)((bins + slice - 1) / slice);
}

// Runs the photon transport. The forward render is one launch per kLaunchPhotons photons; the
// replay runs pass 1, the pass-2 list and pass 2 per kReplayChunk photons (the size of its
// per-photon buffers). The launches fold their FP32 tiles while they run; a last fold after each
// launch takes what is left. store_events (forward of a full gradient, one launch): the forward
// also stores its events and each photon's event count for the stored-event adjoint.
int run_photons(mst_grid* g, const mst_params* p, bool replay, double* cimg, cudaStream_t st,
                bool store_events = false) {
    TransportArgs a = transport_args(g, p);
    a.cimg = cimg;
    const uint64_t n = p->n_photons;
    const uint64_t span = replay ? kReplayChunk : kLaunchPhotons;
    const int nl = (int)((n + span - 1) / span);
    MST_CK(cudaMemsetAsync(g->tickets, 0, sizeof(unsigned int) * nl * (replay ? 2 : 1), st));
    const int est = replay ? 0 : p->estimator;
    // replay modes: 3 / 2 for the voxel estimator, 5 / 6 for the classic one (w_s from its images)
    const bool classic_adj = replay && p->estimator == MST_EST_CLASSIC;
    const int m_p1 = classic_adj ? 5 : 3, m_p2 = classic_adj ? 6 : 2;
    if (classic_adj) a.cres = g->resid;
    const int b_fwd = transport_blocks(g, p->grid_dtype, est);
    const int b_p1 = transport_blocks(g, p->grid_dtype, m_p1);
    const int b_p2 = transport_blocks(g, p->grid_dtype, m_p2);
    if (replay) set_fold(a, (uint64_t)g->geo.npad);
    else if (est == MST_EST_VOXEL) set_fold(a, (uint64_t)g->geo.nvox * g->cp);
    if (store_events) {
        a.evrec = g->evrec;
        a.ev_cap = g->ev_cap;
        a.ev_count = g->ev_count;
        a.ch_next = g->ch_next;
        a.warp_head = g->warp_head;
        g->ev_warps = (uint32_t)b_fwd * kTransportWarps;
        MST_CK(cudaMemsetAsync(g->ev_count, 0, sizeof(unsigned long long), st));
    }
    for (int l = 0; l < nl; ++l) {
        const uint64_t base = (uint64_t)l * span;
        a.first_id = p->photon_offset + base;
        a.out_base = (uint32_t)base;
        a.n = (uint32_t)((n - base) < span ? (n - base) : span);
        if (replay) {
            a.ticket = g->tickets + 2 * l;
            {
                Phase ph(g, MST_PH_REPLAY, st);
                MST_CK(launch_transport(g, a, p->grid_dtype, m_p1, b_p1, st));
            }
            {
                Phase ph(g, MST_PH_REPLAY_LIST, st);
                MST_CK(launch_score_list(g, a.n, st));
            }
            a.ticket = g->tickets + 2 * l + 1;
            {
                Phase ph(g, MST_PH_REPLAY2, st);
                MST_CK(launch_transport(g, a, p->grid_dtype, m_p2, b_p2, st));
            }
            Phase ph(g, MST_PH_FOLD, st);
            MST_CK(launch_fold_grad(g, st));
        } else {
            a.ticket = g->tickets + l;
            {
                Phase ph(g, MST_PH_TRANSPORT, st);
                MST_CK(launch_transport(g, a, p->grid_dtype, est, b_fwd, st));
            }
            if (est == MST_EST_VOXEL) {
                Phase ph(g, MST_PH_FOLD, st);
                MST_CK(launch_fold_L(g, st));
            }
        }
    }
    if (store_events) {  // the count reaches the host for the next call's sizing, without a wait
        MST_CK(cudaMemcpyAsync(g->ev_seen, g->ev_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        if (!g->capturing) {  // a batch graph instead records one event after each launch
            MST_CK(cudaEventRecord(g->ev_seen_ready, st));
            g->ev_seen_pending = true;
        }
    }
    return MST_OK;
}

// The replay of a call whose forward stored its events: W per photon from the stored events
// (replay pass 1 over all photons instead, on the device, when they did not fit), the list of
// photons with W != 0 over the whole call, and one pass-2 launch over it.
int run_replay_stored(mst_grid* g, const mst_params* p, cudaStream_t st) {
    TransportArgs a = transport_args(g, p);
    const uint64_t n = p->n_photons;
    set_fold(a, (uint64_t)g->geo.npad);
    a.evrec = g->evrec;
    a.ev_cap = g->ev_cap;
    a.ev_count = g->ev_count;
    a.wseq = g->wseq;
    a.evoff = g->evoff;
    a.ch_next = g->ch_next;
    a.warp_head = g->warp_head;
    a.n_warps = g->ev_warps;
    a.first_id = p->photon_offset;
    a.out_base = 0;
    a.n = (uint32_t)n;
    MST_CK(cudaMemsetAsync(g->tickets, 0, sizeof(unsigned int) * 3, st));
    MST_CK(cudaMemsetAsync(g->wbuf, 0, sizeof(double) * n, st));
    {
        Phase ph(g, MST_PH_EVENT_ADJOINT, st);
        MST_CK(launch_event_offsets(g, a.n, st));
        // the counts are spent: the adjoint leaves in them each photon's last event with w_s != 0
        MST_CK(cudaMemsetAsync(g->nevbuf, 0, sizeof(uint32_t) * n, st));
        a.ticket = g->tickets + 2;  // the adjoint's blocks take the forward warps' lists from it
        MST_CK(launch_event_adjoint(g, a, p->grid_dtype, st));
    }
    auto blocks = [&](int mode) { return transport_blocks(g, p->grid_dtype, mode); };
    a.ticket = g->tickets;
    {
        Phase ph(g, MST_PH_REPLAY, st);  // returns at once when the events fitted
        MST_CK(launch_transport(g, a, p->grid_dtype, 3, blocks(3), st));
    }
    {
        Phase ph(g, MST_PH_REPLAY_LIST, st);
        MST_CK(launch_score_list(g, a.n, st));
    }
    a.ticket = g->tickets + 1;
    {
        Phase ph(g, MST_PH_REPLAY2, st);  // on the stored w_s (mode 4), or recomputing them when they did not fit
        MST_CK(launch_transport(g, a, p->grid_dtype, 4, blocks(4), st));
        MST_CK(launch_transport(g, a, p->grid_dtype, 2, blocks(2), st));
    }
    Phase ph(g, MST_PH_FOLD, st);
    MST_CK(launch_fold_grad(g, st));
    return MST_OK;
}

// Per-photon buffers of the replay for n photons (at least kReplayChunk), allocated by the
// first full-gradient call that needs them and grown when a call needs more.
int ensure_replay(mst_grid* g, uint64_t n) {
    n = std::max<uint64_t>(n, kReplayChunk);
    if (g->wbuf && g->replay_cap >= n) return MST_OK;
    cudaFree(g->wbuf);
    cudaFree(g->nevbuf);
    cudaFree(g->plist);
    cudaFree(g->evoff);
    g->wbuf = nullptr;
    g->nevbuf = nullptr;
    g->plist = nullptr;
    g->evoff = nullptr;
    g->replay_cap = 0;
    if (cudaMalloc(&g->wbuf, n * 8) != cudaSuccess || cudaMalloc(&g->nevbuf, n * 4) != cudaSuccess ||
        cudaMalloc(&g->plist, n * sizeof(ScoreRec)) != cudaSuccess || cudaMalloc(&g->evoff, n * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(g->wbuf);
        cudaFree(g->nevbuf);
        cudaFree(g->plist);
        cudaFree(g->evoff);
        g->wbuf = nullptr;
        g->nevbuf = nullptr;
        g->plist = nullptr;
        g->evoff = nullptr;
        return fail(g, MST_ERR_OOM, "replay buffers: out of device memory");
    }
    g->replay_cap = n;
    return MST_OK;
}

// Whether the forward of a full-gradient call of n photons stores its events, with the buffer
// sized for them: room for 4 events per photon at first, then 1.25 x the events the last
// storing call offered (the handle's first count waited for, later ones read without a wait once
// their copy has landed), within the budget. Never
// fails the call: too many photons, no budget, a failed allocation or a call inside a stream
// capture (no allocation there) all mean W by replay.
bool ensure_records(mst_grid* g, uint64_t n, int dtype) {
    const uint64_t rec_bytes = (uint64_t)kEventBytes;
    if (g->capturing || n > kRecordMaxPhotons || g->rec_budget < rec_bytes * 1024) return false;
    if (!g->ev_count) {
        if (cudaMalloc(&g->ev_count, sizeof(unsigned long long)) != cudaSuccess ||
            cudaMallocHost(&g->ev_seen, sizeof(unsigned long long)) != cudaSuccess ||
            cudaEventCreateWithFlags(&g->ev_seen_ready, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    }
    unsigned long long seen = 0;
    if (g->ev_seen_pending) {
        // the first count of the handle is waited for (once: the first call's buffer came from a
        // guess); later ones are taken when they have arrived
        const cudaError_t q =
            g->ev_counted ? cudaEventQuery(g->ev_seen_ready) : cudaEventSynchronize(g->ev_seen_ready);
        if (q == cudaSuccess) {
            seen = *g->ev_seen;
            g->ev_seen_pending = false;
            g->ev_counted = true;
            g->ev_last = seen;
        } else {
            cudaGetLastError();  // not ready yet: size from the last count that arrived
        }
    }
    const uint64_t max_ev = std::min<uint64_t>(g->rec_budget / rec_bytes, 0xFFFFFFFFull);  // 32-bit slot indices
    // the forward reserves slots in per-warp chunks: one chunk per resident warp of headroom
    const uint64_t tails = (uint64_t)g->sm_count * transport_blocks_per_sm(dtype, 0, g->air != nullptr) *
                           kTransportWarps * kEventChunk;
    // need: the last count this handle's forward reserved (4 per photon before any), plus the
    // tails; a buffer below it is replaced by one 1.25 x the need, so that counts that drift by a
    // few chunks from call to call do not reallocate it every time
    const uint64_t need = std::min<uint64_t>(std::max<uint64_t>((g->ev_last ? g->ev_last : 4 * n) + tails, 1024), max_ev);
    uint64_t want = std::min<uint64_t>(need + need / 4, max_ev);
    if (!g->warp_head) {  // the forward's warps: at most kMaxWarpsPerSm per SM
        if (cudaMalloc(&g->warp_head, sizeof(uint32_t) * (size_t)g->sm_count * kMaxWarpsPerSm) != cudaSuccess) {
            cudaGetLastError();
            g->warp_head = nullptr;
            return false;
        }
    }
    if ((uint64_t)g->sm_count * transport_blocks_per_sm(dtype, 0, g->air != nullptr) * kTransportWarps >
        (uint64_t)g->sm_count * kMaxWarpsPerSm)
        return false;
    if (g->evrec && g->ev_cap >= need) return true;
    cudaFree(g->evrec);
    cudaFree(g->wseq);
    cudaFree(g->ch_next);
    g->evrec = nullptr;
    g->wseq = nullptr;
    g->ch_next = nullptr;
    g->ev_cap = 0;
    // leave a sixteenth of the device (at least 4 GiB) free for the call's other buffers, other
    // handles (a batch sizes all of its handles before it runs) and the caller: a buffer that
    // would not leave it is made smaller, and one below the need is not made (W by replay)
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const uint64_t reserve = std::max<uint64_t>(total_b / 16, 4ull << 30);
    want = std::min<uint64_t>(want, free_b > reserve ? (free_b - reserve) / rec_bytes : 0);
    if (want < need) return false;
    if (cudaMalloc(&g->evrec, want * kEventWords * 4) != cudaSuccess ||
        cudaMalloc(&g->wseq, want * sizeof(EventStep)) != cudaSuccess ||
        cudaMalloc(&g->ch_next, sizeof(uint32_t) * (want / kEventChunk + 1)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(g->evrec);
        cudaFree(g->wseq);
        cudaFree(g->ch_next);
        g->evrec = nullptr;
        g->wseq = nullptr;
        g->ch_next = nullptr;
        return false;
    }
    g->ev_cap = want;
    return true;
}

int ensure_q(mst_grid* g, int mode, cudaStream_t st) {
    if (mode == MST_COND_NONE) return MST_OK;
    if (!g->Qw) MST_CK(cudaMalloc(&g->Qw, sizeof(float) * (size_t)g->n_cams * g->geo.nvox));
    if (g->qw_mode != mode) {
        MST_CK(launch_ray_counts(g, g->Qw, mode, st));
        g->qw_mode = mode;
    }
    return MST_OK;
}

double rect_solid_angle(double x1, double x2, double y1, double y2) {
    auto F = [](double x, double y) { return std::atan(x * y / std::sqrt(1.0 + x * x + y * y)); };
    return F(x2, y2) - F(x1, y2) - F(x2, y1) + F(x1, y1);
}

double radical_inverse(int base, int i) {
    double f = 1.0, r = 0.0;
    while (i > 0) {
        f /= base;
        r += f * (i % base);
        i /= base;
    }
    return r;
}

void free_all(mst_grid* g) {
    void* ptrs[] = {g->ext, g->ext_pad, g->Lacc, g->L64, g->T, g->R, g->bacc, g->gT, g->adj, g->gacc, g->g64,
                    g->resid, g->cimg, g->lap, g->omega, g->Qw, g->stats, g->tickets, g->wbuf, g->nevbuf, g->plist, g->score_cnt};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    cudaFree(g->evrec);
    cudaFree(g->wseq);
    cudaFree(g->ch_next);
    cudaFree(g->warp_head);
    cudaFree(g->evoff);
    cudaFree(g->reg_wz);
    cudaFree(g->ch_beta);
    cudaFree(g->ch_grad);
    cudaFree(g->btot);
    cudaFree(g->btot_ref);
    cudaFree(g->ev_count);
    if (g->ev_seen) cudaFreeHost(g->ev_seen);
    if (g->ev_seen_ready) cudaEventDestroy(g->ev_seen_ready);
}

int check_render_grad(mst_grid* g, const float* beta, const mst_params* p, const double* meas, const double* grad);

// Two species: the FP32 totals beta + beta_air (and beta_ref + beta_air) of the surrogate.
int ensure_air_totals(mst_grid* g) {
    const size_t n = sizeof(float) * (size_t)g->geo.nvox;
    if (!g->btot && cudaMalloc(&g->btot, n) != cudaSuccess) {
        cudaGetLastError();
        return fail(g, MST_ERR_OOM, "air buffers: out of device memory");
    }
    if (!g->btot_ref && cudaMalloc(&g->btot_ref, n) != cudaSuccess) {
        cudaGetLastError();
        return fail(g, MST_ERR_OOM, "air buffers: out of device memory");
    }
    return MST_OK;
}

int render_grad_impl(mst_grid* g, const float* beta, const mst_params* p, const double* meas, const uint8_t* mask,
                     double* images, double* grad, double* loss, cudaStream_t st);

}  // namespace

extern "C" {

int mst_version(void) { return kVersion; }

void mst_default_params(mst_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->albedo = 0.99;
    p->g = 0.85;
    p->sun_irradiance = 1.0;
    p->rr_threshold = 0.01;
    p->rr_survival = 0.1;
    p->n_photons = 1000000;
    p->seed = 3;
    p->max_events = 100000;
    p->estimator = MST_EST_VOXEL;
    p->grid_dtype = MST_GRID_F32;
    p->grad_mode = MST_GRAD_SURROGATE;
    p->conditioning = MST_COND_NONE;
}

int mst_create_grid(const mst_grid_desc* d, int n_cams, const mst_camera* cams, int n_rays, mst_grid** out) {
    mst_grid* g = nullptr;
    if (!out) return MST_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d || !cams) return MST_ERR_INVALID_ARG;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return MST_ERR_INVALID_ARG;
    if ((long long)d->nx * d->ny * d->nz > (1ll << 30)) return MST_ERR_INVALID_ARG;
    if (d->nx > 2048 || d->ny > 2048 || d->nz > 1024) return MST_ERR_INVALID_ARG;  // packed voxel index
    if (!(d->dx > 0 && d->dy > 0 && d->dz > 0) || !std::isfinite(d->dx + d->dy + d->dz) || !finite3(d->origin))
        return MST_ERR_INVALID_ARG;
    if (n_cams < 1 || n_cams > MST_MAX_CAMERAS) return MST_ERR_INVALID_ARG;
    if (n_rays < 1 || n_rays > MST_MAX_SUBPIXEL_RAYS) return MST_ERR_INVALID_ARG;
    long long total_pix = 0;
    for (int c = 0; c < n_cams; ++c) {
        const mst_camera& cm = cams[c];
        if (cm.width < 1 || cm.height < 1 || !(cm.fov_x_rad > 0 && cm.fov_x_rad < M_PI) || !finite3(cm.pos))
            return MST_ERR_INVALID_ARG;
        // the camera may sit outside the grid, but within 1e6 voxels of it
        const double hh[3] = {d->dx, d->dy, d->dz};
        const int nn[3] = {d->nx, d->ny, d->nz};
        for (int a = 0; a < 3; ++a)
            if (std::fabs(cm.pos[a] - d->origin[a]) > (nn[a] + 1e6) * hh[a]) return MST_ERR_INVALID_ARG;
        for (int q = 0; q < 9; ++q)
            if (!std::isfinite(cm.rot[q])) return MST_ERR_INVALID_ARG;
        for (int u = 0; u < 3; ++u)
            for (int v = u; v < 3; ++v) {
                const double* A = cm.rot + 3 * u;
                const double* B = cm.rot + 3 * v;
                const double dot = A[0] * B[0] + A[1] * B[1] + A[2] * B[2];
                if (std::fabs(dot - (u == v ? 1.0 : 0.0)) > 1e-3) return MST_ERR_INVALID_ARG;
            }
        total_pix += (long long)cm.width * cm.height;
    }
    if (total_pix > (1ll << 30)) return MST_ERR_INVALID_ARG;
    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return MST_ERR_NO_DEVICE;
    if (cudaGetDevice(&dev) != cudaSuccess) return MST_ERR_NO_DEVICE;

    g = new mst_grid();
    g->device = dev;
    cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (g->sm_count < 1) g->sm_count = 1;
    Geo& geo = g->geo;
    geo.nx = d->nx; geo.ny = d->ny; geo.nz = d->nz;
    geo.hx = (float)d->dx; geo.hy = (float)d->dy; geo.hz = (float)d->dz;
    geo.ex = (float)(d->nx * d->dx); geo.ey = (float)(d->ny * d->dy); geo.ez = (float)(d->nz * d->dz);
    geo.nvox = d->nx * d->ny * d->nz;
    geo.max_steps = d->nx + d->ny + d->nz + 8;
    geo.p0 = d->nx + 2 * kHalo;
    geo.p01 = (d->nx + 2 * kHalo) * (d->ny + 2 * kHalo);
    geo.inv_p0 = (float)(1.0 / geo.p0);
    geo.inv_p01 = (float)(1.0 / geo.p01);
    geo.npad = geo.p01 * (d->nz + 2 * kHalo);
    for (int a = 0; a < 3; ++a) g->origin[a] = d->origin[a];
    g->voxel_volume = d->dx * d->dy * d->dz;
    g->n_cams = n_cams;
    g->cp = (n_cams + 3) / 4 * 4;
    g->n_rays = n_rays;
    g->cams.n = n_cams;
    int off = 0;
    for (int c = 0; c < n_cams; ++c) {
        const mst_camera& s = cams[c];
        Cam& t = g->cams.c[c];
        t.px = (float)(s.pos[0] - d->origin[0]);
        t.py = (float)(s.pos[1] - d->origin[1]);
        t.pz = (float)(s.pos[2] - d->origin[2]);
        // voxel holding the centre of projection (may be outside the grid) and the offset inside
        // it, in FP64 here so the device sees the camera to ~1e-6 m
        const double hh[3] = {d->dx, d->dy, d->dz};
        const int nn[3] = {d->nx, d->ny, d->nz};
        int iv[3];
        float lv[3];
        bool inside = true;
        for (int a = 0; a < 3; ++a) {
            const double x = s.pos[a] - d->origin[a];
            const double f = std::floor(x / hh[a]);
            iv[a] = (int)std::max(-1e9, std::min(1e9, f));
            double off = x - f * hh[a];
            off = std::min(std::max(off, 0.0), hh[a]);
            lv[a] = (float)off;
            if (iv[a] < 0 || iv[a] >= nn[a]) inside = false;
        }
        t.ix = iv[0]; t.iy = iv[1]; t.iz = iv[2];
        t.lx = lv[0]; t.ly = lv[1]; t.lz = lv[2];
        t.inside = inside ? 1 : 0;
        t.rx = (float)s.rot[0]; t.ry = (float)s.rot[1]; t.rz = (float)s.rot[2];
        t.ux = (float)s.rot[3]; t.uy = (float)s.rot[4]; t.uz = (float)s.rot[5];
        t.fx = (float)s.rot[6]; t.fy = (float)s.rot[7]; t.fz = (float)s.rot[8];
        const double tx = std::tan(0.5 * s.fov_x_rad);
        t.tx = (float)tx;
        t.ty = (float)(tx * s.height / s.width);
        t.w = s.width;
        t.h = s.height;
        t.pix_off = off;
        off += s.width * s.height;
    }
    g->total_pix = off;
    g->halton.n = n_rays;
    for (int r = 0; r < n_rays; ++r) {
        g->halton.a[r] = (float)radical_inverse(2, r + 1);
        g->halton.b[r] = (float)radical_inverse(3, r + 1);
    }

    const size_t nvox = (size_t)geo.nvox, C = (size_t)n_cams;
    struct A {
        void** p;
        size_t bytes;
    } allocs[] = {
        {&g->ext, nvox * 4},
        {&g->ext_pad, (size_t)geo.npad * 4},
        {(void**)&g->Lacc, nvox * g->cp * 4},
        {(void**)&g->L64, C * nvox * 8},
        {(void**)&g->T, C * nvox * 4},
        {(void**)&g->R, C * nvox * 4},
        {(void**)&g->bacc, C * nvox * 4},
        {(void**)&g->gT, C * nvox * 4},
        {(void**)&g->adj, nvox * g->cp * 4},
        {(void**)&g->gacc, (size_t)geo.npad * 4},
        {(void**)&g->score_cnt, (2 * kScoreBins + 1) * 4},
        {(void**)&g->g64, nvox * 8},
        {(void**)&g->resid, (size_t)off * 8},
        {(void**)&g->cimg, (size_t)off * 8},
        {(void**)&g->lap, nvox * 8},
        {(void**)&g->omega, (size_t)off * 4},
        {(void**)&g->stats, MST_NSTATS * 8 + 64},
        {(void**)&g->tickets, (size_t)kMaxTickets * 4},
    };
    for (auto& a : allocs) {
        if (cudaMalloc(a.p, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            free_all(g);
            delete g;
            return MST_ERR_OOM;
        }
    }
    // pixel solid angles for the classic estimator (exact rectangle formula, FP64 on the host)
    float* om = new float[off];
    for (int c = 0; c < n_cams; ++c) {
        const Cam& t = g->cams.c[c];
        const double tx = std::tan(0.5 * cams[c].fov_x_rad), ty = tx * t.h / t.w;
        for (int j = 0; j < t.h; ++j)
            for (int i = 0; i < t.w; ++i) {
                const double x1 = (2.0 * i / t.w - 1.0) * tx, x2 = (2.0 * (i + 1) / t.w - 1.0) * tx;
                const double y1 = (2.0 * j / t.h - 1.0) * ty, y2 = (2.0 * (j + 1) / t.h - 1.0) * ty;
                om[t.pix_off + j * t.w + i] = (float)rect_solid_angle(x1, x2, y1, y2);
            }
    }
    cudaError_t e = cudaMemcpy(g->omega, om, sizeof(float) * off, cudaMemcpyHostToDevice);
    delete[] om;
    if (e == cudaSuccess) e = cudaMemset(g->Lacc, 0, nvox * g->cp * 4);
    if (e == cudaSuccess) e = cudaMemset(g->gacc, 0, (size_t)geo.npad * 4);
    if (e == cudaSuccess) e = cudaMemset(g->stats, 0, MST_NSTATS * 8 + 64);
    if (e != cudaSuccess) {
        free_all(g);
        delete g;
        return MST_ERR_CUDA;
    }
    *out = g;
    return MST_OK;
}

void mst_destroy(mst_grid* g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
    free_all(g);
    delete g;
}

int mst_render(mst_grid* g, const float* beta, const mst_params* p, double* images, double* L, void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!beta) return fail(g, MST_ERR_INVALID_ARG, "beta is NULL");
    int rc = check_params(g, p, true);
    if (rc) return rc;
    if (p->estimator == MST_EST_CLASSIC && L) return fail(g, MST_ERR_INVALID_ARG, "L is not defined for the classic estimator");
    DeviceGuard dg(g->device);
    cudaStream_t st = as_stream(stream);
    prof_reset(g);
    g->beta_in = beta;
    {
        Phase ph(g, MST_PH_STAGE, st);
        MST_CK(launch_stage(g, beta, g->air, p->grid_dtype, st));
    }
    MST_CK(cudaMemsetAsync(g->stats, 0, MST_NSTATS * 8, st));
    const size_t nL = (size_t)g->n_cams * g->geo.nvox;
    if (p->estimator == MST_EST_CLASSIC) {
        if (!images) return MST_OK;
        MST_CK(cudaMemsetAsync(images, 0, sizeof(double) * g->total_pix, st));
        return run_photons(g, p, false, images, st);
    }
    MST_CK(cudaMemsetAsync(g->L64, 0, sizeof(double) * nL, st));
    rc = run_photons(g, p, false, nullptr, st);
    if (rc) return rc;
    if (L) MST_CK(cudaMemcpyAsync(L, g->L64, sizeof(double) * nL, cudaMemcpyDeviceToDevice, st));
    if (images) {
        {
            Phase ph(g, MST_PH_LOS, st);
            MST_CK(launch_los(g, p->grid_dtype, g->L64, nullptr, nullptr, beta, g->T, g->R, st));
        }
        {
            Phase ph(g, MST_PH_IMAGES, st);
            MST_CK(launch_images(g, g->R, images, nullptr, nullptr, nullptr, nullptr, st));
        }
    }
    return MST_OK;
}

int mst_render_bmc(mst_grid* g, const float* beta, const mst_params* p, uint32_t n_per_pixel, double* images,
                   double* var, void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!beta || !images) return fail(g, MST_ERR_INVALID_ARG, "beta and images are required");
    int rc = check_params(g, p, false);
    if (rc) return rc;
    if (n_per_pixel < 1) return fail(g, MST_ERR_INVALID_ARG, "n_per_pixel must be >= 1");
    if (p->max_events < 1) return fail(g, MST_ERR_INVALID_ARG, "max_events must be >= 1");
    if (p->max_order < 0) return fail(g, MST_ERR_INVALID_ARG, "max_order must be >= 0");
    if (g->air) return fail(g, MST_ERR_UNSUPPORTED, "backward Monte Carlo renders one species (mst_set_air is set)");
    DeviceGuard dg(g->device);
    cudaStream_t st = as_stream(stream);
    prof_reset(g);
    {
        Phase ph(g, MST_PH_STAGE, st);
        MST_CK(launch_stage(g, beta, nullptr, p->grid_dtype, st));
    }
    MST_CK(cudaMemsetAsync(g->stats, 0, MST_NSTATS * 8, st));
    MST_CK(cudaMemsetAsync(images, 0, sizeof(double) * g->total_pix, st));
    MST_CK(cudaMemsetAsync(g->resid, 0, sizeof(double) * g->total_pix, st));  // sum of squares
    Phase ph(g, MST_PH_BMC, st);
    MST_CK(launch_bmc(g, p, n_per_pixel, images, g->resid, var, st));
    return MST_OK;
}

int mst_render_grad(mst_grid* g, const float* beta, const mst_params* p, const double* meas, const uint8_t* mask,
                    double* images, double* grad, double* loss, void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    int rc = check_render_grad(g, beta, p, meas, grad);
    if (rc) return rc;
    DeviceGuard dg(g->device);
    prof_reset(g);
    return render_grad_impl(g, beta, p, meas, mask, images, grad, loss, as_stream(stream));
}

}  // extern "C"

namespace {

int check_render_grad(mst_grid* g, const float* beta, const mst_params* p, const double* meas, const double* grad) {
    if (!beta || !meas || !grad) return fail(g, MST_ERR_INVALID_ARG, "beta, images_meas and grad are required");
    const int rc = check_params(g, p, true);
    if (rc) return rc;
    if (p->estimator != MST_EST_VOXEL && p->grad_mode != MST_GRAD_FULL)
        return fail(g, MST_ERR_UNSUPPORTED, "the surrogate gradient needs the voxel estimator");
    return MST_OK;
}

// Forward render, loss and gradient of one handle, enqueued on st (Sec. 2.1.2, Sec. 3, Sec. 5).
int render_grad_impl(mst_grid* g, const float* beta, const mst_params* p, const double* meas, const uint8_t* mask,
                     double* images, double* grad, double* loss, cudaStream_t st) {
    int rc = MST_OK;
    const size_t nL = (size_t)g->n_cams * g->geo.nvox;
    double* lossp = loss ? loss : g->stats + MST_NSTATS;
    g->beta_in = beta;
    {
        Phase ph(g, MST_PH_STAGE, st);
        MST_CK(launch_stage(g, beta, g->air, p->grid_dtype, st));
    }
    MST_CK(cudaMemsetAsync(g->stats, 0, MST_NSTATS * 8, st));
    if (p->estimator == MST_EST_CLASSIC) {  // Eq. fle images, their loss, and the score replay
        MST_CK(cudaMemsetAsync(g->cimg, 0, sizeof(double) * g->total_pix, st));
        rc = run_photons(g, p, false, g->cimg, st);
        if (rc) return rc;
        MST_CK(cudaMemsetAsync(lossp, 0, sizeof(double), st));
        {
            Phase ph(g, MST_PH_IMAGES, st);
            MST_CK(launch_classic_residual(g, g->cimg, meas, mask, g->resid, lossp, st));
        }
        if (images)
            MST_CK(cudaMemcpyAsync(images, g->cimg, sizeof(double) * g->total_pix, cudaMemcpyDeviceToDevice, st));
        rc = ensure_replay(g, kReplayChunk);
        if (rc) return rc;
        MST_CK(cudaMemsetAsync(g->g64, 0, sizeof(double) * g->geo.nvox, st));
        rc = run_photons(g, p, true, nullptr, st);
        if (rc) return rc;
        {
            Phase ph(g, MST_PH_COMBINE, st);
            MST_CK(launch_combine_full(g, nullptr, g->g64, grad, st));
        }
        if (p->reg_eta != 0.0) {
            Phase ph(g, MST_PH_COMBINE, st);
            MST_CK(launch_regularizer(g, beta, p->reg_eta, g->lap, g->stats + MST_NSTATS + 1, lossp, grad, st));
        }
        return MST_OK;
    }
    MST_CK(cudaMemsetAsync(g->L64, 0, sizeof(double) * nL, st));
    // full gradient: the forward stores its events when they can be held (W without pass 1)
    bool stored = false;
    if (p->grad_mode == MST_GRAD_FULL) {
        if (g->capturing) {  // a batch graph: the buffers were sized before the capture
            stored = g->batch_stored;
        } else {
            stored = ensure_records(g, p->n_photons, p->grid_dtype);
            if (stored && ensure_replay(g, p->n_photons) != MST_OK) {
                stored = false;
                g->err.clear();
            }
        }
    }
    rc = run_photons(g, p, false, nullptr, st, stored);
    if (rc) return rc;
    {
        Phase ph(g, MST_PH_LOS, st);
        MST_CK(launch_los(g, p->grid_dtype, g->L64, nullptr, nullptr, beta, g->T, g->R, st));
    }
    MST_CK(cudaMemsetAsync(lossp, 0, sizeof(double), st));
    {
        Phase ph(g, MST_PH_IMAGES, st);
        MST_CK(launch_images(g, g->R, images, meas, mask, g->resid, lossp, st));
    }
    MST_CK(cudaMemsetAsync(g->bacc, 0, sizeof(float) * nL, st));
    {
        Phase ph(g, MST_PH_BACKPROJECT, st);
        MST_CK(launch_backproject(g, g->resid, g->bacc, st));
    }
    MST_CK(cudaMemsetAsync(g->gT, 0, sizeof(float) * nL, st));
    {
        Phase ph(g, MST_PH_LOS_ADJOINT, st);
        MST_CK(launch_los_adjoint(g, g->R, g->bacc, g->gT, st));
    }
    if (p->grad_mode == MST_GRAD_SURROGATE) {
        rc = ensure_q(g, p->conditioning, st);
        if (rc) return rc;
        {
            Phase ph(g, MST_PH_COMBINE, st);
            const float* bt = g->air ? g->btot : beta;  // two species: j = L / (beta + beta_air)
            MST_CK(launch_combine_surrogate(g, g->L64, nullptr, bt, bt, g->T, g->bacc, g->gT,
                                            p->conditioning ? g->Qw : nullptr, grad, st));
        }
    } else {
        rc = ensure_replay(g, stored ? p->n_photons : kReplayChunk);
        if (rc) return rc;
        {
            Phase ph(g, MST_PH_COMBINE, st);
            MST_CK(launch_adjoint_tiles(g, g->T, g->bacc, g->adj, st));
        }
        MST_CK(cudaMemsetAsync(g->g64, 0, sizeof(double) * g->geo.nvox, st));
        rc = stored ? run_replay_stored(g, p, st) : run_photons(g, p, true, nullptr, st);
        if (rc) return rc;
        {
            Phase ph(g, MST_PH_COMBINE, st);
            MST_CK(launch_combine_full(g, g->gT, g->g64, grad, st));
        }
    }
    if (p->reg_eta != 0.0) {
        Phase ph(g, MST_PH_COMBINE, st);
        MST_CK(launch_regularizer(g, beta, p->reg_eta, g->lap, g->stats + MST_NSTATS + 1, lossp, grad, st));
    }
    return MST_OK;
}

}  // namespace

extern "C" {

int mst_transmittance(mst_grid* g, const float* beta, int dtype, float* T, void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!beta || !T) return fail(g, MST_ERR_INVALID_ARG, "beta and T are required");
    if (dtype < 0 || dtype > 2) return fail(g, MST_ERR_INVALID_ARG, "unknown grid_dtype");
    DeviceGuard dg(g->device);
    cudaStream_t st = as_stream(stream);
    prof_reset(g);
    {
        Phase ph(g, MST_PH_STAGE, st);
        MST_CK(launch_stage(g, beta, nullptr, dtype, st));
    }
    {
        Phase ph(g, MST_PH_LOS, st);
        MST_CK(launch_los(g, dtype, nullptr, nullptr, nullptr, beta, T, nullptr, st));
    }
    return MST_OK;
}

int mst_form_images(mst_grid* g, const float* beta, int dtype, const double* L, double* images, void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!beta || !L || !images) return fail(g, MST_ERR_INVALID_ARG, "beta, L and images are required");
    if (dtype < 0 || dtype > 2) return fail(g, MST_ERR_INVALID_ARG, "unknown grid_dtype");
    DeviceGuard dg(g->device);
    cudaStream_t st = as_stream(stream);
    prof_reset(g);
    {
        Phase ph(g, MST_PH_STAGE, st);
        MST_CK(launch_stage(g, beta, nullptr, dtype, st));
    }
    {
        Phase ph(g, MST_PH_LOS, st);
        MST_CK(launch_los(g, dtype, L, nullptr, nullptr, beta, g->T, g->R, st));
    }
    {
        Phase ph(g, MST_PH_IMAGES, st);
        MST_CK(launch_images(g, g->R, images, nullptr, nullptr, nullptr, nullptr, st));
    }
    return MST_OK;
}

int mst_surrogate_grad(mst_grid* g, const float* beta, const double* L_ref, const float* beta_ref, const mst_params* p,
                       const double* meas, const uint8_t* mask, double* images, double* grad, double* loss,
                       void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!beta || !L_ref || !beta_ref || !meas || !grad)
        return fail(g, MST_ERR_INVALID_ARG, "beta, L_ref, beta_ref, images_meas and grad are required");
    int rc = check_params(g, p, false);
    if (rc) return rc;
    DeviceGuard dg(g->device);
    cudaStream_t st = as_stream(stream);
    prof_reset(g);
    const size_t nL = (size_t)g->n_cams * g->geo.nvox;
    double* lossp = loss ? loss : g->stats + MST_NSTATS;
    // two species: j = L_ref / (beta_ref + beta_air) and L = j (beta + beta_air); the terms of
    // the gradient are derivatives w.r.t. the total, which equal those w.r.t. the aerosol
    const float* bt = g->air ? g->btot : beta;
    const float* btr = g->air ? g->btot_ref : beta_ref;
    {
        Phase ph(g, MST_PH_STAGE, st);
        MST_CK(launch_stage(g, beta, g->air, p->grid_dtype, st));
        if (g->air) MST_CK(launch_add_air(g, beta_ref, g->air, g->btot_ref, st));
    }
    {
        Phase ph(g, MST_PH_LOS, st);
        MST_CK(launch_los(g, p->grid_dtype, L_ref, nullptr, btr, bt, g->T, g->R, st));
    }
    MST_CK(cudaMemsetAsync(lossp, 0, sizeof(double), st));
    {
        Phase ph(g, MST_PH_IMAGES, st);
        MST_CK(launch_images(g, g->R, images, meas, mask, g->resid, lossp, st));
    }
    MST_CK(cudaMemsetAsync(g->bacc, 0, sizeof(float) * nL, st));
    {
        Phase ph(g, MST_PH_BACKPROJECT, st);
        MST_CK(launch_backproject(g, g->resid, g->bacc, st));
    }
    MST_CK(cudaMemsetAsync(g->gT, 0, sizeof(float) * nL, st));
    {
        Phase ph(g, MST_PH_LOS_ADJOINT, st);
        MST_CK(launch_los_adjoint(g, g->R, g->bacc, g->gT, st));
    }
    rc = ensure_q(g, p->conditioning, st);
    if (rc) return rc;
    {
        Phase ph(g, MST_PH_COMBINE, st);
        MST_CK(launch_combine_surrogate(g, L_ref, nullptr, btr, bt, g->T, g->bacc, g->gT,
                                        p->conditioning ? g->Qw : nullptr, grad, st));
    }
    if (p->reg_eta != 0.0) {
        Phase ph(g, MST_PH_COMBINE, st);
        MST_CK(launch_regularizer(g, beta, p->reg_eta, g->lap, g->stats + MST_NSTATS + 1, lossp, grad, st));
    }
    return MST_OK;
}

int mst_sun_mask(mst_grid* g, double zenith, double azimuth, double radius, uint8_t* mask, void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!mask) return fail(g, MST_ERR_INVALID_ARG, "mask is NULL");
    if (!(radius >= 0.0 && radius <= M_PI)) return fail(g, MST_ERR_INVALID_ARG, "radius must be in [0, pi]");
    if (!std::isfinite(zenith) || !std::isfinite(azimuth))
        return fail(g, MST_ERR_INVALID_ARG, "sun angles must be finite");
    DeviceGuard dg(g->device);
    MST_CK(launch_sun_mask(g, zenith, azimuth, radius, mask, as_stream(stream)));
    return MST_OK;
}

int mst_ray_counts(mst_grid* g, float* Q, void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!Q) return fail(g, MST_ERR_INVALID_ARG, "Q is NULL");
    DeviceGuard dg(g->device);
    MST_CK(launch_ray_counts(g, Q, 0, as_stream(stream)));
    return MST_OK;
}

int mst_regularizer(mst_grid* g, const float* beta, double eta, double* psi, double* grad, void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!beta) return fail(g, MST_ERR_INVALID_ARG, "beta is NULL");
    if (!std::isfinite(eta)) return fail(g, MST_ERR_INVALID_ARG, "eta must be finite");
    DeviceGuard dg(g->device);
    double* ps = psi ? psi : g->stats + MST_NSTATS + 1;
    MST_CK(launch_regularizer(g, beta, eta, g->lap, ps, nullptr, grad, as_stream(stream)));
    return MST_OK;
}

int mst_set_debug(mst_grid* g, uint32_t* hash, const uint8_t* skip) {
    if (!g) return MST_ERR_INVALID_ARG;
    g->dbg_hash = hash;
    g->dbg_skip = skip;
    return MST_OK;
}

int mst_set_debug_points(mst_grid* g, float* points) {
    if (!g) return MST_ERR_INVALID_ARG;
    g->dbg_point = reinterpret_cast<float4*>(points);
    return MST_OK;
}

int mst_get_stats(mst_grid* g, double* out) {
    if (!g || !out) return MST_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    MST_CK(cudaDeviceSynchronize());
    MST_CK(cudaMemcpy(out, g->stats, sizeof(double) * MST_NSTATS, cudaMemcpyDeviceToHost));
    return MST_OK;
}

int mst_set_profiling(mst_grid* g, int enable) {
    if (!g) return MST_ERR_INVALID_ARG;
    g->prof = enable != 0;
    prof_reset(g);
    return MST_OK;
}

int mst_get_phase_times(mst_grid* g, double* ms, int* launches) {
    if (!g || !ms) return MST_ERR_INVALID_ARG;
    if (!g->prof) return fail(g, MST_ERR_INVALID_ARG, "profiling is off (mst_set_profiling)");
    DeviceGuard dg(g->device);
    MST_CK(cudaDeviceSynchronize());
    for (int i = 0; i < MST_NPHASES; ++i) {
        ms[i] = 0.0;
        if (launches) launches[i] = 0;
    }
    for (const auto& r : g->prof_recs) {
        float t = 0.f;
        MST_CK(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.phase] += (double)t;
        if (launches) launches[r.phase] += 1;
    }
    return MST_OK;
}

int mst_set_reg_weights(mst_grid* g, const double* wz) {
    if (!g) return MST_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    if (!wz) {
        if (g->reg_wz) {
            MST_CK(cudaDeviceSynchronize());
            cudaFree(g->reg_wz);
            g->reg_wz = nullptr;
        }
        return MST_OK;
    }
    for (int z = 0; z < g->geo.nz; ++z)
        if (!std::isfinite(wz[z])) return fail(g, MST_ERR_INVALID_ARG, "altitude weights must be finite");
    if (!g->reg_wz) MST_CK(cudaMalloc(&g->reg_wz, sizeof(double) * g->geo.nz));
    MST_CK(cudaMemcpy(g->reg_wz, wz, sizeof(double) * g->geo.nz, cudaMemcpyHostToDevice));
    return MST_OK;
}

int mst_set_air(mst_grid* g, const float* beta_air, double albedo_air) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!(albedo_air >= 0.0 && albedo_air <= 1.0)) return fail(g, MST_ERR_INVALID_ARG, "albedo_air must be in [0, 1]");
    if (beta_air) {
        const int rc = ensure_air_totals(g);
        if (rc) return rc;
    }
    g->air = beta_air;
    g->albedo_air = albedo_air;
    return MST_OK;
}

int mst_render_grad_channels(mst_grid* g, const float* beta, int n, const mst_channel* ch, const uint8_t* mask,
                             double eta, double* grad, double* loss, void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!beta || !ch || !grad) return fail(g, MST_ERR_INVALID_ARG, "beta, channels and grad are required");
    if (n < 1 || n > MST_MAX_CHANNELS) return fail(g, MST_ERR_INVALID_ARG, "n_channels must be in 1..MST_MAX_CHANNELS");
    if (!std::isfinite(eta)) return fail(g, MST_ERR_INVALID_ARG, "eta must be finite");
    const float* air0 = g->air;
    const double alb0 = g->albedo_air;
    for (int i = 0; i < n; ++i) {
        const std::string tag = "channel " + std::to_string(i) + ": ";
        if (!(ch[i].sigma_ratio > 0.0 && std::isfinite(ch[i].sigma_ratio)))
            return fail(g, MST_ERR_INVALID_ARG, tag + "sigma_ratio must be finite and > 0");
        if (!(ch[i].albedo_air >= 0.0 && ch[i].albedo_air <= 1.0))
            return fail(g, MST_ERR_INVALID_ARG, tag + "albedo_air must be in [0, 1]");
        if (ch[i].beta_air_dev) {
            const int rc = ensure_air_totals(g);
            if (rc) return rc;
        }
        const int rc = check_render_grad(g, beta, &ch[i].params, ch[i].images_meas_dev, grad);
        if (rc) return fail(g, rc, tag + g->err);
    }
    DeviceGuard dg(g->device);
    cudaStream_t st = as_stream(stream);
    prof_reset(g);
    const size_t nvox = (size_t)g->geo.nvox;
    if (!g->ch_beta && cudaMalloc(&g->ch_beta, sizeof(float) * nvox) != cudaSuccess) {
        cudaGetLastError();
        return fail(g, MST_ERR_OOM, "channel buffers: out of device memory");
    }
    if (!g->ch_grad && cudaMalloc(&g->ch_grad, sizeof(double) * nvox) != cudaSuccess) {
        cudaGetLastError();
        return fail(g, MST_ERR_OOM, "channel buffers: out of device memory");
    }
    double* lossp = loss ? loss : g->stats + MST_NSTATS + 2;  // slots past the statistics: scratch
    double* loss_mu = g->stats + MST_NSTATS + 3;
    MST_CK(cudaMemsetAsync(grad, 0, sizeof(double) * nvox, st));
    MST_CK(cudaMemsetAsync(lossp, 0, sizeof(double), st));
    int rc = MST_OK;
    for (int i = 0; i < n && rc == MST_OK; ++i) {
        if (launch_channel_beta(g, beta, ch[i].sigma_ratio, g->ch_beta, st) != cudaSuccess) {
            rc = fail(g, MST_ERR_CUDA, "launch_channel_beta failed");
            break;
        }
        g->air = ch[i].beta_air_dev;
        g->albedo_air = ch[i].albedo_air;
        mst_params pc = ch[i].params;
        pc.reg_eta = 0.0;
        rc = render_grad_impl(g, g->ch_beta, &pc, ch[i].images_meas_dev, mask, ch[i].images_dev, g->ch_grad, loss_mu,
                              st);
        if (rc == MST_OK && launch_channel_add(g, grad, ch[i].sigma_ratio, g->ch_grad, lossp, loss_mu, st) != cudaSuccess)
            rc = fail(g, MST_ERR_CUDA, "launch_channel_add failed");
    }
    g->air = air0;
    g->albedo_air = alb0;
    if (rc) return rc;
    if (eta != 0.0) {
        Phase ph(g, MST_PH_COMBINE, st);
        MST_CK(launch_regularizer(g, beta, eta, g->lap, g->stats + MST_NSTATS + 1, lossp, grad, st));
    }
    return MST_OK;
}

int mst_set_wavefront(mst_grid* g, int forward_trip, int forward_blocks, int replay_trip, int replay_blocks) {
    if (!g) return MST_ERR_INVALID_ARG;
    const bool ft = forward_trip == 0 || forward_trip == 8 || forward_trip == 10 || forward_trip == 12 ||
                    forward_trip == 16;
    const bool rt = replay_trip == 0 || replay_trip == 4 || replay_trip == 6 || replay_trip == 8 || replay_trip == 10;
    if (!ft || !rt || forward_blocks < 0 || forward_blocks > 8 || replay_blocks < 0 || replay_blocks > 8)
        return fail(g, MST_ERR_INVALID_ARG,
                    "forward trip in {0, 8, 10, 12, 16}, pass-2 trip in {0, 4, 6, 8, 10}, blocks per SM in 0..8");
    g->wf_trip[0] = forward_trip;  // forward, voxel estimator (the classic one keeps its defaults)
    g->wf_blocks[0] = forward_blocks;
    for (int m : {2, 4}) {  // replay pass 2, recomputing or reading the stored w_s
        g->wf_trip[m] = replay_trip;
        g->wf_blocks[m] = replay_blocks;
    }
    return MST_OK;
}

int mst_autotune(mst_grid* g, const float* beta, const mst_params* p, uint64_t n_sample, int* choice, void* stream) {
    if (!g) return MST_ERR_INVALID_ARG;
    if (!beta || !choice) return fail(g, MST_ERR_INVALID_ARG, "beta and choice are required");
    int rc = check_params(g, p, false);
    if (rc) return rc;
    if (n_sample < 65536 || n_sample > kRecordMaxPhotons)
        return fail(g, MST_ERR_INVALID_ARG, "n_sample must be in [2^16, 2^27]");
    DeviceGuard dg(g->device);
    cudaStream_t st = as_stream(stream);
    mst_params q = *p;  // a full-gradient call of the voxel estimator on the sample, against zero images
    q.n_photons = n_sample;
    q.n_photons_total = 0;
    q.photon_offset = 0;
    q.estimator = MST_EST_VOXEL;
    q.grad_mode = MST_GRAD_FULL;
    q.reg_eta = 0.0;
    double *meas = nullptr, *grad = nullptr, *loss = nullptr;
    if (cudaMalloc(&meas, sizeof(double) * g->total_pix) != cudaSuccess ||
        cudaMalloc(&grad, sizeof(double) * g->geo.nvox) != cudaSuccess || cudaMalloc(&loss, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(meas);
        cudaFree(grad);
        return fail(g, MST_ERR_OOM, "autotune buffers: out of device memory");
    }
    MST_CK(cudaMemsetAsync(meas, 0, sizeof(double) * g->total_pix, st));
    const bool prof0 = g->prof;
    // the sample's event counts must not size the buffers of the handle's real calls
    const unsigned long long ev_last0 = g->ev_last;
    const bool ev_counted0 = g->ev_counted;
    const int saved_trip[7] = {g->wf_trip[0], 0, g->wf_trip[2], 0, g->wf_trip[4], 0, 0};
    const int saved_blocks[7] = {g->wf_blocks[0], 0, g->wf_blocks[2], 0, g->wf_blocks[4], 0, 0};
    const int occ_f = transport_blocks_per_sm(q.grid_dtype, 0, g->air != nullptr);
    const int occ_r = transport_blocks_per_sm(q.grid_dtype, 4, g->air != nullptr);
    // candidates: voxels per trip around the defaults, at full occupancy and one block less
    std::vector<std::pair<int, int>> cf, cr;
    for (int t : {8, 10, 12, 16})
        for (int b = occ_f; b >= std::max(1, occ_f - 1); --b) cf.push_back({t, b});
    for (int t : {4, 6, 8, 10})
        for (int b = occ_r; b >= std::max(1, occ_r - 1); --b) cr.push_back({t, b});
    std::vector<double> tf(cf.size(), 1e30), tr(cr.size(), 1e30);
    g->prof = true;
    auto run = [&](double& ms_f, double& ms_r) -> int {  // one timed call: forward and pass-2 phases
        prof_reset(g);
        int e = render_grad_impl(g, beta, &q, meas, nullptr, nullptr, grad, loss, st);
        if (e) return e;
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail(g, MST_ERR_CUDA, "autotune: stream error");
        ms_f = ms_r = 0.0;
        for (const auto& pr : g->prof_recs) {
            float t = 0.f;
            cudaEventElapsedTime(&t, pr.a, pr.b);
            if (pr.phase == MST_PH_TRANSPORT) ms_f += t;
            if (pr.phase == MST_PH_REPLAY2) ms_r += t;
        }
        return MST_OK;
    };
    double wf = 0.0, wr = 0.0;
    rc = run(wf, wr);  // warm-up (buffers sized, kernels loaded)
    const size_t n = std::max(cf.size(), cr.size());
    for (size_t i = 0; i < n && rc == MST_OK; ++i) {  // forward and pass-2 candidates paired in one call
        const size_t jf = i % cf.size(), jr = i % cr.size();
        rc = mst_set_wavefront(g, cf[jf].first, cf[jf].second, cr[jr].first, cr[jr].second);
        for (int rep = 0; rep < 2 && rc == MST_OK; ++rep) {
            double ms_f = 0.0, ms_r = 0.0;
            rc = run(ms_f, ms_r);
            tf[jf] = std::min(tf[jf], ms_f);
            tr[jr] = std::min(tr[jr], ms_r);
        }
    }
    g->prof = prof0;
    prof_reset(g);
    g->ev_last = ev_last0;
    g->ev_counted = ev_counted0;
    g->ev_seen_pending = false;  // a count pending from before was overwritten by the sample's
    cudaFree(meas);
    cudaFree(grad);
    cudaFree(loss);
    if (rc) {  // keep the setting the handle had
        for (int m : {0, 2, 4}) {
            g->wf_trip[m] = saved_trip[m];
            g->wf_blocks[m] = saved_blocks[m];
        }
        return rc;
    }
    const size_t bf = std::min_element(tf.begin(), tf.end()) - tf.begin();
    const size_t br = std::min_element(tr.begin(), tr.end()) - tr.begin();
    rc = mst_set_wavefront(g, cf[bf].first, cf[bf].second, cr[br].first, cr[br].second);
    choice[0] = cf[bf].first;
    choice[1] = cf[bf].second;
    choice[2] = cr[br].first;
    choice[3] = cr[br].second;
    return rc;
}

int mst_set_replay_memory(mst_grid* g, uint64_t bytes) {
    if (!g) return MST_ERR_INVALID_ARG;
    g->rec_budget = bytes;
    if (g->evrec && g->ev_cap * (uint64_t)kEventBytes > bytes) {  // shrink to the new budget at the next call
        DeviceGuard dg(g->device);
        MST_CK(cudaDeviceSynchronize());
        cudaFree(g->evrec);
        cudaFree(g->wseq);
        cudaFree(g->ch_next);
        g->evrec = nullptr;
        g->wseq = nullptr;
        g->ch_next = nullptr;
        g->ev_cap = 0;
    }
    return MST_OK;
}

int mst_sync(mst_grid* g) {
    if (!g) return MST_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    MST_CK(cudaDeviceSynchronize());
    MST_CK(cudaGetLastError());
    return MST_OK;
}

const char* mst_last_error(mst_grid* g) { return g ? g->err.c_str() : "null handle"; }

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Batched scenes: one CUDA graph holds the forward + gradient sequences of n handles, each on
// its own branch, so independent scenes of uneven size overlap on the GPU and the whole batch
// costs one graph launch. The graph is captured on the first call and replayed while every
// pointer and parameter stays the same; any change re-captures it.

struct mst_batch {
    int n = 0;
    int device = 0;
    std::vector<mst_grid*> grids;
    std::vector<cudaStream_t> branch;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
    cudaEvent_t done = nullptr;  // after the last graph launch: the handles' event counts have landed
    bool launched = false;
    std::string err;
    // the persistent form: the photon transport of all scenes in single launches
    int form = MST_BATCH_BRANCHES;    // requested form
    bool persistent = false;          // form of the captured graph
    int trip_fwd = 0, blocks_fwd = 0, trip_p2 = 0, blocks_p2 = 0;  // its wavefront (0: defaults)
    TransportArgs* tables = nullptr;  // device [4][n]: forward, event adjoint, pass 1, pass 2
};

namespace {

void batch_free(mst_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->tables) cudaFree(b->tables);
    for (cudaStream_t s : b->branch)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->cap) cudaStreamDestroy(b->cap);
}

template <typename T>
void key_add(std::vector<unsigned char>& k, const T& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    k.insert(k.end(), p, p + sizeof(T));
}

// blocks of a persistent batch launch of a transport mode (per_sm 0: the register budget's occupancy)
int batch_launch_blocks(const mst_batch* b, int mode, int per_sm) {
    const int occ = transport_batch_blocks_per_sm(mode);
    return b->grids[0]->sm_count * (per_sm > 0 && per_sm < occ ? per_sm : occ);
}

// Whether every scene of the call can run in the persistent form: the voxel estimator's full
// gradient with the forward's events stored (buffers sized before the capture), FP32 grid, one
// species. Otherwise the batch keeps one graph branch per scene.
bool persistent_ok(const mst_batch* b, const mst_params* params) {
    if (b->form != MST_BATCH_PERSISTENT) return false;
    for (int i = 0; i < b->n; ++i) {
        const mst_grid* g = b->grids[i];
        const mst_params& p = params[i];
        if (p.estimator != MST_EST_VOXEL || p.grad_mode != MST_GRAD_FULL || p.grid_dtype != MST_GRID_F32 ||
            g->air || !g->batch_stored || p.n_photons > kRecordMaxPhotons)
            return false;
    }
    return true;
}

// Arguments of the persistent launches, one per scene and launch, as mst_render_grad builds them
// for one handle (forward storing its events; event adjoint, pass 1 and pass 2 with their tickets).
int persistent_tables(mst_batch* b, const float* const* betas, const mst_params* params) {
    const int n = b->n;
    std::vector<TransportArgs> t(4 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        mst_grid* g = b->grids[i];
        const mst_params* p = &params[i];
        g->beta_in = betas[i];
        TransportArgs f = transport_args(g, p);
        set_fold(f, (uint64_t)g->geo.nvox * g->cp);
        f.evrec = g->evrec;
        f.ev_cap = g->ev_cap;
        f.ev_count = g->ev_count;
        f.ch_next = g->ch_next;
        f.warp_head = g->warp_head;
        g->ev_warps = (uint32_t)batch_launch_blocks(b, 0, b->blocks_fwd) * kTransportWarps;
        f.first_id = p->photon_offset;
        f.out_base = 0;
        f.n = (uint32_t)p->n_photons;
        f.ticket = g->tickets;
        t[i] = f;
        TransportArgs r = transport_args(g, p);
        set_fold(r, (uint64_t)g->geo.npad);
        r.evrec = g->evrec;
        r.ev_cap = g->ev_cap;
        r.ev_count = g->ev_count;
        r.wseq = g->wseq;
        r.evoff = g->evoff;
        r.ch_next = g->ch_next;
        r.warp_head = g->warp_head;
        r.n_warps = g->ev_warps;
        r.first_id = p->photon_offset;
        r.out_base = 0;
        r.n = (uint32_t)p->n_photons;
        r.ticket = g->tickets + 2;  // the event adjoint's blocks take the forward warps' lists from it
        t[n + i] = r;
        r.ticket = g->tickets;      // pass 1 (returns at once when the events fitted)
        t[2 * n + i] = r;
        r.ticket = g->tickets + 1;  // pass 2
        t[3 * n + i] = r;
    }
    if (!b->tables && cudaMalloc(&b->tables, sizeof(TransportArgs) * t.size()) != cudaSuccess) {
        cudaGetLastError();
        b->tables = nullptr;
        b->err = "batch tables: out of device memory";
        return MST_ERR_OOM;
    }
    if (cudaMemcpy(b->tables, t.data(), sizeof(TransportArgs) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        b->err = "batch tables: copy failed";
        return MST_ERR_CUDA;
    }
    return MST_OK;
}

// The persistent form of one batch call, enqueued while the capture stream records: each scene's
// small kernels run on its own branch (the steps of mst_render_grad for one handle, in order),
// and the photon transport, the stored-event adjoint and both replay passes of all scenes run as
// single persistent launches on the capture stream between them.
int persistent_sequence(mst_batch* b, const float* const* betas, const mst_params* params, const double* const* meas,
                        const uint8_t* const* masks, double* const* images, double* const* grads, double* losses) {
    const int n = b->n;
    mst_grid* g = nullptr;  // the scene in hand, for the error messages of MST_CK
    cudaStream_t cap = b->cap;
    const TransportArgs* t_fwd = b->tables;
    const TransportArgs* t_adj = b->tables + n;
    const TransportArgs* t_p1 = b->tables + 2 * n;
    const TransportArgs* t_p2 = b->tables + 3 * n;
    auto fork = [&]() {
        cudaEventRecord(b->fork, cap);
        for (int i = 0; i < n; ++i) cudaStreamWaitEvent(b->branch[i], b->fork, 0);
    };
    auto join = [&]() {
        for (int i = 0; i < n; ++i) {
            cudaEventRecord(b->join[i], b->branch[i]);
            cudaStreamWaitEvent(cap, b->join[i], 0);
        }
    };
    const int sm = b->grids[0]->sm_count;
    auto blocks = [&](int mode, int per_sm) { return batch_launch_blocks(b, mode, per_sm); };
    // 1. staging and the counters of the forward
    fork();
    for (int i = 0; i < n; ++i) {
        g = b->grids[i];
        cudaStream_t st = b->branch[i];
        g->beta_in = betas[i];
        MST_CK(launch_stage(g, betas[i], nullptr, MST_GRID_F32, st));
        MST_CK(cudaMemsetAsync(g->stats, 0, MST_NSTATS * 8, st));
        MST_CK(cudaMemsetAsync(g->L64, 0, sizeof(double) * (size_t)g->n_cams * g->geo.nvox, st));
        MST_CK(cudaMemsetAsync(g->tickets, 0, sizeof(unsigned int), st));
        MST_CK(cudaMemsetAsync(g->ev_count, 0, sizeof(unsigned long long), st));
    }
    join();
    g = b->grids[0];
    MST_CK(launch_transport_batch(t_fwd, n, 0, b->trip_fwd, blocks(0, b->blocks_fwd), cap));
    // 2. L, images, loss, back-projection, LOS adjoint, adjoint tiles, the event slots
    fork();
    for (int i = 0; i < n; ++i) {
        g = b->grids[i];
        cudaStream_t st = b->branch[i];
        const size_t nL = (size_t)g->n_cams * g->geo.nvox;
        const uint64_t np = params[i].n_photons;
        double* lossp = losses + i;
        MST_CK(launch_fold_L(g, st));
        MST_CK(cudaMemcpyAsync(g->ev_seen, g->ev_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        MST_CK(launch_los(g, MST_GRID_F32, g->L64, nullptr, nullptr, betas[i], g->T, g->R, st));
        MST_CK(cudaMemsetAsync(lossp, 0, sizeof(double), st));
        MST_CK(launch_images(g, g->R, images ? images[i] : nullptr, meas[i], masks ? masks[i] : nullptr, g->resid,
                             lossp, st));
        MST_CK(cudaMemsetAsync(g->bacc, 0, sizeof(float) * nL, st));
        MST_CK(launch_backproject(g, g->resid, g->bacc, st));
        MST_CK(cudaMemsetAsync(g->gT, 0, sizeof(float) * nL, st));
        MST_CK(launch_los_adjoint(g, g->R, g->bacc, g->gT, st));
        MST_CK(launch_adjoint_tiles(g, g->T, g->bacc, g->adj, st));
        MST_CK(cudaMemsetAsync(g->g64, 0, sizeof(double) * g->geo.nvox, st));
        MST_CK(cudaMemsetAsync(g->tickets, 0, sizeof(unsigned int) * 3, st));
        MST_CK(cudaMemsetAsync(g->wbuf, 0, sizeof(double) * np, st));
        MST_CK(launch_event_offsets(g, (uint32_t)np, st));
        MST_CK(cudaMemsetAsync(g->nevbuf, 0, sizeof(uint32_t) * np, st));
    }
    join();
    g = b->grids[0];
    MST_CK(launch_event_adjoint_batch(t_adj, n, sm * 8, cap));
    MST_CK(launch_transport_batch(t_p1, n, 3, 0, blocks(3, 0), cap));  // only scenes whose events overflowed
    // 3. the pass-2 lists
    fork();
    for (int i = 0; i < n; ++i) {
        g = b->grids[i];
        MST_CK(launch_score_list(g, (uint32_t)params[i].n_photons, b->branch[i]));
    }
    join();
    g = b->grids[0];
    MST_CK(launch_transport_batch(t_p2, n, 4, b->trip_p2, blocks(4, b->blocks_p2), cap));
    MST_CK(launch_transport_batch(t_p2, n, 2, 0, blocks(2, 0), cap));  // only scenes whose events overflowed
    // 4. gradient: fold, W^T term, regulariser
    fork();
    for (int i = 0; i < n; ++i) {
        g = b->grids[i];
        cudaStream_t st = b->branch[i];
        MST_CK(launch_fold_grad(g, st));
        MST_CK(launch_combine_full(g, g->gT, g->g64, grads[i], st));
        if (params[i].reg_eta != 0.0)
            MST_CK(launch_regularizer(g, betas[i], params[i].reg_eta, g->lap, g->stats + MST_NSTATS + 1, losses + i,
                                      grads[i], st));
    }
    join();
    return MST_OK;
}

}  // namespace

extern "C" {

int mst_batch_create(int n, mst_grid* const* grids, mst_batch** out) {
    if (!out) return MST_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || n > MST_MAX_BATCH || !grids) return MST_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!grids[i] || grids[i]->device != grids[0]->device) return MST_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (grids[j] == grids[i]) return MST_ERR_INVALID_ARG;  // each scene needs its own scratch
    }
    mst_batch* b = new mst_batch();
    b->n = n;
    b->device = grids[0]->device;
    b->grids.assign(grids, grids + n);
    DeviceGuard dg(b->device);
    bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
    b->branch.assign(n, nullptr);
    b->join.assign(n, nullptr);
    for (int i = 0; ok && i < n; ++i)
        ok = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        delete b;
        return MST_ERR_CUDA;
    }
    *out = b;
    return MST_OK;
}

void mst_batch_destroy(mst_batch* b) {
    if (!b) return;
    DeviceGuard dg(b->device);
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
}

const char* mst_batch_last_error(mst_batch* b) { return b ? b->err.c_str() : "null batch"; }

int mst_batch_set_form(mst_batch* b, int form) {
    if (!b) return MST_ERR_INVALID_ARG;
    if (form != MST_BATCH_BRANCHES && form != MST_BATCH_PERSISTENT) {
        b->err = "form must be MST_BATCH_BRANCHES or MST_BATCH_PERSISTENT";
        return MST_ERR_INVALID_ARG;
    }
    b->form = form;
    return MST_OK;
}

int mst_batch_get_form(mst_batch* b) { return b ? (b->persistent ? MST_BATCH_PERSISTENT : MST_BATCH_BRANCHES) : -1; }

int mst_batch_set_wavefront(mst_batch* b, int forward_trip, int forward_blocks, int replay_trip, int replay_blocks) {
    if (!b) return MST_ERR_INVALID_ARG;
    const bool ft = forward_trip == 0 || forward_trip == 8 || forward_trip == 10 || forward_trip == 12 ||
                    forward_trip == 16;
    const bool rt = replay_trip == 0 || replay_trip == 4 || replay_trip == 6 || replay_trip == 8 || replay_trip == 10;
    if (!ft || !rt || forward_blocks < 0 || forward_blocks > 8 || replay_blocks < 0 || replay_blocks > 8) {
        b->err = "forward trip in {0, 8, 10, 12, 16}, pass-2 trip in {0, 4, 6, 8, 10}, blocks per SM in 0..8";
        return MST_ERR_INVALID_ARG;
    }
    b->trip_fwd = forward_trip == 12 ? 0 : forward_trip;  // 12 and 6 are the kernels' defaults
    b->blocks_fwd = forward_blocks;
    b->trip_p2 = replay_trip == 6 ? 0 : replay_trip;
    b->blocks_p2 = replay_blocks;
    return MST_OK;
}

int mst_batch_autotune(mst_batch* b, const float* const* betas, const mst_params* params, const double* const* meas,
                       int sample_div, int* choice, void* stream) {
    if (!b) return MST_ERR_INVALID_ARG;
    if (!betas || !params || !meas || !choice || sample_div < 1) {
        b->err = "betas, params, images_meas and choice are required, sample_div >= 1";
        return MST_ERR_INVALID_ARG;
    }
    const int n = b->n;
    DeviceGuard dg(b->device);
    cudaStream_t st = as_stream(stream);
    // the sample: each scene's photons divided by sample_div, no regulariser, images not returned
    std::vector<mst_params> q(params, params + n);
    for (auto& x : q) {
        x.n_photons = std::max<uint64_t>(1, x.n_photons / (uint64_t)sample_div);
        x.n_photons_total = 0;
        x.reg_eta = 0.0;
    }
    std::vector<double*> grads(n, nullptr);
    double* losses = nullptr;
    bool ok = cudaMalloc(&losses, sizeof(double) * n) == cudaSuccess;
    for (int i = 0; i < n && ok; ++i) ok = cudaMalloc(&grads[i], sizeof(double) * b->grids[i]->geo.nvox) == cudaSuccess;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ok = ok && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    std::vector<unsigned long long> ev_last0(n);
    std::vector<char> ev_counted0(n);
    for (int i = 0; i < n; ++i) {
        ev_last0[i] = b->grids[i]->ev_last;
        ev_counted0[i] = b->grids[i]->ev_counted;
    }
    const int saved[4] = {b->trip_fwd, b->blocks_fwd, b->trip_p2, b->blocks_p2};
    int rc = ok ? MST_OK : MST_ERR_OOM;
    if (!ok) b->err = "autotune buffers: out of device memory";
    auto timed = [&](double& ms) -> int {  // best of two sample calls (one graph launch each)
        ms = 1e30;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, st);
            const int e = mst_batch_render_grad(b, betas, q.data(), meas, nullptr, nullptr, grads.data(), losses, st);
            if (e) return e;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return MST_ERR_CUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, (double)t);
        }
        return MST_OK;
    };
    // one axis at a time: the forward's trip and blocks, then pass 2's
    int best[4] = {12, 0, 6, 0};
    double ms = 0.0;
    if (rc == MST_OK) rc = mst_batch_set_wavefront(b, 12, 0, 6, 0);
    if (rc == MST_OK) rc = timed(ms);  // warm-up: buffers sized, graph captured
    const int occ_f = transport_batch_blocks_per_sm(0);
    const int occ_r = transport_batch_blocks_per_sm(4);
    double best_ms = 1e30;
    for (int t : {8, 10, 12, 16})
        for (int bl = occ_f; bl >= std::max(1, occ_f - 1) && rc == MST_OK; --bl) {
            rc = mst_batch_set_wavefront(b, t, bl, best[2], best[3]);
            if (rc == MST_OK) rc = timed(ms);
            if (rc == MST_OK && ms < best_ms) {
                best_ms = ms;
                best[0] = t;
                best[1] = bl;
            }
        }
    best_ms = 1e30;
    for (int t : {4, 6, 8, 10})
        for (int bl = occ_r; bl >= std::max(1, occ_r - 1) && rc == MST_OK; --bl) {
            rc = mst_batch_set_wavefront(b, best[0], best[1], t, bl);
            if (rc == MST_OK) rc = timed(ms);
            if (rc == MST_OK && ms < best_ms) {
                best_ms = ms;
                best[2] = t;
                best[3] = bl;
            }
        }
    for (int i = 0; i < n; ++i) {  // the sample's event counts must not size the real calls' buffers
        b->grids[i]->ev_last = ev_last0[i];
        b->grids[i]->ev_counted = ev_counted0[i] != 0;
        b->grids[i]->ev_seen_pending = false;
    }
    if (b->launched) {
        cudaEventSynchronize(b->done);
        b->launched = false;
    }
    cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (double* p : grads) cudaFree(p);
    cudaFree(losses);
    if (rc) {
        b->trip_fwd = saved[0];
        b->blocks_fwd = saved[1];
        b->trip_p2 = saved[2];
        b->blocks_p2 = saved[3];
        return rc;
    }
    for (int k = 0; k < 4; ++k) choice[k] = best[k];
    return mst_batch_set_wavefront(b, best[0], best[1], best[2], best[3]);
}

int mst_batch_render_grad(mst_batch* b, const float* const* betas, const mst_params* params,
                          const double* const* meas, const uint8_t* const* masks, double* const* images,
                          double* const* grads, double* losses, void* stream) {
    if (!b) return MST_ERR_INVALID_ARG;
    if (!betas || !params || !meas || !grads || !losses) {
        b->err = "betas, params, images_meas, grads and losses are required";
        return MST_ERR_INVALID_ARG;
    }
    for (int i = 0; i < b->n; ++i) {
        const int rc = check_render_grad(b->grids[i], betas[i], &params[i], meas[i], grads[i]);
        if (rc) {
            b->err = "scene " + std::to_string(i) + ": " + b->grids[i]->err;
            return rc;
        }
    }
    DeviceGuard dg(b->device);
    cudaStream_t st = as_stream(stream);
    // The graph bakes in the call's pointers and each handle's scratch buffers; any change
    // (including a buffer a direct call on the handle reallocated) re-captures it.
    auto make_key = [&]() {
        std::vector<unsigned char> k;
        for (int i = 0; i < b->n; ++i) {
            const mst_grid* g = b->grids[i];
            key_add(k, betas[i]);
            key_add(k, params[i]);
            key_add(k, meas[i]);
            key_add(k, masks ? masks[i] : nullptr);
            key_add(k, images ? images[i] : nullptr);
            key_add(k, grads[i]);
            key_add(k, g->dbg_hash);
            key_add(k, g->dbg_skip);
            key_add(k, g->air);
            key_add(k, g->albedo_air);
            key_add(k, g->reg_wz);
            const void* bufs[] = {g->wbuf, g->nevbuf, g->plist, g->evoff, g->evrec, g->wseq, g->ch_next,
                                  g->warp_head, g->Qw, g->btot, g->btot_ref};
            for (const void* q : bufs) key_add(k, q);
            key_add(k, g->ev_cap);
            key_add(k, g->batch_stored);
        }
        key_add(k, losses);
        key_add(k, b->form);
        key_add(k, b->trip_fwd);
        key_add(k, b->blocks_fwd);
        key_add(k, b->trip_p2);
        key_add(k, b->blocks_p2);
        return k;
    };
    // A handle whose events overflowed its buffer in the last launch (W then came from replay
    // pass 1 on the device) gets a buffer for the count it saw; the new buffer re-captures.
    if (b->launched && cudaEventQuery(b->done) == cudaSuccess) {
        for (int i = 0; i < b->n; ++i) {
            mst_grid* g = b->grids[i];
            if (g->batch_stored && *g->ev_seen > g->ev_cap) {
                g->ev_last = *g->ev_seen;
                g->ev_counted = true;
                g->batch_stored = ensure_records(g, params[i].n_photons, params[i].grid_dtype);
                g->err.clear();
            }
        }
        b->launched = false;
    }
    cudaGetLastError();  // a query that found the launch still running
    std::vector<unsigned char> key = make_key();
    if (!b->exec || key != b->key) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        // everything that allocates or sets function attributes happens before the capture
        for (int i = 0; i < b->n; ++i) {
            mst_grid* g = b->grids[i];
            g->prof = false;
            prof_reset(g);
            int rc = ensure_q(g, params[i].grad_mode == MST_GRAD_SURROGATE ? params[i].conditioning : 0, st);
            if (rc == MST_OK && params[i].grad_mode == MST_GRAD_FULL) rc = ensure_replay(g, kReplayChunk);  // no allocation in capture
            if (rc) {
                b->err = g->err;
                return rc;
            }
            // full gradient: the forward stores its events in buffers sized here (W without pass 1)
            g->batch_stored = params[i].grad_mode == MST_GRAD_FULL &&
                              ensure_records(g, params[i].n_photons, params[i].grid_dtype) &&
                              ensure_replay(g, params[i].n_photons) == MST_OK;
            g->err.clear();
            for (int mode = 0; mode < 7; ++mode)
                transport_blocks_per_sm(params[i].grid_dtype, mode, g->air != nullptr);
        }
        key = make_key();  // with the buffers as the graph will use them
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            b->err = "stream error before capture";
            return MST_ERR_CUDA;
        }
        b->persistent = persistent_ok(b, params);
        if (b->persistent) {
            transport_batch_blocks_per_sm(0);  // function attributes and occupancy, outside the capture
            const int rc0 = persistent_tables(b, betas, params);
            if (rc0) return rc0;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            b->err = "cudaStreamBeginCapture failed";
            return MST_ERR_CUDA;
        }
        int rc = MST_OK;
        for (int i = 0; i < b->n; ++i) b->grids[i]->capturing = true;  // no allocation in the branches
        if (b->persistent) {
            rc = persistent_sequence(b, betas, params, meas, masks, images, grads, losses);
            if (rc) {
                for (int i = 0; i < b->n; ++i)
                    if (!b->grids[i]->err.empty()) b->err = "scene " + std::to_string(i) + ": " + b->grids[i]->err;
            }
        } else {
            cudaEventRecord(b->fork, b->cap);
            for (int i = 0; i < b->n && rc == MST_OK; ++i) {
                cudaStreamWaitEvent(b->branch[i], b->fork, 0);
                rc = render_grad_impl(b->grids[i], betas[i], &params[i], meas[i], masks ? masks[i] : nullptr,
                                      images ? images[i] : nullptr, grads[i], losses + i, b->branch[i]);
                if (rc) b->err = "scene " + std::to_string(i) + ": " + b->grids[i]->err;
                cudaEventRecord(b->join[i], b->branch[i]);
                cudaStreamWaitEvent(b->cap, b->join[i], 0);
            }
        }
        const cudaError_t ec = cudaStreamEndCapture(b->cap, &graph);
        for (int i = 0; i < b->n; ++i) b->grids[i]->capturing = false;
        if (rc == MST_OK && (ec != cudaSuccess || !graph)) {
            b->err = std::string("graph capture failed: ") + cudaGetErrorString(ec);
            rc = MST_ERR_CUDA;
        }
        if (rc == MST_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
            b->err = "cudaGraphInstantiate failed";
            b->exec = nullptr;
            rc = MST_ERR_CUDA;
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (rc) return rc;
        b->key = key;
    }
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) {
        b->err = "cudaGraphLaunch failed";
        return MST_ERR_CUDA;
    }
    if (!b->launched && cudaEventRecord(b->done, st) == cudaSuccess) b->launched = true;
    return MST_OK;
}

}  // extern "C"

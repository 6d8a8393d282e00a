// LOS transmittance for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: a host that hands out device memory only through
// its own arena, or a plugin whose process forbids allocation after start-up.
// mst_transmittance_noalloc serves them: it takes no
// handle, and the only scratch it needs (the staged extinction grid) lives in
// a file-scope device array that every GPU loading this library holds until the process ends.
// The caller passes beta and T; nothing is allocated or freed here.
#include <cmath>
#include <cstring>
#include <mutex>

#include "mst_internal.h"

namespace {

// 2^21 voxels (8 MiB of FP32): grids up to 128 x 128 x 128 voxels.
constexpr int kNoAllocMaxVoxels = 1 << 21;
static_assert(kNoAllocMaxVoxels == MST_NOALLOC_MAX_VOXELS, "header and library disagree");

static __device__ __align__(256) float g_noalloc_ext[kNoAllocMaxVoxels];

// Device address of g_noalloc_ext, resolved once per device. In host code the symbol name
// is only a host-side stand-in for the array, so the address must come from the runtime.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int ext_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return MST_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_ext) != cudaSuccess || !p) {
            cudaGetLastError();
            return MST_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MST_OK;
}

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

}  // namespace

extern "C" int mst_transmittance_noalloc(const mst_grid_desc* d, int n_cams, const mst_camera* cams,
                                         const float* beta_dev, float* T_dev, void* stream) {
    if (!d || !cams || !beta_dev || !T_dev) return MST_ERR_INVALID_ARG;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nx > 2048 || d->ny > 2048 || d->nz > 1024)
        return MST_ERR_INVALID_ARG;
    if (!(d->dx > 0 && d->dy > 0 && d->dz > 0) || !std::isfinite(d->dx + d->dy + d->dz) || !finite3(d->origin))
        return MST_ERR_INVALID_ARG;
    if (n_cams < 1 || n_cams > MST_MAX_CAMERAS) return MST_ERR_INVALID_ARG;
    if ((long long)d->nx * d->ny * d->nz > kNoAllocMaxVoxels) return MST_ERR_TOO_LARGE;
    const double hh[3] = {d->dx, d->dy, d->dz};
    const int nn[3] = {d->nx, d->ny, d->nz};
    for (int c = 0; c < n_cams; ++c) {
        const mst_camera& cm = cams[c];
        if (!finite3(cm.pos)) return MST_ERR_INVALID_ARG;
        for (int a = 0; a < 3; ++a)
            if (std::fabs(cm.pos[a] - d->origin[a]) > (nn[a] + 1e6) * hh[a]) return MST_ERR_INVALID_ARG;
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MST_ERR_NO_DEVICE;
    void* scratch = nullptr;
    const int rc = ext_address(dev, &scratch);
    if (rc != MST_OK) return rc;

    // A descriptor on the host stack for the two launchers below (launch_stage, launch_los):
    // grid geometry, cameras and the static extinction array; no statistics and no padded grid
    // are kept (stats and ext_pad stay NULL, which both launchers accept).
    mst_grid g;
    g.device = dev;
    cudaDeviceGetAttribute(&g.sm_count, cudaDevAttrMultiProcessorCount, dev);
    mst::Geo& geo = g.geo;
    geo.nx = d->nx; geo.ny = d->ny; geo.nz = d->nz;
    geo.hx = (float)d->dx; geo.hy = (float)d->dy; geo.hz = (float)d->dz;
    geo.ex = (float)(d->nx * d->dx); geo.ey = (float)(d->ny * d->dy); geo.ez = (float)(d->nz * d->dz);
    geo.nvox = d->nx * d->ny * d->nz;
    geo.max_steps = d->nx + d->ny + d->nz + 8;
    g.n_cams = n_cams;
    g.cams.n = n_cams;
    for (int c = 0; c < n_cams; ++c) {
        const mst_camera& s = cams[c];
        mst::Cam& t = g.cams.c[c];
        std::memset(&t, 0, sizeof(t));
        t.px = (float)(s.pos[0] - d->origin[0]);
        t.py = (float)(s.pos[1] - d->origin[1]);
        t.pz = (float)(s.pos[2] - d->origin[2]);
        int iv[3];
        float lv[3];
        bool inside = true;
        for (int a = 0; a < 3; ++a) {
            const double x = s.pos[a] - d->origin[a];
            const double f = std::floor(x / hh[a]);
            iv[a] = (int)f;
            double off = x - f * hh[a];
            off = off < 0.0 ? 0.0 : (off > hh[a] ? hh[a] : off);
            lv[a] = (float)off;
            if (iv[a] < 0 || iv[a] >= nn[a]) inside = false;
        }
        t.ix = iv[0]; t.iy = iv[1]; t.iz = iv[2];
        t.lx = lv[0]; t.ly = lv[1]; t.lz = lv[2];
        t.inside = inside ? 1 : 0;
    }
    g.ext = scratch;
    g.stats = nullptr;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // staging writes every voxel of this grid, so no clearing is needed
    if (mst::launch_stage(&g, beta_dev, nullptr, MST_GRID_F32, st) != cudaSuccess) return MST_ERR_CUDA;
    if (mst::launch_los(&g, MST_GRID_F32, nullptr, nullptr, nullptr, beta_dev, T_dev, nullptr, st) != cudaSuccess)
        return MST_ERR_CUDA;
    g.ext = nullptr;  // not owned
    return MST_OK;
}

"""Pins of the CPU oracle against what the paper and the mathematics fix, independent of the
oracle's own code: a library Philox, closed forms, invariants, brute-force integrals."""
import math

import numpy as np
import pytest
from scipy import integrate

import synth
from tests import raygeom as rg


# ------------------------------------------------------------------------------------------
# random numbers


def _philox_generic(ctr, key, M, W, bits, rounds=10):
    """Philox round structure written from its definition for any word size."""
    mask = (1 << bits) - 1
    c, k = [int(x) for x in ctr], [int(x) for x in key]
    for r in range(rounds):
        if r:
            k = [(k[0] + W[0]) & mask, (k[1] + W[1]) & mask]
        p0, p1 = M[0] * c[0], M[1] * c[2]
        c = [(p1 >> bits) ^ c[1] ^ k[0], p1 & mask, (p0 >> bits) ^ c[3] ^ k[1], p0 & mask]
    return c


M64 = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
W64 = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)
M32 = (0xD2511F53, 0xCD9E8D57)
W32 = (0x9E3779B9, 0xBB67AE85)


def test_philox_structure_matches_numpy_4x64():
    """The generic round structure reproduces numpy's Philox-4x64-10 bit generator, which
    emits the block of counter+1 first."""
    for key, ctr in [((0, 0), (0, 0, 0, 0)), ((123456789, 987654321), (5, 7, 11, 13)),
                     ((2 ** 64 - 1, 2 ** 63 + 5), (2 ** 64 - 2, 3, 2 ** 40, 9))]:
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
        got = [int(x) for x in bg.random_raw(4)]
        c1 = list(ctr)
        c1[0] = (c1[0] + 1) & (2 ** 64 - 1)
        if c1[0] == 0:
            c1[1] += 1
        assert got == _philox_generic(c1, key, M64, W64, 64)


def test_oracle_philox4x32_matches_generic(orc):
    rng = np.random.default_rng(0)
    for _ in range(200):
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64)
        assert [int(x) for x in orc.philox4x32_10(ctr, key)] == _philox_generic(ctr, key, M32, W32, 32)


def test_uniform_map_exact_and_open_interval(orc):
    assert orc.u01(0) == 2.0 ** -24
    assert orc.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert orc.u01(0x80000000) == 0.5 + 2.0 ** -24
    # exactly representable in float32 and symmetric: u(x) + u(~x) = 1
    for x in [1, 12345, 0xDEADBEEF, 0x7FFFFFFF]:
        u = orc.u01(x)
        assert float(np.float32(u)) == u
        assert u + orc.u01(0xFFFFFFFF ^ x) == 1.0


def test_philox_uniform_chi2(orc):
    vals = []
    for p in range(4000):
        vals.extend(orc.philox4x32_10([p, 0, 3, 0], [3, 0]).tolist())
    u = (np.array(vals, dtype=np.uint64) >> 9).astype(np.float64) / 2 ** 23
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    e = len(u) / 64
    chi2 = float(((hist - e) ** 2 / e).sum())
    assert chi2 < 120  # 63 dof, p ~ 1e-5
    # neighbouring counters decorrelated
    a, b = u[0::4], u[1::4]
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.05


# ------------------------------------------------------------------------------------------
# Henyey-Greenstein (Eq. Phg, Eq. thetaHG)


@pytest.mark.parametrize("g", [-0.7, 0.0, 0.3, 0.85, 0.95])
def test_hg_phase_normalised(orc, g):
    val, _ = integrate.quad(lambda mu: 2 * math.pi * orc.hg_phase(g, mu), -1, 1, limit=200)
    assert abs(val - 1.0) < 1e-8


@pytest.mark.parametrize("g", [-0.5, 1e-9, 0.3, 0.85])
def test_hg_sampling_matches_phase(orc, g):
    """Stratified u through the inverse CDF reproduces the bin masses of Eq. Phg and E[cos] = g."""
    n = 200_000
    u = (np.arange(n) + 0.5) / n
    mu = np.array([orc.hg_sample(g, x) for x in u])
    assert abs(mu.mean() - g) < 2e-4
    edges = np.linspace(-1, 1, 41)
    hist, _ = np.histogram(mu, bins=edges)
    for a, b, h in zip(edges[:-1], edges[1:], hist):
        mass, _ = integrate.quad(lambda m: 2 * math.pi * orc.hg_phase(g, m), a, b)
        assert abs(h / n - mass) < 2.0 / n + 1e-6
    assert np.all(np.diff(mu) >= 0)


def test_rotation_geometry(orc):
    rng = np.random.default_rng(5)
    for _ in range(300):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        if _ % 10 == 0:
            d = np.array([0.0, 0.0, -1.0]) if _ % 20 == 0 else np.array([0.3, 0.0, math.sqrt(1 - 0.09)])
        ct = rng.uniform(-1, 1)
        phis = np.linspace(0, 2 * math.pi, 64, endpoint=False)
        outs = np.array([orc.rotate(d, ct, ph) for ph in phis])
        assert np.allclose(np.linalg.norm(outs, axis=1), 1.0, atol=1e-12)
        assert np.allclose(outs @ d, ct, atol=1e-12)
        assert np.allclose(outs.mean(axis=0), ct * d, atol=1e-12)


# ------------------------------------------------------------------------------------------
# helpers


def slab_scene(beta, nx=50, nz=20, dx=20.0, dz=10.0, cam_z=1.0, fov=20.0, npx=4, n_rays=10):
    shape, h = (nx, nx, nz), (dx, dx, dz)
    L = nx * dx
    cams = synth.make_cameras([(L / 2 + 0.25 * dx, L / 2 + 0.25 * dx, cam_z)], npx, npx, fov)
    return synth.make_scene(shape, h, synth.homogeneous(shape, beta), cams, n_rays=n_rays)


def batched(orc, scene, params, nb, fn):
    """Runs fn over nb photon sub-ranges (normalised to the full count); returns stacked results."""
    n = params.n_photons
    out = []
    for b in range(nb):
        p = params.replace(n_photons=n // nb, photon_offset=b * (n // nb), n_photons_total=n)
        out.append(fn(p))
    return np.array(out)


# ------------------------------------------------------------------------------------------
# (i) Beer-Lambert


def test_beer_lambert_zero_albedo(orc):
    beta = 2e-3
    sc = slab_scene(beta, nx=8, nz=10, dx=50.0, dz=20.0)
    p = synth.Params(albedo=0.0, g=0.5, sun_zenith=0.0, n_photons=200_000, seed=9)
    r = orc.render(sc, p)
    assert np.all(r["L"] == 0.0)
    H = 10 * 20.0
    frac = r["stats"]["esc_zm"] / r["stats"]["launched"]
    expect = math.exp(-beta * H)
    sig = math.sqrt(expect * (1 - expect) / p.n_photons)
    assert abs(frac - expect) < 3.5 * sig


def test_homogeneous_transmittance_closed_form(orc):
    beta = 1.7e-3
    sc = slab_scene(beta, nx=6, nz=5, dx=30.0, dz=40.0, cam_z=57.0)
    sc.cam_pos[0] = [61.3, 95.2, 57.0]
    tau, T = orc.transmittance(sc)
    nx, ny, nz = sc.shape
    k = np.arange(sc.nvox)
    c = np.stack([(k % nx + 0.5) * 30.0, ((k // nx) % ny + 0.5) * 30.0, (k // (nx * ny) + 0.5) * 40.0], 1)
    dist = np.linalg.norm(c - sc.cam_pos[0], axis=1)
    assert np.allclose(tau[0], beta * dist, rtol=1e-12, atol=1e-15)
    assert np.allclose(T[0], np.exp(-beta * dist), rtol=1e-12)


def test_inhomogeneous_los_depth_brute_force(orc):
    sc, _ = synth.cfg_blobs16()
    tau, _ = orc.transmittance(sc)
    rng = np.random.default_rng(2)
    nx, ny, nz = sc.shape
    for c in (0, 3):
        for k in rng.integers(0, sc.nvox, 12):
            ctr = np.array([(k % nx + 0.5), ((k // nx) % ny + 0.5), (k // (nx * ny) + 0.5)]) * 50.0
            v = sc.cam_pos[c] - ctr
            dist = np.linalg.norm(v)
            ref = rg.line_integral(sc, sc.beta, ctr, v / dist, 0.0, dist)
            assert abs(tau[c, k] - ref) < 1e-4 * max(ref, 1e-3)


# ------------------------------------------------------------------------------------------
# (iii) energy


@pytest.mark.parametrize("albedo,rr", [(1.0, 0.0), (0.9, 0.0), (0.97, 0.05)])
def test_energy_balance(orc, albedo, rr):
    sc, _ = synth.cfg_blobs16()
    p = synth.Params(albedo=albedo, g=0.85, sun_zenith=math.radians(30), n_photons=20_000, seed=5,
                     rr_threshold=rr, rr_survival=0.25)
    s = orc.render(sc, p)["stats"]
    esc = sum(s[k] for k in ["esc_xm", "esc_xp", "esc_ym", "esc_yp", "esc_zm", "esc_zp"])
    out = esc + s["absorbed"] + s["rr_killed"] + s["forced"] - s["rr_gained"]
    incident = math.cos(p.sun_zenith) * 800.0 * 800.0
    assert abs(s["launched"] - incident) < 1e-9 * incident
    assert abs(out - incident) < 1e-10 * incident
    if albedo == 1.0:
        assert abs(esc - incident) < 1e-10 * incident


# ------------------------------------------------------------------------------------------
# (vi) deterministic parts: chords, Pi, W, adjoints


def test_pixel_chords_sum(orc):
    """With L T = V in every voxel, Eq. Icpixel returns the mean chord of the sub-pixel rays."""
    sc, _ = synth.cfg_blobs16()
    sc.cam_pos[1] = [-100.0, 300.0, 420.0]          # outside the box, looking in
    sc.cam_rot[1] = synth.look_at_rot([1.0, 0.2, 0.1])
    V = float(np.prod(sc.h))
    one = np.ones((sc.n_cams, sc.nvox))
    img = orc.images(sc, one * V, one)
    lo, hi = rg.box(sc)
    off = 0
    rng = np.random.default_rng(1)
    for c in range(sc.n_cams):
        W, H = sc.cam_w[c], sc.cam_h[c]
        for p in rng.integers(0, W * H, 25):
            i, j = p % W, p // W
            ref = np.mean([rg.chord(sc.cam_pos[c], d, lo, hi) for d in rg.subpixel_dirs(sc, c, i, j)])
            assert abs(img[off + p] - ref) < 1e-9 * max(ref, 1.0)
        off += W * H


def test_pixel_chords_sum_wide_field(orc):
    """The same identity for wide pinholes on a flat, wide box (the haze reconstruction's
    cameras: 150 deg, rays up to 79 deg from the axis, chords of up to ~10 km through voxels of
    625 x 625 x 83 m), including a camera looking sideways from inside the box."""
    shape, h = (20, 20, 30), (625.0, 625.0, 10000.0 / 120)
    pos = [(3100.0, 4700.0, 1.0), (9350.0, 6300.0, 1.0), (6300.0, 6300.0, 1200.0)]
    rots = [synth.look_up_rot(), synth.look_up_rot(), synth.look_at_rot([0.3, 1.0, 0.05])]
    sc = synth.make_scene(shape, h, np.zeros(int(np.prod(shape))), synth.make_cameras(pos, 8, 6, 150.0, rots=rots))
    V = float(np.prod(sc.h))
    one = np.ones((sc.n_cams, sc.nvox))
    img = orc.images(sc, one * V, one)
    lo, hi = rg.box(sc)
    off = 0
    for c in range(sc.n_cams):
        W, H = sc.cam_w[c], sc.cam_h[c]
        for p in range(W * H):
            i, j = p % W, p // W
            ref = np.mean([rg.chord(sc.cam_pos[c], d, lo, hi) for d in rg.subpixel_dirs(sc, c, i, j)])
            assert abs(img[off + p] - ref) < 1e-9 * max(ref, 1.0), (c, p, img[off + p], ref)
        off += W * H
    assert img.max() > 8000.0  # oblique rays cross the 2.5 km high box over ~10 km


def test_pixel_integral_brute_force(orc):
    """Per-voxel chord attribution: image of an arbitrary field equals the dense line integral."""
    sc, _ = synth.cfg_blobs16()
    V = float(np.prod(sc.h))
    f = np.random.default_rng(4).random(sc.nvox)
    img = orc.images(sc, np.tile(f * V, (sc.n_cams, 1)), np.ones((sc.n_cams, sc.nvox)))
    lo, hi = rg.box(sc)
    for c, p in [(0, 17 * 32 + 5), (2, 31 * 32 + 31), (4, 3)]:
        i, j = p % 32, p // 32
        acc = 0.0
        for d in rg.subpixel_dirs(sc, c, i, j):
            r = rg.ray_box(sc.cam_pos[c], d, lo, hi)
            if r:
                acc += rg.line_integral(sc, f, sc.cam_pos[c], d, max(r[0], 0.0), r[1], n=100_000)
        ref = acc / sc.n_rays
        assert abs(img[sum(sc.cam_w[:c] * sc.cam_h[:c]) + p] - ref) < 2e-4 * ref


def test_adjoint_identities(orc):
    """<Pi R, r> = <R, Pi^T r> and <W beta, s> = <beta, W^T s> (Eq. IcP, Eq. bTck)."""
    sc, _ = synth.cfg_blobs16()
    rng = np.random.default_rng(3)
    R = rng.random((sc.n_cams, sc.nvox))
    r = rng.standard_normal(sc.n_pix)
    lhs = float(orc.images(sc, R, np.ones_like(R)) @ r)
    rhs = float((R * orc.backproject(sc, r)).sum())
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    s = rng.standard_normal((sc.n_cams, sc.nvox))
    tau, _ = orc.transmittance(sc)
    lhs = float((tau * s).sum())
    rhs = float((orc.los_adjoint(sc, s) * sc.beta[None, :]).sum())
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_ray_counts_brute_force(orc):
    sc, _ = synth.cfg_blobs16()
    sc = synth.make_scene((4, 4, 4), (50.0, 50.0, 50.0), synth.homogeneous((4, 4, 4), 1e-3),
                          synth.make_cameras([(101.0, 87.0, -20.0)], 6, 6, 50.0), n_rays=4)
    Q = orc.ray_counts(sc)
    ref = np.zeros(sc.nvox)
    for k in range(sc.nvox):
        v = np.array([k % 4, (k // 4) % 4, k // 16])
        lo, hi = v * 50.0, (v + 1) * 50.0
        for p in range(36):
            for d in rg.subpixel_dirs(sc, 0, p % 6, p // 6):
                if rg.chord(sc.cam_pos[0], d, lo, hi) >= 1e-4 * 50.0:
                    ref[k] += 1
    assert np.array_equal(Q[0], ref)


# ------------------------------------------------------------------------------------------
# (ii) single scattering in a homogeneous slab


def _slab_radiance(F, albedo, g, beta, H, mu0, sun, d):
    mu = d[2]
    tau = beta * H
    cos_scat = float(np.dot(sun, -d))
    P = (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * cos_scat) ** 1.5)
    if abs(mu - mu0) < 1e-9:
        return albedo * F * P * tau / mu0 * math.exp(-tau / mu0)
    return albedo * F * P * mu0 / (mu - mu0) * (math.exp(-tau / mu) - math.exp(-tau / mu0))


def test_slab_single_scatter_voxelised(orc):
    """Voxelised FMC (Eq. Lcupdate + Eq. Icpixel), first order, isotropic: the closed form of the
    slab, averaged over the same sub-pixel rays; tolerance 3.5 MC sigma + 0.5% voxelisation bias."""
    beta, albedo, g = 2.5e-3, 0.9, 0.0
    sc = slab_scene(beta)
    p = synth.Params(albedo=albedo, g=g, sun_zenith=math.radians(30), n_photons=1_600_000, seed=21, max_order=1,
                     rr_threshold=0.0)
    _, T = orc.transmittance(sc)
    imgs = batched(orc, sc, p, 8, lambda q: orc.images(sc, orc.render(sc, q)["L"], T))
    est, sig = imgs.sum(0), imgs.std(0, ddof=1) * math.sqrt(8)
    sun = np.array([-math.sin(p.sun_zenith), 0.0, -math.cos(p.sun_zenith)])
    for pix in range(16):
        i, j = pix % 4, pix // 4
        ref = np.mean([_slab_radiance(1.0, albedo, g, beta, 200.0, math.cos(p.sun_zenith), sun, d)
                       for d in rg.subpixel_dirs(sc, 0, i, j)])
        assert abs(est[pix] - ref) < 3.5 * sig[pix] + 5e-3 * ref, (pix, est[pix], ref, sig[pix])


def test_slab_single_scatter_classic(orc):
    """Classic local estimate (Eq. fle), first order, anisotropic: unbiased against the closed
    form averaged over each pixel's solid angle."""
    beta, albedo, g = 2.5e-3, 0.9, 0.5
    sc = slab_scene(beta, cam_z=-50.0)   # away from the medium: bounded 1/r^2, finite variance
    p = synth.Params(albedo=albedo, g=g, sun_zenith=math.radians(30), n_photons=1_600_000, seed=22, max_order=1,
                     rr_threshold=0.0)
    imgs = batched(orc, sc, p, 8, lambda q: orc.render(sc, q, want_L=False, classic=True)["classic"])
    est, sig = imgs.sum(0), imgs.std(0, ddof=1) * math.sqrt(8)
    sun = np.array([-math.sin(p.sun_zenith), 0.0, -math.cos(p.sun_zenith)])
    n = 12
    for pix in range(16):
        i, j = pix % 4, pix // 4
        acc = wsum = 0.0
        for a in range(n):
            for b in range(n):
                px, py = i + (a + 0.5) / n, j + (b + 0.5) / n
                d = rg.pixel_dir(sc, 0, px, py)
                tx = math.tan(0.5 * sc.cam_fov[0])
                x, y = (2 * px / 4 - 1) * tx, (2 * py / 4 - 1) * tx
                w = (1 + x * x + y * y) ** -1.5
                acc += w * _slab_radiance(1.0, albedo, g, beta, 200.0, math.cos(p.sun_zenith), sun, d)
                wsum += w
        ref = acc / wsum
        assert abs(est[pix] - ref) < 3.5 * sig[pix] + 2e-3 * ref, (pix, est[pix], ref, sig[pix])


# ------------------------------------------------------------------------------------------
# (iv) Helmholtz reciprocity: forward classic LE vs backward MC with the sun LE (Eq. ble)


def test_reciprocity_fmc_bmc(orc):
    shape, h = (8, 8, 8), (50.0, 50.0, 50.0)
    beta = synth.blob_field(shape, h, 2, (60.0, 120.0), 5e-3, 2e-4, seed=7)
    sc = synth.make_scene(shape, h, beta, synth.make_cameras([(212.0, 188.0, -5.0)], 8, 8, 60.0))
    p = synth.Params(albedo=0.99, g=0.7, sun_zenith=math.radians(30), n_photons=1_600_000, seed=31,
                     rr_threshold=0.0, max_order=0)
    imgs = batched(orc, sc, p, 8, lambda q: orc.render(sc, q, want_L=False, classic=True)["classic"])
    est, sig = imgs.sum(0), imgs.std(0, ddof=1) * math.sqrt(8)
    for (i, j) in [(3, 4), (4, 3), (2, 2), (5, 6)]:
        m, s = orc.bmc_pixel(sc, p.replace(seed=77), 0, i, j, 40_000)
        pix = j * 8 + i
        assert abs(est[pix] - m) < 3.5 * math.hypot(sig[pix], s), (i, j, est[pix], m, sig[pix], s)


# ------------------------------------------------------------------------------------------
# (v) brute-force quadrature on a 2^3 grid, orders 1 and 2


def _q2_setup():
    shape, h = (2, 2, 2), (100.0, 100.0, 100.0)
    beta = np.array([2e-4, 5e-4, 3e-4, 4e-4, 5e-4, 2.5e-4, 3.5e-4, 4.5e-4]) * 4.0
    cams = synth.make_cameras([(120.0, 83.0, -30.0), (55.0, 140.0, -10.0)], 4, 4, 90.0)
    return synth.make_scene(shape, h, beta, cams)


def _tau_along(beta, o, d, tmax, lo_all, hi_all):
    """Optical depth from o along d to parameter tmax, by per-voxel slab clipping."""
    tau = np.zeros(o.shape[0])
    for k in range(8):
        t0, t1 = _clip(o, d, lo_all[k], hi_all[k])
        a, b = np.maximum(t0, 0.0), np.minimum(t1, tmax)
        tau += beta[k] * np.maximum(b - a, 0.0)
    return tau


def _clip(o, d, lo, hi):
    """Parameter interval of rays o + t d inside the box [lo, hi] (slab method, vectorised)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = (lo[None, :] - o) / d
        tb = (hi[None, :] - o) / d
    inside = (o >= lo) & (o <= hi)
    lower = np.where(d == 0, np.where(inside, -np.inf, np.inf), np.minimum(ta, tb))
    upper = np.where(d == 0, np.where(inside, np.inf, -np.inf), np.maximum(ta, tb))
    return np.max(lower, axis=1), np.min(upper, axis=1)


def _hg(g, mu):
    return (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * mu) ** 1.5)


def _quadrature_L(sc, albedo, g, nq=6, nmu=16, nphi=16, nl=5):
    """E[L_c(k)] for orders 1 and 2 with the sun at zenith, by Gauss quadrature."""
    beta = sc.beta
    lo_all = np.array([[(k % 2) * 100.0, ((k // 2) % 2) * 100.0, (k // 4) * 100.0] for k in range(8)])
    hi_all = lo_all + 100.0
    xg, wg = np.polynomial.legendre.leggauss(nq)
    x01, w01 = (xg + 1) / 2, wg / 2
    sun = np.array([0.0, 0.0, -1.0])
    C = sc.n_cams
    Q1 = np.zeros((C, 8))
    Q2 = np.zeros((C, 8))
    # first-collision points X1 in every voxel (density beta e^{-tau_sun}, flux F = 1)
    pts, wts, vox = [], [], []
    for k in range(8):
        P = np.stack(np.meshgrid(x01, x01, x01, indexing="ij"), -1).reshape(-1, 3) * 100.0 + lo_all[k]
        W = np.einsum("i,j,l->ijl", w01, w01, w01).ravel() * 1e6
        pts.append(P); wts.append(W); vox.append(np.full(len(W), k))
    X1, W1, K1 = np.concatenate(pts), np.concatenate(wts), np.concatenate(vox)
    tau_sun = _tau_along(beta, X1, np.tile(-sun, (len(X1), 1)), np.full(len(X1), np.inf), lo_all, hi_all)
    src = beta[K1] * np.exp(-tau_sun) * W1          # first-collision density x volume weight
    for c in range(C):
        v = sc.cam_pos[c][None, :] - X1
        v /= np.linalg.norm(v, axis=1)[:, None]
        contrib = albedo * src * _hg(g, v @ sun)
        Q1[c] = np.bincount(K1, weights=contrib, minlength=8)
    # second order: direction omega from X1, then a collision at distance l (all pairs at once)
    mg, mw = np.polynomial.legendre.leggauss(nmu)
    phis = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    MU, PH = np.meshgrid(mg, phis, indexing="ij")
    ST = np.sqrt(1 - MU ** 2)
    OM = np.stack([ST * np.cos(PH), ST * np.sin(PH), MU], -1).reshape(-1, 3)
    WD = (np.repeat(mw, nphi) * (2 * math.pi / nphi)) * _hg(g, OM @ sun)
    n1, nd = len(X1), len(OM)
    O = np.repeat(X1, nd, axis=0)
    D = np.tile(OM, (n1, 1))
    base0 = albedo * albedo * np.repeat(src, nd) * np.tile(WD, n1)
    lg, lw = np.polynomial.legendre.leggauss(nl)
    for k2 in range(8):
        t0, t1 = _clip(O, D, lo_all[k2], hi_all[k2])
        a, b = np.maximum(t0, 0.0), t1
        ok = b > a
        a, b, o2, d2, b0 = a[ok], b[ok], O[ok], D[ok], base0[ok]
        for q in range(nl):
            t = a + (lg[q] + 1) / 2 * (b - a)
            X2 = o2 + t[:, None] * d2
            tau12 = _tau_along(beta, o2, d2, t, lo_all, hi_all)
            w = b0 * beta[k2] * np.exp(-tau12) * lw[q] / 2 * (b - a)
            for c in range(C):
                v = sc.cam_pos[c][None, :] - X2
                v /= np.linalg.norm(v, axis=1)[:, None]
                Q2[c, k2] += float(np.sum(w * _hg(g, np.einsum("ij,ij->i", v, d2))))
    return Q1, Q2


@pytest.mark.slow
def test_quadrature_orders_1_and_2(orc):
    sc = _q2_setup()
    albedo, g = 0.95, 0.5
    Q1, Q2 = _quadrature_L(sc, albedo, g)
    n = 4_000_000
    for order, ref in [(1, Q1), (2, Q1 + Q2)]:
        p = synth.Params(albedo=albedo, g=g, sun_zenith=0.0, n_photons=n, seed=6 + order, max_order=order,
                         rr_threshold=0.0)
        Ls = batched(orc, sc, p, 16, lambda q: orc.render(sc, q)["L"])
        est, sig = Ls.sum(0), Ls.std(0, ddof=1) * math.sqrt(16)
        assert np.all(np.abs(est - ref) < 4.0 * sig + 2e-3 * ref), (order, (est - ref) / sig)
    # the second order is resolved: dropping it would fail by more than 5 sigma in every bin
    assert np.all(Q2 > 5 * sig), Q2 / sig


# ------------------------------------------------------------------------------------------
# surrogate gradient (Eq. Jaco1-DivTc) against central differences of the j-fixed surrogate


@pytest.mark.parametrize("cond", ["none", "inv_count"])
def test_surrogate_gradient_fd(orc, cond):
    sc, p = synth.cfg_blobs16(20_000)
    sc = synth.make_scene((8, 8, 8), (100.0, 100.0, 100.0), synth.blob_field((8, 8, 8), (100.0,) * 3, 2, (150.0, 250.0),
                          8e-3, 1e-4, seed=3), synth.make_cameras([(412.0, 388.0, 1.0), (150.0, 620.0, 250.0)], 8, 8, 70.0))
    p = p.replace(n_photons=20_000)
    Lref = orc.render(sc, p)["L"]
    beta_ref = sc.beta.copy()
    meas = orc.surrogate_grad(sc.with_beta(0.8 * beta_ref), Lref, beta_ref, np.zeros(sc.n_pix))["images"]
    beta = synth.smoothed(beta_ref, sc.shape, 0.4)
    sc1 = sc.with_beta(beta)
    mask = (np.arange(sc.n_pix) % 7 != 0).astype(np.uint8)
    out = orc.surrogate_grad(sc1, Lref, beta_ref, meas, mask, "none", eta=0.0)
    g = out["grad"]
    rng = np.random.default_rng(8)
    for k in rng.choice(np.nonzero(beta > 1e-4)[0], 12, replace=False):
        hstep = 1e-3 * beta[k]
        bp, bm = beta.copy(), beta.copy()
        bp[k] += hstep
        bm[k] -= hstep
        Ep = orc.surrogate_grad(sc.with_beta(bp), Lref, beta_ref, meas, mask)["loss"]
        Em = orc.surrogate_grad(sc.with_beta(bm), Lref, beta_ref, meas, mask)["loss"]
        fd = (Ep - Em) / (2 * hstep)
        assert abs(g[k] - fd) < 1e-6 * np.abs(g).max() + 1e-7 * abs(fd), (k, g[k], fd)
    if cond == "inv_count":
        # conditioning rescales each camera's share by 1/max(1, ray count)
        gq = orc.surrogate_grad(sc1, Lref, beta_ref, meas, mask, "inv_count")["grad"]
        gc = [orc.surrogate_grad(synth.make_scene(sc.shape, sc.h, beta, dict(
            cam_pos=sc.cam_pos[c:c + 1], cam_rot=sc.cam_rot[c:c + 1], cam_w=sc.cam_w[c:c + 1],
            cam_h=sc.cam_h[c:c + 1], cam_fov=sc.cam_fov[c:c + 1])), Lref[c:c + 1], beta_ref,
            meas[c * 64:(c + 1) * 64], mask[c * 64:(c + 1) * 64])["grad"] for c in range(2)]
        Q = orc.ray_counts(sc)
        ref = sum(gc[c] / np.maximum(Q[c], 1.0) for c in range(2))
        assert np.allclose(gq, ref, rtol=1e-10, atol=1e-14 * np.abs(ref).max())


def test_laplacian_regulariser(orc):
    sc = synth.make_scene((5, 4, 3), (10.0, 10.0, 10.0), synth.homogeneous((5, 4, 3), 0.0),
                          synth.make_cameras([(1.0, 1.0, -1.0)], 2, 2, 40.0))
    # a delta at an interior voxel of degree 6 (Lap delta = -6 at k, +1 at its neighbours)
    b = np.zeros(sc.nvox)
    k = 2 + 5 * (1 + 4 * 1)
    b[k] = 1.0
    psi, _ = orc.laplacian(sc, b)
    assert psi == 36 + 6
    # a linear ramp has zero interior Laplacian; Psi comes only from boundary voxels
    x = np.tile(np.arange(5.0), 12)
    psi, _ = orc.laplacian(sc, x)
    assert psi == 2 * 12  # ends of each x-row: +1 and -1
    # gradient is exact for a quadratic
    rng = np.random.default_rng(0)
    b = rng.random(sc.nvox)
    psi, g = orc.laplacian(sc, b)
    for k in range(0, sc.nvox, 7):
        e = np.zeros(sc.nvox)
        e[k] = 1e-3
        fd = (orc.laplacian(sc, b + e)[0] - orc.laplacian(sc, b - e)[0]) / 2e-3
        assert abs(fd - g[k]) < 1e-9 * max(1.0, abs(g[k]))


def test_altitude_weighted_laplacian(orc):
    """Psi = |W Lap beta|^2 with W diagonal by altitude (Sec. 6): the delta pin with a weight on
    the delta's layer and on its neighbours' layers, zero weights removing layers, and the
    gradient 2 Lap^T W^T W Lap beta against central differences."""
    import dataclasses
    base = synth.make_scene((5, 4, 3), (10.0, 10.0, 10.0), synth.homogeneous((5, 4, 3), 0.0),
                            synth.make_cameras([(1.0, 1.0, -1.0)], 2, 2, 40.0))
    b = np.zeros(base.nvox)
    b[2 + 5 * (1 + 4 * 1)] = 1.0  # interior voxel of layer 1: Lap = -6 there, +1 at its 6 neighbours
    wz = np.array([0.5, 3.0, 2.0])
    sc = dataclasses.replace(base, reg_wz=wz)
    psi, _ = orc.laplacian(sc, b)
    # layer 1 holds the voxel (-6) and its 4 in-layer neighbours; layers 0 and 2 one neighbour each
    assert abs(psi - (3.0 ** 2 * (36 + 4) + 0.5 ** 2 + 2.0 ** 2)) < 1e-12
    psi0, _ = orc.laplacian(dataclasses.replace(base, reg_wz=np.array([0.0, 1.0, 0.0])), b)
    assert psi0 == 36 + 4
    rng = np.random.default_rng(1)
    b = rng.random(base.nvox)
    psi1, g1 = orc.laplacian(dataclasses.replace(base, reg_wz=np.full(3, 2.0)), b)
    psi_u, g_u = orc.laplacian(base, b)
    assert abs(psi1 - 4.0 * psi_u) < 1e-9 * psi1 and np.allclose(g1, 4.0 * g_u, rtol=1e-12)
    psi, g = orc.laplacian(sc, b)
    for k in range(0, sc.nvox, 5):
        e = np.zeros(sc.nvox)
        e[k] = 1e-3
        fd = (orc.laplacian(sc, b + e)[0] - orc.laplacian(sc, b - e)[0]) / 2e-3
        assert abs(fd - g[k]) < 1e-9 * max(1.0, abs(g[k]))


# ------------------------------------------------------------------------------------------
# full gradient by the score of the free-flight density, against central differences with
# common random numbers (FD-CRN)


@pytest.mark.slow
def test_full_gradient_matches_fd_crn(orc):
    shape, h = (6, 6, 6), (50.0, 50.0, 50.0)
    beta_true = synth.blob_field(shape, h, 2, (60.0, 110.0), 1e-2, 3e-4, seed=12)
    cams = synth.make_cameras([(160.0, 140.0, -10.0), (137.0, 162.0, 120.0)], 8, 8, 70.0)
    sc = synth.make_scene(shape, h, beta_true, cams)
    base = synth.Params(albedo=0.95, g=0.6, sun_zenith=math.radians(20), n_photons=200_000, rr_threshold=0.0)
    meas = orc.forward_images(sc, base.replace(seed=4))[0]
    beta = synth.smoothed(beta_true, shape, 0.5)
    sce = sc.with_beta(beta)
    voxels = np.argsort(-beta)[[0, 3, 10, 25, 40]]
    nseed = 8
    diffs = np.zeros((nseed, len(voxels)))
    gs = np.zeros((nseed, len(voxels)))
    for s in range(nseed):
        p = base.replace(seed=100 + s)
        g = orc.full_grad(sce, p, meas)["grad"]
        for i, k in enumerate(voxels):
            hstep = 0.02 * beta[k]
            bp, bm = beta.copy(), beta.copy()
            bp[k] += hstep
            bm[k] -= hstep
            Ep = orc.full_grad(sc.with_beta(bp), p, meas)["loss"]
            Em = orc.full_grad(sc.with_beta(bm), p, meas)["loss"]
            diffs[s, i] = g[k] - (Ep - Em) / (2 * hstep)
            gs[s, i] = g[k]
    t = diffs.mean(0) / (diffs.std(0, ddof=1) / math.sqrt(nseed))
    assert np.all(np.abs(t) < 5.0), t
    # and the gradient is resolved: its mean is many standard errors from zero
    tg = gs.mean(0) / (gs.std(0, ddof=1) / math.sqrt(nseed))
    assert np.median(np.abs(tg)) > 5.0, tg


def _voxel_chords(sc, d, o):
    """Chord of the ray o + t d (t >= 0) in every voxel of the scene, by the slab method on each
    voxel box (dense [nvox] array; no voxel walk)."""
    nx, ny, nz = sc.shape
    h = np.array(sc.h)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lo = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1) * h
    hi = lo + h
    t0 = np.zeros(lo.shape[0])
    t1 = np.full(lo.shape[0], np.inf)
    for a in range(3):
        if d[a] == 0.0:
            out = (o[a] < lo[:, a]) | (o[a] > hi[:, a])
            t1 = np.where(out, -np.inf, t1)
            continue
        ta, tb = (lo[:, a] - o[a]) / d[a], (hi[:, a] - o[a]) / d[a]
        t0, t1 = np.maximum(t0, np.minimum(ta, tb)), np.minimum(t1, np.maximum(ta, tb))
    return np.maximum(t1 - t0, 0.0)


def _voxelised_slab_images(sc, beta, albedo, mu0, chords):
    """Expectation of the voxelised first-order images (Eq. Lcupdate, Eq. Icpixel) of a homogeneous
    slab with isotropic scattering, far from its lateral edges. Photons enter the top along the
    sun (cosine mu0) with weight F mu0 A / N, so first collisions have density
    (N / A) (beta / mu0) exp(-beta z' / mu0) per unit volume at depth z' below the top, and each adds
    albedo I0 / (4 pi): E[L_c(k)] = albedo F beta / (4 pi) dx dy (mu0 / beta)
    (exp(-beta (H - z1) / mu0) - exp(-beta (H - z0) / mu0)) over the voxel's layer [z0, z1], F = 1.
    Then i_p = 1 / (N_rays V) sum_rho sum_k l^rho(k) T_c(k) E[L_c(k)] with T_c(k) from the voxel
    centre to the camera (Eq. Tck)."""
    nx, ny, nz = sc.shape
    hx, hy, hz = sc.h
    H, V = nz * hz, hx * hy * hz
    z0 = np.repeat(np.arange(nz) * hz, nx * ny)
    EL = albedo * beta / (4 * math.pi) * hx * hy * (mu0 / beta) * (
        np.exp(-beta * (H - z0 - hz) / mu0) - np.exp(-beta * (H - z0) / mu0))
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cen = (np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1) + 0.5) * np.array(sc.h)
    T = np.exp(-beta * np.linalg.norm(cen - sc.cam_pos[0], axis=1))
    return np.array([sum(float(np.dot(l, T * EL)) for l in ls) for ls in chords]) / (sc.n_rays * V)


@pytest.mark.slow
def test_voxelised_gradient_along_beta_matches_the_slab_expectation(orc):
    """The full gradient of the voxelised estimator (score of the free-flight density through L,
    Sec. 5.1 Eq. divCost1 with Eq. beer-lambert, plus the W^T term through T), first order, in the
    homogeneous slab with the camera on the floor: with a measured value M far above the images the
    loss is linear in them, so beta . dE/dbeta / (-2M) estimates sum_p tau d i_p / d tau, the
    derivative along beta of the voxelised model's expected images, which the closed form of the
    first-collision density gives exactly (no voxelisation bias: the reference is the voxelised
    model itself). The images are pinned against the same expectation. Planted in the oracle, a
    20 % scale error in the suffix sums S_j moves the estimate by ~20 sigma, one in the chord term
    of the score by ~7 sigma and one in the collision term 1 / beta by ~60 sigma."""
    beta, albedo = 2.5e-3, 0.9
    sc = slab_scene(beta)
    p = synth.Params(albedo=albedo, g=0.0, sun_zenith=math.radians(30), n_photons=16_000_000, seed=25, max_order=1,
                     rr_threshold=0.0)
    M = 1e6
    meas = np.full(sc.n_pix, M)

    def one(q):
        r = orc.full_grad(sc, q, meas)
        return [float(np.dot(sc.beta, r["grad"])) / (-2.0 * M), float(r["images"].sum())]

    nb = 32
    out = batched(orc, sc, p, nb, one)
    est, sig = out[:, 0].sum(), out[:, 0].std(ddof=1) * math.sqrt(nb)
    img, isig = out[:, 1].sum(), out[:, 1].std(ddof=1) * math.sqrt(nb)
    mu0 = math.cos(p.sun_zenith)
    chords = [[_voxel_chords(sc, d, sc.cam_pos[0]) for d in rg.subpixel_dirs(sc, 0, pix % 4, pix // 4)]
              for pix in range(16)]
    ref_img = _voxelised_slab_images(sc, beta, albedo, mu0, chords).sum()
    e = 1e-4
    ref = (_voxelised_slab_images(sc, beta * (1 + e), albedo, mu0, chords).sum()
           - _voxelised_slab_images(sc, beta * (1 - e), albedo, mu0, chords).sum()) / (2 * e)
    assert abs(img - ref_img) < 3.5 * isig, (img, ref_img, isig)
    assert abs(est - ref) < 3.5 * sig, (est, ref, sig)
    assert abs(ref) > 30 * sig  # resolved


@pytest.mark.slow
def test_classic_gradient_along_beta_matches_the_slab_closed_form(orc):
    """Classic-estimator gradient (path score plus shadow-ray terms), first order in the
    homogeneous slab with the camera below the medium: with a measured value M far above the
    images the loss is linear in them, so beta . dE/dbeta / (-2M) estimates
    sum_p tau d i_p / d tau, which the closed form of the slab gives exactly (derivative in tau
    of the single-scattering radiance, averaged over each pixel's solid angle)."""
    beta, albedo, g = 2.5e-3, 0.9, 0.5
    sc = slab_scene(beta, cam_z=-50.0)
    p = synth.Params(albedo=albedo, g=g, sun_zenith=math.radians(30), n_photons=1_600_000, seed=23, max_order=1,
                     rr_threshold=0.0)
    M = 1e6
    meas = np.full(sc.n_pix, M)
    dots = batched(orc, sc, p, 8, lambda q: float(np.dot(sc.beta, orc.full_grad(sc, q, meas, classic=True)["grad"])))
    est_b = dots / (-2.0 * M)                     # per batch: its share of sum_p tau d i_p / d tau
    est, sig = est_b.sum(), est_b.std(ddof=1) * math.sqrt(8)
    sun = np.array([-math.sin(p.sun_zenith), 0.0, -math.cos(p.sun_zenith)])
    mu0, n, ref = math.cos(p.sun_zenith), 12, 0.0
    for pix in range(16):
        i, j = pix % 4, pix // 4
        acc = wsum = 0.0
        for a in range(n):
            for b in range(n):
                px, py = i + (a + 0.5) / n, j + (b + 0.5) / n
                d = rg.pixel_dir(sc, 0, px, py)
                tx = math.tan(0.5 * sc.cam_fov[0])
                x, y = (2 * px / 4 - 1) * tx, (2 * py / 4 - 1) * tx
                w = (1 + x * x + y * y) ** -1.5
                e = 1e-4  # tau d I / d tau of the closed form, by a central difference in beta
                dI = (_slab_radiance(1.0, albedo, g, beta * (1 + e), 200.0, mu0, sun, d)
                      - _slab_radiance(1.0, albedo, g, beta * (1 - e), 200.0, mu0, sun, d)) / (2 * e)
                acc += w * dI
                wsum += w
        ref += acc / wsum
    assert abs(est - ref) < 3.5 * sig + 5e-3 * abs(ref), (est, ref, sig)
    assert abs(ref) > 10 * sig  # resolved


# ------------------------------------------------------------------------------------------
# two species: air (Rayleigh, Eq. Pray / Eq. thetaREY) and aerosol (HG), particle chosen by
# beta_air / beta at each event (Sec. 2.1.2, step iv)


def test_rayleigh_phase_and_sampler(orc):
    # normalised over the sphere (midpoint rule in mu is exact to 1e-9 for this quadratic)
    mus = (np.arange(20000) + 0.5) / 10000.0 - 1.0
    assert abs(2 * math.pi * sum(orc.rayleigh_phase(m) for m in mus) / 10000.0 - 1.0) < 1e-8
    # the sampler inverts the CDF of (3/8)(1 + mu^2) on [-1, 1]: F(mu) = (mu^3 + 3 mu + 4) / 8
    for u in np.linspace(1e-6, 1 - 1e-6, 101):
        c = orc.rayleigh_sample(u)
        assert -1.0 <= c <= 1.0 and abs((c ** 3 + 3 * c + 4) / 8 - u) < 1e-12, (u, c)
    # moments of the sampled cosine: E[mu] = 0, E[mu^2] = 2/5
    us = (np.arange(200000) + 0.5) / 200000
    cs = np.array([orc.rayleigh_sample(u) for u in us])
    assert abs(cs.mean()) < 1e-9 and abs((cs ** 2).mean() - 0.4) < 1e-6


def test_particle_uniform_is_uniform_and_independent_of_the_event_draws(orc):
    """The particle's uniform (the low bits the event's four 23-bit uniforms leave unused) is
    uniform on (0, 1), its bits are those of the Philox block the same counter gives, and it is
    uncorrelated with the event's other draws (HG cosine, azimuth, roulette, free path)."""
    from scipy import stats
    seed, n = 0x1234_5678_9ABC, 200_000
    us, draws = np.empty(n), np.empty((n, 4))
    for t in range(n):
        photon, event = 7919 * t + 13, 1 + t % 37
        us[t] = orc.particle_uniform(seed, photon, event)
        x = orc.philox4x32_10([photon & 0xFFFFFFFF, photon >> 32, event, 0], [seed & 0xFFFFFFFF, seed >> 32])
        draws[t] = [orc.u01(w) for w in x]
        if t < 64:
            m = (x[0] & 511) | ((x[1] & 511) << 9) | ((x[2] & 31) << 18)
            assert us[t] == (2 * m + 1) / 2 ** 24
    assert stats.kstest(us, "uniform").pvalue > 1e-3
    for c in range(4):
        assert abs(np.corrcoef(us, draws[:, c])[0, 1]) < 5.0 / math.sqrt(n)


def _slab_two_species(F, alb_air, alb_aer, g, b_air, b_aer, H, mu0, sun, d):
    """Single scattering by a homogeneous two-species slab: the one-species closed form with
    the scattering phase replaced by the species-weighted sum (b_air alb_air P_Ray + b_aer alb_aer
    P_HG) / (b_air + b_aer) and the total optical depth."""
    b = b_air + b_aer
    mu, tau = d[2], b * H
    cs = float(np.dot(sun, -d))
    p_hg = (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * cs) ** 1.5)
    p_ray = 3.0 / (16 * math.pi) * (1 + cs * cs)
    mix = (b_air * alb_air * p_ray + b_aer * alb_aer * p_hg) / b
    if abs(mu - mu0) < 1e-9:
        return F * mix * tau / mu0 * math.exp(-tau / mu0)
    return F * mix * mu0 / (mu - mu0) * (math.exp(-tau / mu) - math.exp(-tau / mu0))


def _two_species_slab(b_air, b_aer):
    import dataclasses
    sc = slab_scene(b_aer, cam_z=-50.0)
    return dataclasses.replace(sc, beta_air=np.full(sc.nvox, b_air))


def _pixel_avg(sc, fn, pix, n=12):
    i, j = pix % 4, pix // 4
    acc = wsum = 0.0
    tx = math.tan(0.5 * sc.cam_fov[0])
    for a in range(n):
        for b in range(n):
            px, py = i + (a + 0.5) / n, j + (b + 0.5) / n
            x, y = (2 * px / 4 - 1) * tx, (2 * py / 4 - 1) * tx
            w = (1 + x * x + y * y) ** -1.5
            acc += w * fn(rg.pixel_dir(sc, 0, px, py))
            wsum += w
    return acc / wsum


@pytest.mark.slow
def test_two_species_slab_single_scatter(orc):
    """Classic estimate, first order, air + aerosol: the species-weighted closed form."""
    b_air, b_aer, alb_aer, alb_air, g = 1.0e-3, 1.5e-3, 0.8, 1.0, 0.6
    sc = _two_species_slab(b_air, b_aer)
    p = synth.Params(albedo=alb_aer, albedo_air=alb_air, g=g, sun_zenith=math.radians(30), n_photons=6_400_000,
                     seed=24, max_order=1, rr_threshold=0.0)
    nb = 16
    imgs = batched(orc, sc, p, nb, lambda q: orc.render(sc, q, want_L=False, classic=True)["classic"])
    est, sig = imgs.sum(0), imgs.std(0, ddof=1) * math.sqrt(nb)
    sun = np.array([-math.sin(p.sun_zenith), 0.0, -math.cos(p.sun_zenith)])
    mu0 = math.cos(p.sun_zenith)
    ref = np.array([_pixel_avg(sc, lambda d: _slab_two_species(1.0, alb_air, alb_aer, g, b_air, b_aer, 200.0, mu0,
                                                                 sun, d), pix) for pix in range(16)])
    # each pixel sees a few thousand events, so its estimate is skewed (the sum of inverse-square
    # weighted contributions); the total over the pixels is tested at 3.5 sigma, pixels at 5
    tot = imgs.sum(1)
    assert abs(tot.sum() - ref.sum()) < 3.5 * tot.std(ddof=1) * math.sqrt(nb), (tot.sum(), ref.sum())
    assert np.all(np.abs(est - ref) < 5.0 * sig + 2e-3 * ref), ((est - ref) / sig)


@pytest.mark.slow
def test_two_species_gradient_along_the_aerosol(orc):
    """The aerosol gradient with two species (collision score 1/beta_aerosol for aerosol events,
    none for air events): beta_aer . dE/dbeta_aer / (-2M), with a measured value M far above the
    images, estimates sum_p beta_aer d i_p / d beta_aer, from the closed form of the slab."""
    b_air, b_aer, alb_aer, g = 1.0e-3, 1.5e-3, 0.8, 0.6
    sc = _two_species_slab(b_air, b_aer)
    p = synth.Params(albedo=alb_aer, albedo_air=1.0, g=g, sun_zenith=math.radians(30), n_photons=6_400_000, seed=25,
                     max_order=1, rr_threshold=0.0)
    M = 1e6
    meas = np.full(sc.n_pix, M)
    dots = batched(orc, sc, p, 16, lambda q: float(np.dot(sc.beta, orc.full_grad(sc, q, meas, classic=True)["grad"])))
    est_b = dots / (-2.0 * M)
    est, sig = est_b.sum(), est_b.std(ddof=1) * math.sqrt(16)
    sun = np.array([-math.sin(p.sun_zenith), 0.0, -math.cos(p.sun_zenith)])
    mu0, e = math.cos(p.sun_zenith), 1e-4
    ref = 0.0
    for pix in range(16):
        ref += _pixel_avg(sc, lambda d: (_slab_two_species(1.0, 1.0, alb_aer, g, b_air, b_aer * (1 + e), 200.0, mu0,
                                                           sun, d)
                                         - _slab_two_species(1.0, 1.0, alb_aer, g, b_air, b_aer * (1 - e), 200.0, mu0,
                                                             sun, d)) / (2 * e), pix)
    assert abs(est - ref) < 3.5 * sig + 5e-3 * abs(ref), (est, ref, sig)
    assert abs(ref) > 10 * sig


# ------------------------------------------------------------------------------------------
# sun mask M_c (Eq. Cost)


def test_sun_mask_zenith_sun_is_an_image_plane_disc(orc):
    """Upward cameras and the sun at zenith: a pixel centre is masked exactly when its
    image-plane point lies inside the disc of radius tan(rho) (pinhole geometry, no angles)."""
    sc, _ = synth.cfg_blobs16(10)
    rho = math.radians(12.0)
    m = orc.sun_mask(sc, 0.0, 0.0, rho)
    off = 0
    for c in range(sc.n_cams):
        w, h = int(sc.cam_w[c]), int(sc.cam_h[c])
        tx = math.tan(0.5 * sc.cam_fov[c])
        ty = tx * h / w
        i, j = np.meshgrid(np.arange(w) + 0.5, np.arange(h) + 0.5)
        r = np.hypot((2 * i / w - 1) * tx, (2 * j / h - 1) * ty).ravel()
        ref = np.where(r < math.tan(rho), 0, 1).astype(np.uint8)
        far = np.abs(r - math.tan(rho)) > 1e-9
        assert np.array_equal(m[off:off + w * h][far], ref[far])
        assert 0 < (ref == 0).sum() < w * h
        off += w * h


def test_sun_mask_oblique_sun_and_limits(orc):
    """An oblique sun: the masked set equals the pixels whose centre ray makes an angle below
    rho with the sun direction, the angle taken as atan2(|d x s|, d . s); rho = 0 masks
    nothing and rho = pi everything."""
    sc, _ = synth.cfg_blobs16(10)
    zen, az, rho = math.radians(20.0), 0.7, math.radians(8.0)
    s = np.array([math.sin(zen) * math.cos(az), math.sin(zen) * math.sin(az), math.cos(zen)])
    m = orc.sun_mask(sc, zen, az, rho)
    off = 0
    for c in range(sc.n_cams):
        w, h = int(sc.cam_w[c]), int(sc.cam_h[c])
        dirs = [rg.pixel_dir(sc, c, i + 0.5, j + 0.5) for j in range(h) for i in range(w)]
        ang = np.array([math.atan2(np.linalg.norm(np.cross(d, s)), float(np.dot(d, s))) for d in dirs])
        ref = np.where(ang < rho, 0, 1).astype(np.uint8)
        far = np.abs(ang - rho) > 1e-9
        assert np.array_equal(m[off:off + w * h][far], ref[far])
        off += w * h
    assert (m == 0).sum() > 0
    assert np.all(orc.sun_mask(sc, zen, az, 0.0) == 1)
    assert np.all(orc.sun_mask(sc, zen, az, math.pi + 1e-6) == 0)


# ------------------------------------------------------------------------------------------
# colour channels (Eq. channelBeta, Eq. Cost, Eq. divCost1)


def _channel_case(orc):
    import dataclasses
    sc, p = synth.cfg_blobs16(3000)
    air = synth.air_profile(sc.shape, sc.h, 2.0 * synth.KM)
    sc = dataclasses.replace(sc, beta_air=air)
    p = p.replace(albedo_air=0.97)
    meas = orc.forward_images(sc, p.replace(seed=4))[0]
    b = synth.smoothed(sc.beta, sc.shape, 0.3)
    return sc, p, air, meas, b


@pytest.mark.parametrize("surrogate", [False, True])
def test_channels_reparametrisation(orc, surrogate):
    """A channel with sigma = 2 at beta_ref = b / 2 renders the same medium as the one-channel
    problem at b: the same loss, and by the chain rule through Eq. channelBeta twice the
    gradient w.r.t. the aerosol field (a dropped or inverted sigma fails here)."""
    import dataclasses
    sc, p, air, meas, b = _channel_case(orc)
    sb = dataclasses.replace(sc, beta=b)
    if surrogate:
        r0 = orc.surrogate_grad(sb, orc.render(sb, p)["L"], b + air, meas)
    else:
        r0 = orc.full_grad(sb, p, meas)
    r1 = orc.channels_grad(sc, b / 2, [dict(params=p, sigma=2.0, beta_air=air, meas=meas)], surrogate=surrogate)
    assert abs(r1["loss"] - r0["loss"]) <= 1e-12 * r0["loss"]
    assert np.allclose(r1["grad"], 2.0 * r0["grad"], rtol=1e-10, atol=1e-12 * np.abs(r0["grad"]).max())
    assert np.allclose(r1["images"][0], r0["images"], rtol=1e-12, atol=0)


def test_channels_sum_and_single_regulariser(orc):
    """Two identical channels: twice the one-channel loss and gradient, with eta Psi(beta_ref)
    counted once (Eq. Cost), not once per channel."""
    import dataclasses
    sc, p, air, meas, b = _channel_case(orc)
    eta = 0.1
    r0 = orc.full_grad(dataclasses.replace(sc, beta=b), p, meas)
    ch = dict(params=p, sigma=1.0, beta_air=air, meas=meas)
    r2 = orc.channels_grad(sc, b, [ch, ch], eta=eta)
    psi, dpsi = orc.laplacian(dataclasses.replace(sc, beta_air=None), b)
    assert psi > 0
    assert abs(r2["loss"] - (2 * r0["loss"] + eta * psi)) <= 1e-12 * r2["loss"]
    assert np.allclose(r2["grad"], 2 * r0["grad"] + eta * dpsi, rtol=1e-10, atol=1e-12 * np.abs(r2["grad"]).max())


# ------------------------------------------------------------------------------------------
# sharding and threading: the photon-id split does not change the result


def test_photon_range_split_and_threads(orc):
    sc, p = synth.cfg_blobs16(30_000)
    full = orc.render(sc, p, hashes=True, nthreads=3)
    a = orc.render(sc, p.replace(n_photons=10_000, n_photons_total=30_000), hashes=True, nthreads=1)
    b = orc.render(sc, p.replace(n_photons=20_000, photon_offset=10_000, n_photons_total=30_000), hashes=True,
                   nthreads=5)
    assert np.allclose(full["L"], a["L"] + b["L"], rtol=1e-12, atol=1e-300)
    assert np.array_equal(full["hash"], np.concatenate([a["hash"], b["hash"]]))
    skip = np.zeros(30_000, np.uint8)
    skip[10_000:] = 1
    c = orc.render(sc, p, skip=skip, hashes=True)
    assert np.allclose(c["L"], a["L"], rtol=1e-12, atol=1e-300)

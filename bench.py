#!/usr/bin/env python
"""Benchmark: one forward render + full gradient (Eq. Cost, score-function adjoint) of the
64^3 cumulus scene (20 m voxels, cloud fraction 0.3, up to 80 1/km, albedo 0.999, g 0.85,
sun zenith 45 deg) seen by 9 in-situ 128x128 cameras, 1e8 photons per step.

Metric: photon path segments per second = forward-transport voxel crossings of one step
(the same count for any implementation that traces the same photons) / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun each rank traces its own 1e8 photons (distinct
photon ids; weak scaling, no collective on the data path); the timed region is bracketed by
a barrier and a device synchronize, and the max over ranks is taken.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "photon path segments/s (forward + full gradient, 64^3, 9 in-situ cams, 1e8 photons)"
UNIT = "segments/s"
WORKLOAD = "cumulus64: 64^3 x 20 m k^-5/3 cloud field (cf 0.3, max 80 1/km), albedo 0.999, g 0.85, " \
           "sun zenith 45 deg, 9 in-situ 128x128 cams (2 inside the cloud base), 1e8 photons, full gradient"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--photons", type=float, default=1e8)
    ap.add_argument("--grad", default="full", choices=["full", "surrogate"])
    ap.add_argument("--grid-dtype", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--estimator", default="voxel", choices=["voxel", "classic"],
                    help="local estimate of the --single call (the benchmark uses the voxelised one)")
    ap.add_argument("--ref-photons", type=float, default=2e4, help="photons per oracle step (bounded sample)")
    ap.add_argument("--recon-iters", type=int, default=50,
                    help="iterations of --study recon; --study haze runs 2x for L-BFGS")
    ap.add_argument("--render-photons", type=float, default=1e8, help="photons per render of --study haze")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default wavefront shape")
    ap.add_argument("--wavefront", default=None,
                    help="forward trip, forward blocks per SM, pass-2 trip, pass-2 blocks per SM (e.g. 16,3,8,3): set "
                         "instead of autotuning")
    ap.add_argument("--no-replay-form", action="store_true",
                    help="skip the timing of the replay form (W by replay pass 1, no stored events)")
    ap.add_argument("--cpu-photons", type=float, default=1e6, help="photons of the CPU-baseline sample")
    ap.add_argument("--workload", default="cumulus64", choices=["cumulus64", "batch16"])
    ap.add_argument("--single", action="store_true", help="one untimed forward+gradient call (for ncu captures)")
    ap.add_argument("--study", default=None, choices=["precision", "recon", "haze", "bmc", "classic", "species",
                                                      "identify"],
                    help="FP16/BF16 brick forms against FP32 at equal photon count (prints one JSON line)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            cols = [c.strip() for c in line.split(",")]
            if len(cols) < 10 or (self.uuid and cols[1] != self.uuid):
                continue
            try:
                sm.append(float(cols[2]))
                mx.append(float(cols[3]))
            except ValueError:
                continue
            for n, v in zip(names, cols[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_record(kernel, photons, events):
    """DRAM bytes per launch of `kernel`, scaled from the committed ncu capture of a smaller call
    of the same scene: bytes per stored event for the kernels whose traffic is the event stream
    (the forward writes the events, the adjoint reads them), bytes per photon otherwise. None if
    the kernel source has changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
        src = open(os.path.join(ROOT, "paper_1512_02110_gb300", "csrc", "transport.cu"), "rb").read()
        if d.get("transport_cu_sha1") != hashlib.sha1(src).hexdigest():
            return None
        rec = d.get("kernels", {}).get(kernel)
        if rec is None:
            return None
        if rec.get("scale") == "events":
            return float(rec["dram_bytes"]) * events / float(d["events"])
        return float(rec["dram_bytes"]) * photons / float(d["photons"])
    except Exception:
        return None


# ------------------------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)


def oracle_step(sc, p, meas, nthreads=0):
    import oracle
    t0 = time.perf_counter()
    r = oracle.full_grad(sc, p, meas, nthreads=nthreads)
    return time.perf_counter() - t0, r["stats"]["segments"]


def cpu_baseline(sc, p, meas, n_sample):
    """The oracle on the host cores: n_sample photons on all cores, a tenth of them to fit the
    per-call cost of the deterministic stages (LOS, images, back-projection, LOS adjoint) for the
    linear extrapolation to the benchmark's 1e8 photons, and a fifth of them on one core."""
    import oracle
    oracle.build()
    n = int(n_sample)
    q = p.replace(n_photons=n, n_photons_total=n)
    dt, segs = oracle_step(sc, q, meas)
    n_small = max(1, n // 10)
    dts, _ = oracle_step(sc, q.replace(n_photons=n_small, n_photons_total=n_small), meas)
    n1 = max(1, n // 5)
    dt1, segs1 = oracle_step(sc, q.replace(n_photons=n1, n_photons_total=n1), meas, nthreads=1)
    per_photon = max(dt - dts, 0.0) / (n - n_small)
    fixed = max(dt - per_photon * n, 0.0)
    t_full = fixed + per_photon * 1e8
    cores = os.cpu_count()
    return {"value": segs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"cumulus64 scene, {n} photons forward + full gradient incl. all deterministic "
                      f"stages in full (LOS, images, back-projection, LOS adjoint), FP64, OpenMP over {cores} "
                      f"threads; {dt:.2f} s ({n_small} photons: {dts:.2f} s; {n1} photons on 1 thread: {dt1:.2f} s)",
            "step_s": dt, "value_1_core": segs1 / dt1,
            "extrapolated_1e8_photons_s": t_full,
            "extrapolation": f"linear in the photon count from the {n_small}- and {n}-photon runs: "
                             f"{fixed:.2f} s per call + {per_photon * 1e6:.3f} s per 1e6 photons (extrapolated, "
                             f"not measured)"}


def device_bytes_of(fn):
    """Runs fn() and returns (its result, device bytes it left allocated outside torch's cache)."""
    import torch
    torch.cuda.synchronize()
    f0, r0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    out = fn()
    torch.cuda.synchronize()
    f1, r1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    return out, int((f0 - f1) - (r1 - r0))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    import synth
    oracle.build()
    sc, p = synth.cfg_cumulus64()
    sc = sc.with_beta(sc.beta.astype(np.float32).astype(np.float64))
    n = int(args.ref_photons)
    q = p.replace(n_photons=n, n_photons_total=n)
    meas = np.zeros(sc.n_pix)
    for _ in range(args.warmup):
        oracle_step(sc, q.replace(n_photons=1000, n_photons_total=1000), meas)
    times, segs = [], 0
    for _ in range(args.steps):
        dt, segs = oracle_step(sc, q, meas)
        times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = segs / (ms * 1e-3)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("1e8 photons", f"{n} photons (bounded CPU sample)"),
                       "photons_per_step": n, "parallelism": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} photons per step, forward + full gradient, all deterministic stages "
                                       f"in full; warm-up steps use 1000 photons"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# GPU arm


def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import paper_1512_02110_gb300 as m
    import synth

    sc, p = synth.cfg_cumulus64(int(args.photons))
    n = int(args.photons)
    p = p.replace(photon_offset=rank * n, n_photons_total=n)
    torch.cuda.synchronize()
    mem0 = (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved())
    grid = m.Grid.from_scene(sc)
    beta_np = sc.beta.astype(np.float32)
    beta = torch.from_numpy(beta_np).cuda()
    # measured images: a render of the same field with another seed (the end state of a
    # reconstruction, where paths are longest)
    meas = grid.render(beta, m.make_params(p, seed=4), images=True)["images"]
    params = m.make_params(p, grad_mode=args.grad, grid_dtype=args.grid_dtype)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    # wavefront shape picked by the autotuner on this scene (2^24-photon calls), before the warm-up
    if args.wavefront:
        wf = [int(v) for v in args.wavefront.split(",")]
        grid.set_wavefront(*wf)
        wavefront = dict(forward_trip=wf[0], forward_blocks_per_sm=wf[1], replay_trip=wf[2], replay_blocks_per_sm=wf[3])
    else:
        wavefront = None if args.no_autotune else grid.autotune(beta, m.make_params(p, grid_dtype=args.grid_dtype),
                                                                n_sample=1 << 24)

    for _ in range(args.warmup):
        grid.render_grad(beta, params, meas, images=False)
    torch.cuda.synchronize()
    # device memory the handle holds in the timed steps (outside torch's caching allocator)
    handle_bytes = int((mem0[0] - torch.cuda.mem_get_info()[0]) - (torch.cuda.memory_reserved() - mem0[1]))

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    grid.set_profiling(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phase_acc = {}
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(uuid)
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))          # L2 flush between timed steps, outside the event pair
        ev[i][0].record()
        out = grid.render_grad(beta, params, meas, images=False)
        ev[i][1].record()
        for k, (ms, nl) in grid.phase_times().items():
            a = phase_acc.setdefault(k, [0.0, 0])
            a[0] += ms
            a[1] += nl
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    st = grid.stats()
    grid.set_profiling(False)

    ms_step = sum(step_ms) / len(step_ms)
    segs = st["segments"]
    local_vals = torch.tensor([ms_step, segs], dtype=torch.float64, device="cuda")
    if dist is not None:
        mx = local_vals.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        tot = local_vals.clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        ms_job, segs_job = float(mx[0]), float(tot[1])
    else:
        ms_job, segs_job = ms_step, segs
    value = segs_job / (ms_job * 1e-3)

    # Roofline of the dominant kernel. The transport kernels are issue-bound integer / FP32 work
    # (ncu: DRAM < 1 % and L2 < 20 % of peak, issue slots ~65 % busy, ALU pipe the busiest), so
    # the binding roof is the lane issue rate: SMs x 4 schedulers x 32 lanes x max SM clock.
    # Achieved = algorithmic operations per launch / average launch time, with per-unit counts:
    # 15 per transport segment, 27 per event and camera (local estimate: direction, cosine,
    # Henyey-Greenstein phase, two MUFU), 35 per event (scattering sample, roulette), 2 per replay
    # score scatter; replay pass 2 on the stored events 10 per segment (its flights know their last
    # voxel: no extinction and no free-path test before it), 4 B of extinction per flight and the
    # event's 16 B step; the stored-event adjoint 27 per event and camera, 44 B record + 4 B per
    # camera + 8 B of W + the 16 B step per event. The byte form against the measured HBM copy
    # rate (4 B per segment, 8 B per camera per event) is kept beside it, with the stored events'
    # bytes the forward also writes (44 B per event, 4 B per photon) reported apart.
    C = sc.n_cams
    seg1, ev1 = st["segments"], st["events"]
    stored = st.get("events_stored", 0.0)
    if stored > 0:  # W came from the forward's stored events: the replay counters hold pass 2 alone
        seg2, ev2 = st["replay_segments"], st["replay_events"]
    else:           # pass 1 walked the forward paths again (same segments and events)
        seg2, ev2 = st["replay_segments"] - seg1, st["replay_events"] - ev1
    ops_ev = 27 * C + 35
    kernels = {
        "k_transport": (phase_acc["transport"], 15 * seg1 + ops_ev * ev1, 4 * seg1 + 8 * C * ev1),
        "k_replay_pass1": (phase_acc["replay"], 15 * seg1 + ops_ev * ev1, 4 * seg1 + 4 * C * ev1),
        # with stored events pass 2 reads each event's step (w_s, its voxel, the free path left
        # there) instead of summing over the cameras, and only the last voxel's extinction
        "k_replay_pass2": ((phase_acc["replay2"], 10 * seg2 + 35 * ev2 + 2 * st["replay_scatters"],
                            (4 + 16) * ev2 + 8 * st["replay_scatters"]) if stored > 0 else
                           (phase_acc["replay2"], 15 * seg2 + ops_ev * ev2 + 2 * st["replay_scatters"],
                            4 * seg2 + 4 * C * ev2 + 8 * st["replay_scatters"])),
        "k_event_adjoint": (phase_acc.get("event_adjoint", [0.0, 0]), 27 * C * stored,
                            (44 + 4 * C + 8 + 16) * stored),
    }
    kernels = {k: v for k, v in kernels.items() if v[0][1] > 0 and v[1] > 0}
    kern = max(kernels, key=lambda k: kernels[k][0][0])
    (kms, kn), aops, abytes = kernels[kern]
    calls_per_step = kn / args.steps
    per_launch_s = (kms / kn) * 1e-3
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak_ops = props.multi_processor_count * 128 * sm_max * 1e6
    achieved_ops = aops / calls_per_step / per_launch_s
    hbm_peak, peak_kind = peaks()
    hbm_achieved = abytes / calls_per_step / per_launch_s / 1e9
    traffic = traffic_record(kern, n, st["events"])
    roofline = {"bound": "alu", "kernel": kern, "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12,
                "unit": "TOP/s", "frac": achieved_ops / peak_ops, "traffic": traffic,
                "peak_source": f"derived: {props.multi_processor_count} SMs x 128 lanes x {sm_max:.0f} MHz",
                "algorithmic_ops_per_launch": aops / calls_per_step,
                "algorithmic_bytes_per_launch": abytes / calls_per_step, "ms_per_launch": kms / kn,
                "launches_per_step": calls_per_step,
                "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
                        "peak_source": peak_kind,
                        "bytes": "algorithmic: 4 B of extinction per voxel segment, 8 B per camera per event "
                                 "(FP32 read-modify-write of the L tile)",
                        "stored_event_bytes_per_launch": (44 * stored + 4 * st["traced"]) / calls_per_step
                        if kern == "k_transport" and stored > 0 else 0.0},
                "phase_ms_per_step": {k: v[0] / args.steps for k, v in phase_acc.items()}}
    launches = int(sum(v[1] for v in phase_acc.values()))

    # The form whose device memory stays O(grid + images): W per photon by replay pass 1 (a second
    # walk of every path) instead of from the events the forward stores, on a handle of its own
    # with no event budget; same photons, same step.
    replay_form = None
    if not args.no_replay_form and args.grad == "full" and world == 1:
        def make_replay():
            g2 = m.Grid.from_scene(sc)
            g2.set_replay_memory(0)
            if wavefront:
                g2.set_wavefront(wavefront["forward_trip"], wavefront["forward_blocks_per_sm"],
                                 wavefront["replay_trip"], wavefront["replay_blocks_per_sm"])
            for _ in range(2):
                g2.render_grad(beta, params, meas, images=False)
            return g2
        g2, g2_bytes = device_bytes_of(make_replay)
        g2.set_profiling(True)
        r_ms, r_ph = [], {}
        for i in range(3):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g2.render_grad(beta, params, meas, images=False)
            b.record()
            torch.cuda.synchronize()
            r_ms.append(a.elapsed_time(b))
            for k, (ms, _) in g2.phase_times().items():
                r_ph[k] = r_ph.get(k, 0.0) + ms / 3
        st2 = g2.stats()
        g2.close()
        replay_form = {"adjoint": "replay", "ms_per_step": sum(r_ms) / len(r_ms), "step_ms_all": r_ms,
                       "value": st2["segments"] / (sum(r_ms) / len(r_ms) * 1e-3), "unit": UNIT,
                       "device_bytes": g2_bytes, "events_stored": st2["events_stored"],
                       "phase_ms_per_step": r_ph}

    # end to end through the public API, host buffers in pinned memory
    e2e = None
    if not args.no_e2e:
        beta_h = torch.from_numpy(beta_np).pin_memory()
        meas_h = meas.cpu().pin_memory()
        grad_h = torch.empty(sc.nvox, dtype=torch.float64).pin_memory()
        loss_h = torch.empty(1, dtype=torch.float64).pin_memory()
        e_ms = []
        for i in range(max(1, min(args.steps, 3))):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            bd = beta_h.to("cuda", non_blocking=True)
            md = meas_h.to("cuda", non_blocking=True)
            o = grid.render_grad(bd, params, md, images=False)
            grad_h.copy_(o["grad"], non_blocking=True)
            loss_h.copy_(o["loss"], non_blocking=True)
            b.record()
            torch.cuda.synchronize()
            e_ms.append(a.elapsed_time(b))
        e_mean = sum(e_ms) / len(e_ms)
        e2e = {"value": segs_job / (e_mean * 1e-3) if dist is None else segs / (e_mean * 1e-3) * world,
               "unit": UNIT, "h2d_bytes_per_step": int(beta_np.nbytes + meas.numel() * 8),
               "d2h_bytes_per_step": int(sc.nvox * 8 + 8), "ms_per_step": e_mean}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc.with_beta(beta_np.astype(np.float64)), p, meas.cpu().numpy(), args.cpu_photons)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_job, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "photons_per_gpu": n, "grad_mode": args.grad, "wavefront": wavefront,
                           "adjoint": "stored_events" if st.get("events_stored", 0.0) > 0 else "replay",
                           "device_bytes": handle_bytes,
                           "grid_dtype": args.grid_dtype, "l2": "flushed between timed steps (256 MB write)",
                           "parallelism": f"photon-id shards x{world}" if world > 1 else "1 GPU"},
                "segments_per_step": {"forward": segs, "replay": st["replay_segments"],
                                      "los": st["los_segments"], "pixel": st["pixel_segments"],
                                      "backproject": st["backproj_segments"], "los_adjoint": st["losadj_segments"]},
                "events_per_step": st["events"], "step_ms_all": step_ms, "wall_s": wall,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "replay_form": replay_form}
        print(json.dumps(line), flush=True)
    grid.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------------
# single call, batched scenes, precision study


def run_single(args):
    import torch

    import paper_1512_02110_gb300 as m
    import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    sc, p = synth.cfg_cumulus64(int(args.photons))
    grid = m.Grid.from_scene(sc)
    beta = torch.from_numpy(sc.beta.astype(np.float32)).cuda()
    meas = torch.zeros(sc.n_pix, dtype=torch.float64, device="cuda")
    out = grid.render_grad(beta, m.make_params(p, grad_mode=args.grad, grid_dtype=args.grid_dtype,
                                               estimator=args.estimator), meas, images=False)
    torch.cuda.synchronize()
    st = grid.stats()
    print(json.dumps({"single": True, "photons": int(args.photons), "estimator": args.estimator,
                      "loss": out["loss"].item(), "segments": st["segments"], "events": st["events"],
                      "events_stored": st["events_stored"], "shadow_rays": st["shadow_rays"],
                      "shadow_segments": st["shadow_segments"]}))
    return 0


def _timed(fn, steps, warmup, flush):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for i in range(steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return sum(ms) / len(ms), ms


def run_batch(args):
    """Batched workload: 16 scenes of uneven size (24^3-96^3, 3-12 cameras, 1e7-1e8 photons log-uniform),
    forward + full gradient, as one graph launch (one branch per scene, the default form) against
    the persistent form (each transport pass one launch over all scenes) and 16 sequential calls."""
    import torch

    import paper_1512_02110_gb300 as m
    import synth
    torch.cuda.set_device(0)
    scenes = synth.batch_scenes(16, max_photons=args.photons, min_photons=args.photons / 10)
    grids, betas, meas, params = [], [], [], []
    for sc, p in scenes:
        g = m.Grid.from_scene(sc)
        b = torch.from_numpy(sc.beta.astype(np.float32)).cuda()
        meas.append(g.render(b, m.make_params(p, seed=p.seed + 1000))["images"])
        grids.append(g)
        betas.append(torch.from_numpy(synth.smoothed(sc.beta, sc.shape, 0.2).astype(np.float32)).cuda())
        params.append(m.make_params(p, grad_mode="full"))
    batch = m.Batch(grids)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # the default form: one graph branch per scene, each scene's wavefront from its own autotuner
    # run on an eighth of its photons
    if not args.no_autotune:
        for g, b, q in zip(grids, betas, params):
            g.autotune(b, q, n_sample=max(1 << 16, min(int(q.n_photons) // 8, 1 << 27)))
    ms_batch, all_b = _timed(lambda: batch.render_grad(betas, params, meas), args.steps, args.warmup, flush)
    form = batch.form()
    stored_in_graph = sum(1 for g in grids if g.stats()["events_stored"] > 0)
    # the persistent form (each transport pass one launch over all scenes), its wavefront picked
    # by the batch autotuner on an eighth of the photons
    batch.set_form("persistent")
    wavefront = None if args.no_autotune else batch.autotune(betas, params, meas, sample_div=8)
    ms_persistent, _ = _timed(lambda: batch.render_grad(betas, params, meas), args.steps, args.warmup, flush)
    form_p = batch.form()
    batch.set_form("branches")

    def sequential():
        for g, b, q, mm in zip(grids, betas, params, meas):
            g.render_grad(b, q, mm, images=False)

    ms_seq, all_s = _timed(sequential, args.steps, args.warmup, flush)
    segs = 0.0
    for g, b, q, mm in zip(grids, betas, params, meas):
        g.render_grad(b, q, mm, images=False)
        segs += g.stats()["segments"]
    photons = sum(int(q.n_photons) for q in params)
    print(json.dumps({"metric": "photon path segments/s (batched forward + full gradient, 16 uneven scenes)",
                      "value": segs / (ms_batch * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True,
                      "form": form,
                      "persistent_ms_per_step": ms_persistent, "persistent_value": segs / (ms_persistent * 1e-3),
                      "persistent_form": form_p, "persistent_wavefront": wavefront,
                      "sequential_ms_per_step": ms_seq, "sequential_value": segs / (ms_seq * 1e-3),
                      "photons_per_step": photons, "segments_per_step": segs, "scenes_storing_events_in_graph":
                      stored_in_graph, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "batch16: 16 scenes 24^3-96^3 x 20 m, blob/fractal fields, albedo "
                                             "0.99-0.999, g 0.75-0.9, sun 0-60 deg, 3-12 cams of 64/128 px, "
                                             f"{args.photons / 10:.0e}-{args.photons:.0e} photons each",
                                 "l2": "flushed between timed steps"}}), flush=True)
    batch.close()
    return 0


def run_classic_study(args):
    """Forward + full gradient with the classic local estimator (Eq. fle: shadow ray per camera
    and event, score replay plus shadow-ray terms) against the voxelised estimator, cumulus64 at
    1e7 photons. Prints one JSON line with the times and stage split."""
    import torch

    import paper_1512_02110_gb300 as m
    import synth
    torch.cuda.set_device(0)
    n = int(1e7)
    sc, p = synth.cfg_cumulus64(n)
    grid = m.Grid.from_scene(sc)
    beta = torch.from_numpy(sc.beta.astype(np.float32)).cuda()
    meas = grid.render(beta, m.make_params(p, seed=4))["images"]
    out = {"study": "classic", "workload": "cumulus64, 9 in-situ 128x128 cameras", "photons": n}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for est in ("voxel", "classic"):
        prm = m.make_params(p, grad_mode="full", estimator=est)
        grid.render_grad(beta, prm, meas, images=False)  # warm-up
        grid.set_profiling(True)
        a.record()
        grid.render_grad(beta, prm, meas, images=False)
        b.record()
        torch.cuda.synchronize()
        st = grid.stats()
        out[est] = {"ms": a.elapsed_time(b), "phase_ms": {k: v[0] for k, v in grid.phase_times().items() if v[1]},
                    "segments": st["segments"], "replay_segments": st["replay_segments"], "events": st["events"],
                    "shadow_rays": st["shadow_rays"], "shadow_segments": st["shadow_segments"]}
        grid.set_profiling(False)
        # the forward render alone (images, no gradient)
        prm = m.make_params(p, estimator=est)
        grid.render(beta, prm)
        a.record()
        grid.render(beta, prm)
        b.record()
        torch.cuda.synchronize()
        st = grid.stats()
        out[est]["forward_only"] = {"ms": a.elapsed_time(b), "segments": st["segments"], "events": st["events"],
                                    "shadow_rays": st["shadow_rays"], "shadow_segments": st["shadow_segments"]}
    print(json.dumps(out))
    return 0


def run_bmc_study(args):
    """Backward MC (Eq. ble) on the benchmark scene: throughput (paths and voxel segments per
    second), the pixels' relative standard errors, and the images against the forward render
    with the voxelised local estimate at 1e8 photons (the paper's in-situ check, Sec. 3), for
    256 and 1024 paths per pixel; and the paper's own speed comparison of the two renderers in
    its Sec. 4 setting (the haze scene). Prints one JSON line."""
    import torch

    import paper_1512_02110_gb300 as m
    import synth
    torch.cuda.set_device(0)
    sc, p = synth.cfg_cumulus64(int(args.photons))
    grid = m.Grid.from_scene(sc)
    beta = torch.from_numpy(sc.beta.astype(np.float32)).cuda()
    prm = m.make_params(p)
    grid.render(beta, prm)  # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    fwd = grid.render(beta, prm)["images"]
    b.record()
    torch.cuda.synchronize()
    out = {"study": "bmc", "workload": "cumulus64, 9 in-situ 128x128 cameras",
           "forward_voxel_le": {"photons": int(args.photons), "ms": a.elapsed_time(b)}}
    f = fwd.cpu().numpy()
    lit = f > 1e-3 * f.max()
    for n in (256, 1024):
        grid.render_bmc(beta, prm, 32)  # warm-up
        a.record()
        r = grid.render_bmc(beta, prm, n)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        st = grid.stats()
        img, var = r["images"].cpu().numpy(), r["var"].cpu().numpy()
        rse = np.sqrt(var[lit]) / np.maximum(img[lit], 1e-300)
        out[f"bmc_{n}"] = {"ms": ms, "paths_per_s": st["bmc_paths"] / (ms * 1e-3),
                           "segments_per_s": st["bmc_segments"] / (ms * 1e-3), "events_per_path":
                           st["bmc_events"] / st["bmc_paths"], "median_rel_std_err": float(np.median(rse)),
                           "image_rel_l2_vs_forward": float(np.linalg.norm(img - f) / np.linalg.norm(f))}
    # the paper's own comparison (Sec. 4: the voxelised forward render against backward MC, 1e7
    # photons against 1e4 paths per pixel of 36 ground cameras on 80 x 80 x 120 voxels), on the
    # haze scene's aerosol alone (the backward MC renders one species)
    hs, hp, _, _ = synth.cfg_haze80(10_000_000)
    hg = m.Grid.from_scene(hs)
    hb = torch.from_numpy(hs.beta.astype(np.float32)).cuda()
    hprm = m.make_params(hp)
    hg.render(hb, hprm)  # warm-up
    a.record()
    hf = hg.render(hb, hprm)["images"]
    b.record()
    torch.cuda.synchronize()
    fms = a.elapsed_time(b)
    hg.render_bmc(hb, hprm, 16)  # warm-up
    a.record()
    r = hg.render_bmc(hb, hprm, 10_000)
    b.record()
    torch.cuda.synchronize()
    bms = a.elapsed_time(b)
    st = hg.stats()
    hf_np, himg = hf.cpu().numpy(), r["images"].cpu().numpy()
    out["paper_setting"] = {"scene": "haze80 aerosol, 36 ground cameras 64x64 (150 deg)", "fmc_photons": 10_000_000,
                            "fmc_ms": fms, "bmc_paths_per_pixel": 10_000, "bmc_paths": st["bmc_paths"],
                            "bmc_ms": bms, "bmc_over_fmc_time": bms / fms,
                            "image_rel_l2_fmc_vs_bmc": float(np.linalg.norm(hf_np - himg) / np.linalg.norm(himg))}
    print(json.dumps(out))
    return 0


def run_species_study(args):
    """Two-species medium and colour channels at the benchmark scale (cumulus64, 1e8 photons per
    channel, forward + full gradient): one species; air at the sea-level molecular scattering of
    550 nm (0.0116 1/km, 8 km scale height); air 100 times denser; and three RGB channels through
    mst_render_grad_channels (Sec. 4 cross-section ratios, g and irradiance; air scaled as
    wavelength^-4). Measured images come from a seed-4 render of each medium. Prints one JSON
    line with CUDA-event times (3 calls after 1 warm-up) and the forward work."""
    import torch

    import paper_1512_02110_gb300 as m
    import synth
    torch.cuda.set_device(0)
    n = int(args.photons)
    sc, p = synth.cfg_cumulus64(n)
    beta = torch.from_numpy(sc.beta.astype(np.float32)).cuda()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=3):
        fn()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    air0 = synth.air_profile(sc.shape, sc.h, 0.0116 * synth.KM)
    out = {"study": "species", "workload": "cumulus64, 9 in-situ 128x128 cameras", "photons_per_channel": n}
    for name, scale in (("one_species", None), ("air_550nm", 1.0), ("air_550nm_x100", 100.0)):
        grid = m.Grid.from_scene(sc)
        if scale is not None:
            air = torch.from_numpy((air0 * scale).astype(np.float32)).cuda()
            grid.set_air(air, 1.0)
        meas = grid.render(beta, m.make_params(p, seed=4))["images"]
        prm = m.make_params(p, grad_mode="full")
        ms = timed(lambda: grid.render_grad(beta, prm, meas, images=False))
        st = grid.stats()
        grid.set_profiling(True)
        grid.render_grad(beta, prm, meas, images=False)
        torch.cuda.synchronize()
        phases = {k: round(v[0], 3) for k, v in grid.phase_times().items() if v[1]}
        grid.set_profiling(False)
        out[name] = {"ms": ms, "phase_ms": phases, "segments": st["segments"], "events": st["events"],
                     "segments_per_s": st["segments"] / (ms * 1e-3), "events_stored": st["events_stored"],
                     "air_event_fraction": st["air_events"] / max(st["events"], 1.0)}
        grid.close()
    grid = m.Grid.from_scene(sc)
    chans = []
    for sig, g, F, lam, seed in ((16.5, 0.763, 255, 650.0, 3), (16.2, 0.775, 236, 550.0, 5),
                                 (15.9, 0.786, 224, 450.0, 7)):
        air = torch.from_numpy((air0 * (550.0 / lam) ** 4).astype(np.float32)).cuda()
        pm = m.make_params(p, g=g, sun_irradiance=F / 255.0, seed=seed, grad_mode="full")
        grid.set_air(air, 1.0)
        b_mu = (beta.double() * (sig / 16.2)).float()
        meas = grid.render(b_mu, m.make_params(p, g=g, sun_irradiance=F / 255.0, seed=100 + seed))["images"]
        chans.append(dict(params=pm, sigma=sig / 16.2, beta_air=air, albedo_air=1.0, meas=meas))
    grid.set_air(None)
    ms = timed(lambda: grid.render_grad_channels(beta, chans, images=False))
    out["rgb_3_channels"] = {"ms": ms, "ms_per_channel": ms / 3}
    print(json.dumps(out), flush=True)
    return 0


def run_recon_study(args):
    """Reconstruction of the cumulus64 field from its seed-4 images, 1e8 photons per render,
    from beta = 1 1/km everywhere (Sec. 5 loop at the benchmark scale): projected L-BFGS on the
    full gradient (common random numbers), also over 2^3- and 4^3-voxel blocks (Sec. 5), and the
    paper's surrogate loop (Eq. GD, N_GD = 5)
    under each conditioning of the gradient (none, 1/ray count, ray count). Prints one JSON line
    with the loss, epsilon = |b - b_true|_1 / |b_true|_1 and delta_mass = (|b|_1 - |b_true|_1) /
    |b_true|_1 (the paper's two error measures) along each run, and its GPU time."""
    import torch

    import paper_1512_02110_gb300 as m
    import synth
    torch.cuda.set_device(0)
    n = int(args.photons)
    sc, p = synth.cfg_cumulus64(n)
    grid = m.Grid.from_scene(sc)
    b_true = sc.beta.astype(np.float64)
    meas = grid.render(torch.from_numpy(sc.beta.astype(np.float32)).cuda(), m.make_params(p, seed=4))["images"]
    beta0 = np.full(sc.nvox, 1.0 * synth.KM)
    t1 = np.abs(b_true).sum()

    def errs(b):
        return {"epsilon": float(np.abs(b - b_true).sum() / t1), "delta_mass": float((np.abs(b).sum() - t1) / t1)}

    out = {"study": "recon", "photons_per_render": n, "start": "beta = 1 1/km", "initial": errs(beta0)}
    trace = []
    t0 = time.perf_counter()
    st = m.reconstruct(grid, meas, beta0, m.make_params(p, grad_mode="full"), iters=args.recon_iters,
                       method="lbfgs", callback=lambda s: trace.append({"it": s.it, "loss": s.losses[-1], **errs(s.beta)}))
    torch.cuda.synchronize()
    out["lbfgs_full"] = {"iterations": st.it, "renders": st.n_renders, "s": time.perf_counter() - t0,
                         "loss0": st.losses[0], "trace": trace[::5] + trace[-1:]}
    for blk in ((2, 2, 2), (4, 4, 4)):  # the paper's piecewise-constant blocks (Sec. 5): fewer unknowns
        trace = []
        t0 = time.perf_counter()
        st = m.reconstruct(grid, meas, beta0, m.make_params(p, grad_mode="full"), iters=args.recon_iters,
                           method="lbfgs", block=blk,
                           callback=lambda s: trace.append({"it": s.it, "loss": s.losses[-1], **errs(s.beta)}))
        torch.cuda.synchronize()
        out["lbfgs_full_block%d" % blk[0]] = {"block": blk, "unknowns": int(st.x.size), "iterations": st.it,
                                              "renders": st.n_renders, "s": time.perf_counter() - t0,
                                              "loss0": st.losses[0], "trace": trace[::5] + trace[-1:]}
    for cond in ["none", "inv_count", "count"]:
        prm = m.make_params(p, grad_mode="surrogate", conditioning=cond)
        b0 = torch.from_numpy(beta0.astype(np.float32)).cuda()
        L0 = grid.render(b0, prm, images=False, L=True)["L"]
        g0 = grid.surrogate_grad(b0, L0, b0, prm, meas)["grad"].cpu().numpy()
        step = 0.5 * beta0.max() / max(np.abs(g0).max(), 1e-300)  # first step moves beta by at most half
        trace = []
        t0 = time.perf_counter()
        st = m.reconstruct(grid, meas, beta0, prm, iters=args.recon_iters, method="gd", step=step, n_gd=5,
                           callback=lambda s: trace.append({"outer": s.it, "loss": s.losses[-1], **errs(s.beta)}))
        torch.cuda.synchronize()
        out[f"gd_{cond}"] = {"outer_iterations": st.it, "n_gd": 5, "step": step, "renders": st.n_renders,
                             "s": time.perf_counter() - t0, "loss0": st.losses[0], "trace": trace[::5] + trace[-1:]}
    print(json.dumps(out))
    return 0


def run_identify_study(args):
    """Identifiability of the cumulus64 field from its 9 in-situ cameras (Sec. 5, Sec. 6):
    measured images are the true field rendered with 10x the photons of one reconstruction render
    (seed 4); projected L-BFGS on the full gradient with 1e8 photons per render (common random
    numbers) from 0.5x the true field, without and with the Laplacian prior (eta Psi of the true
    field set to the loss of the true field, the noise floor, as in the haze study), and from the
    uniform 1 1/km start with the prior, and from 0.5x the true field under a diagonal
    preconditioner (beta = w x, w the start field). Also the loss along the ray
    beta = s beta_true, s in 0.25 .. 2, and the full gradient's derivative along beta_true at
    s = 0.5 against a central difference of the loss. Prints one JSON line with epsilon and
    delta_mass along each run."""
    import torch

    import paper_1512_02110_gb300 as m
    import synth
    torch.cuda.set_device(0)
    n = int(args.photons)
    sc, p = synth.cfg_cumulus64(n)
    grid = m.Grid.from_scene(sc)
    b_true = sc.beta.astype(np.float64)
    t1 = np.abs(b_true).sum()
    bt = torch.from_numpy(sc.beta.astype(np.float32)).cuda()
    meas = grid.render(bt, m.make_params(p, seed=4, n_photons=10 * n))["images"]
    prm = m.make_params(p, grad_mode="full")
    loss_true = grid.render_grad(bt, prm, meas, images=False)["loss"].item()
    psi_true = grid.regularizer(bt, 1.0).item()
    eta = loss_true / psi_true

    def errs(b):
        return {"epsilon": float(np.abs(b - b_true).sum() / t1), "delta_mass": float((np.abs(b).sum() - t1) / t1)}

    out = {"study": "identify", "photons_per_render": n, "measured_photons": 10 * n,
           "true_field": {"loss": loss_true, "psi": psi_true}, "eta": eta}
    out["loss_along_scale"] = [
        {"s": sc_, "loss": grid.render_grad(torch.from_numpy((sc_ * b_true).astype(np.float32)).cuda(), prm, meas,
                                            images=False)["loss"].item()} for sc_ in (0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 2.0)]
    # the gradient's direction at 0.5 beta_true: its derivative along beta_true against a central
    # difference of the loss along that ray (same photons)
    half = torch.from_numpy((0.5 * b_true).astype(np.float32)).cuda()
    g_half = grid.render_grad(half, prm, meas, images=False)["grad"].cpu().numpy()
    e_lo = grid.render_grad(torch.from_numpy((0.45 * b_true).astype(np.float32)).cuda(), prm, meas,
                            images=False)["loss"].item()
    e_hi = grid.render_grad(torch.from_numpy((0.55 * b_true).astype(np.float32)).cuda(), prm, meas,
                            images=False)["loss"].item()
    out["direction_at_half"] = {"grad_dot_beta_true": float(np.dot(g_half, b_true)),
                                "central_difference": (e_hi - e_lo) / 0.1}
    # runs: (name, start, prior weight, parametrisation); "scaled": beta = w x with w the start field,
    # a diagonal preconditioner under which every voxel moves in proportion to its extinction
    b_half = 0.5 * b_true
    runs = (("half_true_no_prior", b_half, 0.0, None), ("half_true_prior", b_half, eta, None),
            ("half_true_scaled", np.maximum(b_half, 1e-9), 0.0, "scaled"),
            ("uniform_prior", np.full(sc.nvox, 1.0 * synth.KM), eta, None))
    for name, b0, e, par in runs:
        trace = []
        t0 = time.perf_counter()
        P = m.Scaled(b0) if par == "scaled" else None
        st = m.reconstruct(grid, meas, b0, m.make_params(p, grad_mode="full", reg_eta=e), iters=args.recon_iters,
                           method="lbfgs", block=P,
                           callback=lambda s: trace.append({"it": s.it, "loss": s.losses[-1], **errs(s.beta)}))
        torch.cuda.synchronize()
        fin = errs(st.beta)
        out[name] = {"initial": errs(b0), "eta": e, "iterations": st.it, "renders": st.n_renders,
                     "s": time.perf_counter() - t0, "loss0": st.losses[0], "final": fin,
                     "epsilon_below_start": fin["epsilon"] < errs(b0)["epsilon"], "trace": trace[::5] + trace[-1:]}
    print(json.dumps(out))
    return 0


def run_haze_study(args):
    """Reconstruction in the paper's own setting (Sec. 7; synth.cfg_haze80): aerosol haze over
    air on 80 x 80 x 120 voxels, 36 ground cameras, the unknowns the values of the paper's 20 x
    20 x 40 grid (blocks of 4 x 4 x 3 voxels, 16000 unknowns against 147456 pixels). Measured
    images: the true field rendered with 10x the photons of one reconstruction render, seed 4;
    pixels within 10 deg of the sun masked (M_c). Runs: projected L-BFGS on the full gradient
    from beta_aerosol = 0.001 1/km (the score of the aerosol collisions needs a nonzero aerosol
    density) with the Laplacian prior (Eq. Cost, eta = 3000: eta Psi of the true field equals
    the loss's noise floor at 1e8 photons) and without it; the same with a single-scattering
    model (max order 1, the paper's Table 1 baseline), and the full model started from that
    result (the table's third column); the full model with the altitude-weighted prior (Sec. 6,
    W = 1 + z / 2 km); the paper's surrogate loop (Eq. GD, N_GD = 5) from beta_aerosol = 0, its
    null initialisation, with Q = I and Q = 1 / ray count.
    Prints one JSON line: epsilon = |b - b_true|_1 / |b_true|_1 and delta_mass along each run
    (aerosol only; air is known), its renders and GPU+host time, and the loss of the true field
    (the noise floor)."""
    import torch

    import paper_1512_02110_gb300 as m
    import synth
    torch.cuda.set_device(0)
    n = int(args.render_photons)
    eta = 3000.0
    sc, p, coarse, block = synth.cfg_haze80(n)
    grid = m.Grid.from_scene(sc)
    grid.set_air(torch.from_numpy(sc.beta_air.astype(np.float32)).cuda(), p.albedo_air)
    b_true = sc.beta.astype(np.float64)
    t1 = np.abs(b_true).sum()
    bt = torch.from_numpy(sc.beta.astype(np.float32)).cuda()
    t0 = time.perf_counter()
    meas = grid.render(bt, m.make_params(p, seed=4, n_photons=10 * n))["images"]
    mask = grid.sun_mask(p.sun_zenith, p.sun_azimuth, math.radians(10.0))
    torch.cuda.synchronize()

    def errs(b):
        return {"epsilon": float(np.abs(b - b_true).sum() / t1), "delta_mass": float((np.abs(b).sum() - t1) / t1)}

    out = {"study": "haze", "scene": "80x80x120 voxels of 625x625x83.3 m, haze blobs on 20x20x40, air at 550 nm, "
           "36 ground cameras 64x64 (150 deg pinholes), sun zenith 45 deg", "photons_per_render": n, "eta": eta,
           "measured": {"photons": 10 * n, "seed": 4, "s": time.perf_counter() - t0,
                        "masked_pixels": int((mask == 0).sum().item()), "pixels": sc.n_pix},
           "unknowns": int(np.prod(coarse)),
           "true_field": {"loss": grid.render_grad(bt, m.make_params(p, grad_mode="full"), meas, mask,
                                                   images=False)["loss"].item(),
                          "psi": grid.regularizer(bt, 1.0).item()}}
    beta0 = np.full(sc.nvox, 0.001 * synth.KM)
    # (name, prior weight, max scattering order of the model (0: all), start); the single-
    # scattering model (max order 1) fitted to the multiply scattered images is the paper's
    # Table 1 baseline, and its result the start of the paper's "initialized" column
    runs = (("lbfgs_full_prior", eta, 0, "null"), ("lbfgs_full_no_prior", 0.0, 0, "null"),
            ("lbfgs_single_scattering_prior", eta, 1, "null"), ("lbfgs_full_prior_from_single", eta, 0, "single"))
    ends = {}
    for name, e, order, start in runs:
        b_start = beta0 if start == "null" else ends["lbfgs_single_scattering_prior"]
        trace = []
        t0 = time.perf_counter()
        prm = m.make_params(p, grad_mode="full", reg_eta=e, max_order=order)
        st = m.reconstruct(grid, meas, b_start, prm, iters=2 * args.recon_iters, method="lbfgs", mask=mask,
                           block=block,
                           callback=lambda s: trace.append({"it": s.it, "loss": s.losses[-1], **errs(s.beta)}))
        torch.cuda.synchronize()
        ends[name] = st.beta
        out[name] = {"initial": errs(b_start), "max_order": order, "iterations": st.it, "renders": st.n_renders,
                     "s": time.perf_counter() - t0, "loss0": st.losses[0], "final": errs(st.beta),
                     "trace": trace[::10] + trace[-1:]}
    # the altitude-weighted prior of Sec. 6 (Psi = |W Lap beta|^2, W diagonal in altitude), W = 1 + z / 2 km:
    # smoother aloft, where fewer and more oblique rays see each voxel; eta scaled so that eta Psi_W of the
    # true field again equals the noise floor
    z = (np.arange(sc.shape[2]) + 0.5) * sc.h[2]
    grid.set_reg_weights(1.0 + z / 2000.0)
    eta_w = out["true_field"]["loss"] / grid.regularizer(bt, 1.0).item()
    trace = []
    t0 = time.perf_counter()
    st = m.reconstruct(grid, meas, beta0, m.make_params(p, grad_mode="full", reg_eta=eta_w),
                       iters=2 * args.recon_iters, method="lbfgs", mask=mask, block=block,
                       callback=lambda s: trace.append({"it": s.it, "loss": s.losses[-1], **errs(s.beta)}))
    torch.cuda.synchronize()
    grid.set_reg_weights(None)
    out["lbfgs_full_altitude_prior"] = {"initial": errs(beta0), "W": "1 + z / 2 km", "eta": eta_w,
                                        "iterations": st.it, "renders": st.n_renders, "s": time.perf_counter() - t0,
                                        "loss0": st.losses[0], "final": errs(st.beta),
                                        "trace": trace[::10] + trace[-1:]}
    P = m.Blocks(sc.shape, block)
    for cond in ("none", "inv_count"):
        prm = m.make_params(p, grad_mode="surrogate", conditioning=cond, reg_eta=eta)
        b0 = torch.zeros(sc.nvox, dtype=torch.float32, device="cuda")
        L0 = grid.render(b0, prm, images=False, L=True)["L"]
        g0 = P.reduce(grid.surrogate_grad(b0, L0, b0, prm, meas, mask)["grad"].cpu().numpy())
        step = 0.02 * synth.KM / max(np.abs(g0).max(), 1e-300)  # first step: at most 0.02 1/km per block
        trace = []
        t0 = time.perf_counter()
        st = m.reconstruct(grid, meas, np.zeros(sc.nvox), prm, iters=args.recon_iters, method="gd", step=step,
                           n_gd=5, mask=mask, block=block,
                           callback=lambda s: trace.append({"outer": s.it, "loss": s.losses[-1], **errs(s.beta)}))
        torch.cuda.synchronize()
        out[f"gd_null_init_{cond}"] = {"initial": errs(np.zeros(sc.nvox)), "outer_iterations": st.it, "n_gd": 5,
                                       "step": step, "renders": st.n_renders, "s": time.perf_counter() - t0,
                                       "loss0": st.losses[0], "final": errs(st.beta),
                                       "trace": trace[::10] + trace[-1:]}
    print(json.dumps(out))
    return 0

def run_precision_study(args):
    """Image and gradient error of the FP32 / FP16 / BF16 brick forms at N photons against a
    10 N-photon FP32 reference (relative L2), and their step times."""
    import torch

    import paper_1512_02110_gb300 as m
    import synth
    torch.cuda.set_device(0)
    n = int(args.photons)
    sc, p = synth.cfg_cumulus64(n)
    grid = m.Grid.from_scene(sc)
    beta = torch.from_numpy(sc.beta.astype(np.float32)).cuda()
    meas = grid.render(beta, m.make_params(p, seed=4))["images"]
    beta_e = torch.from_numpy(synth.smoothed(sc.beta, sc.shape, 0.2).astype(np.float32)).cuda()
    reps = 10
    ref = grid.render_grad(beta_e, m.make_params(p, grad_mode="full", seed=11, n_photons=reps * n), meas)
    ref_img, ref_grad = ref["images"], ref["grad"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    res = {}
    for kind in ("f32", "f16", "bf16"):
        q = m.make_params(p, grad_mode="full", seed=12, grid_dtype=kind)
        out = grid.render_grad(beta_e, q, meas)
        ei = float((out["images"] - ref_img).norm() / ref_img.norm())
        eg = float((out["grad"] - ref_grad).norm() / ref_grad.norm())
        ms, _ = _timed(lambda: grid.render_grad(beta_e, q, meas, images=False), args.steps, args.warmup, flush)
        res[kind] = {"image_rel_l2": ei, "grad_rel_l2": eg, "ms_per_step": ms}
    print(json.dumps({"study": "precision", "photons": n, "reference": f"FP32, {reps * n} photons (seed 11)",
                      "forms": res}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.single:
        return run_single(args)
    if args.study == "precision":
        return run_precision_study(args)
    if args.study == "recon":
        return run_recon_study(args)
    if args.study == "haze":
        return run_haze_study(args)
    if args.study == "bmc":
        return run_bmc_study(args)
    if args.study == "classic":
        return run_classic_study(args)
    if args.study == "species":
        return run_species_study(args)
    if args.study == "identify":
        return run_identify_study(args)
    if args.workload == "batch16":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

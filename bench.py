"""Benchmark: rotations/s of 128^3 energy + force (+ torque) fields for the
peg-in-hole skeleton workload (5000 + 5000 points, 1024 random rotations),
with p50/p99 pose-query latency.

One step = the whole path over one batch: splat both parts, derive the
stationary spectrum and the moving grid, energy/force for every rotation,
torque by least squares over the 6 nearest rotations, and a batch of 1024
pose queries.  `value` counts rotations per second with inputs resident on
the device; `e2e` repeats the step through the public API from pinned host
buffers, with the host->device input copies and the device->host read of the
query results inside the timed region.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank runs its own rotation batch (seeded by rank): weak
scaling, no collective on the data path.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "rotations/s of 128^3 energy+force fields (+FD torque, +1024 pose queries per batch)"
UNIT = "rotations/s"
N_GRID = 128
N_ROT = 1024
N_QUERY = 1024


NOMINAL_HBM_GBS = 7700.0  # B300 HBM3e, NVIDIA's figure (context beside the measured copy peak)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ------------------------------------------------------------ clock sampler
REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
           0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
           0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


class ClockSampler:
    def __init__(self, device_index):
        self.samples = []
        self.proc = None
        self.dev = device_index

    def __enter__(self):
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            sel = []
        cmd = ["nvidia-smi", *sel, "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,power.draw",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 3:
                try:
                    self.samples.append((float(parts[0]), float(parts[1]), int(parts[2], 16)))
                except ValueError:
                    pass

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        mask = 0
        for s in self.samples:
            mask |= s[2]
        return {"sm_mhz": statistics.median(s[0] for s in self.samples),
                "sm_max_mhz": max(s[1] for s in self.samples),
                "reasons": [v for k, v in REASONS.items() if mask & k and k != 0x1],
                "samples": len(self.samples)}


# ------------------------------------------------------------------ oracle
def oracle_rotation_sample(s1, s2, quats, n, count):
    """The FP64 oracle, as it stands, on `count` rotations of the workload:
    per rotation the resample and the energy/force fields by the oracle's own
    transform.  Returns (seconds per rotation, splat seconds, the two grids,
    sample description)."""
    import oracle
    t0 = time.perf_counter()
    r1 = oracle.splat(n, s1.pts, s1.sigma)
    r2 = oracle.splat(n, s2.pts, s2.sigma)
    t_splat = time.perf_counter() - t0
    t0 = time.perf_counter()
    for q in quats[:count]:
        oracle.fields(r1, oracle.resample(r2, oracle.quat_to_rot(q)))
    t_rot = (time.perf_counter() - t0) / count
    return t_rot, t_splat, (r1, r2), (f"{count} rotations of the {n}^3 workload (resample + E/F fields by the "
                                      f"oracle's own transform), splat of both parts timed once")


def numpy_fft_sample(r1, r2, quats, count):
    """A library CPU reference: the same E/F build with numpy's pocketfft in
    float64 (one process, one thread): rfftn of the rotated grid, the
    conjugate product, four irfftn with the i pi k~ multipliers (Nyquist 0).
    The rotated grids come from the oracle's resample, outside the timing."""
    import oracle
    n = r1.shape[0]
    h3 = (2.0 / n) ** 3
    k = np.fft.fftfreq(n, 1.0 / n)
    k[n // 2] = 0.0
    kx = np.fft.rfftfreq(n, 1.0 / n)
    kx[-1] = 0.0
    mult = (np.pi * kx[None, None, :], np.pi * k[None, :, None], np.pi * k[:, None, None])
    grids = [oracle.resample(r2, oracle.quat_to_rot(q)) for q in quats[:count]]
    t0 = time.perf_counter()
    A = np.fft.rfftn(r1)
    for g in grids:
        S = A * np.conj(np.fft.rfftn(g)) * h3
        np.fft.irfftn(S, s=(n, n, n), axes=(0, 1, 2))
        for m in mult:
            np.fft.irfftn(S * (1j * m), s=(n, n, n), axes=(0, 1, 2))
    return (time.perf_counter() - t0) / count


def cpu_baselines(s1, s2, n, count=16):
    """The CPU baseline: the oracle on `count` rotations at the bench's grid,
    numpy.fft (float64) on 4 rotations of the same grids, and the oracle's
    direct O(N^6) correlation sum at 32^3 (the c1 pair, identity rotation)."""
    import oracle
    quats = synth.random_quaternions(0, count)
    t_rot, t_splat, (r1, r2), desc = oracle_rotation_sample(s1, s2, quats, n, count)
    t_np = numpy_fft_sample(r1, r2, quats, 4)
    a1, a2 = synth.c1_pair(0)
    g1, g2 = oracle.splat(32, a1.pts, a1.sigma), oracle.splat(32, a2.pts, a2.sigma)
    t0 = time.perf_counter()
    oracle.correlate_direct(g1, g2)
    t_direct = time.perf_counter() - t0
    return {"value": round(1.0 / t_rot, 4), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": desc, "splat_s": round(t_splat, 2), "s_per_rotation": round(t_rot, 3),
            "numpy_fft_f64": {"value": round(1.0 / t_np, 4), "unit": UNIT, "cores": 1,
                              "sample": f"4 rotations of the {n}^3 workload: rfftn + product + 4 irfftn "
                                        f"(numpy pocketfft, float64; resample outside the timing)"},
            "direct_sum_32": {"seconds": round(t_direct, 3), "cores": os.cpu_count(),
                              "sample": "E over all 32^3 lags by the O(N^6) Riemann sum (Eqs. 1/3), c1 pair, "
                                        "identity rotation"}}


# ------------------------------------------------------- multi-rank logic
def rank_rotations(rank, R):
    """Each rank builds its own rotation batch (weak scaling): seed = rank, so
    rank 0 has the workload's own 1024 rotations."""
    return synth.random_quaternions(rank, R).astype(np.float32)


def max_over_ranks(x, world, device=None):
    """Slowest rank's value: the job is done when the last rank is."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job units per second: every rank's units over the slowest time."""
    return world * units_per_rank / seconds


def tune_is_pencil(ctx, n):
    return bool(ctx.tune_get(n)[1]) or os.environ.get("HF_PIPELINE") == "pencil"


# ------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1711_05017_b300 as hf
    from paper_1711_05017_b300 import _binding as hf_binding
    from paper_1711_05017_b300 import build

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    n, R = args.n, args.rotations
    s1, s2 = synth.c2_pair(0)
    quats = rank_rotations(rank, R)
    rng = np.random.default_rng(1000 + rank)
    tq_h = np.concatenate([rng.uniform(-1, 1, (N_QUERY, 3)), synth.random_quaternions(2000 + rank, N_QUERY)],
                          axis=1).astype(np.float32)

    ctx = hf.Context(local_rank)
    pts1, sig1 = torch.as_tensor(s1.pts, dtype=torch.float32, device=dev), torch.as_tensor(s1.sigma, dtype=torch.float32, device=dev)
    pts2, sig2 = torch.as_tensor(s2.pts, dtype=torch.float32, device=dev), torch.as_tensor(s2.sigma, dtype=torch.float32, device=dev)
    g1 = torch.empty((n, n, n), device=dev)
    g2 = torch.empty((n, n, n), device=dev)
    ctx.density_build(n, pts1, sig1, out=g1)
    ctx.density_build(n, pts2, sig2, out=g2)
    p1, p2 = ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING)
    tune = None
    if not args.no_tune:  # launch shape for this grid size, timed on this device or read from --tune-cache
        c, pen, rps = ctx.autotune(n, args.tune_cache)
        tb, tc = ctx.tune_tiles(n)
        tune = {"chunk": c, "pipeline": "pencil" if pen else "slab", "tile_b": tb, "tile_c": tc,
                "lanes_tuned": ctx.tune_lanes(n), "lanes": 1, "ef_rot_per_s": round(rps, 1)}
        # the timed step runs one pipeline, so that each kernel's event time is its own (two
        # pipelines overlap the passes of neighbouring chunks); the two-pipeline rate is measured
        # after it
        ctx.tune_lanes(n, 1)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T)
    tq = torch.as_tensor(tq_h, device=dev)
    qout = torch.empty((N_QUERY, 7), device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ctx.density_build(n, pts1, sig1, out=g1)
        ctx.density_build(n, pts2, sig2, out=g2)
        p1.update(g1)
        p2.update(g2)
        fs.compute(p1, p2, quats)
        fs.query_batch(tq, out=qout)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(reset=True)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        h0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        host_ms = (time.perf_counter() - h0) * 1e3 / args.steps  # issue time: above ms, the GPU waits on the host
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    ms = max_over_ranks(ms, world, dev)
    value = job_throughput(R, world, ms / 1e3)

    # ---- roofline of the dominant kernel (algorithmic bytes / event-timed duration)
    he = n * n * (n // 2 + 1) * 8  # one half-spectrum intermediate, bytes
    n3b = 4 * n**3
    chunk = min(ctx.tune_get(n)[0], R) if not os.environ.get("HF_ROT_CHUNK") else int(os.environ["HF_ROT_CHUNK"])
    alg = {  # bytes per launch: inputs read once + outputs written
        # pass A samples the moving grid through the texture units (read once,
        # then L2/texture-cache resident) and writes the chunk's spectra
        "passA": n3b + chunk * he,
        "passB": chunk * he + he + 2 * chunk * he,
        "passC": 2 * chunk * he + chunk * 4 * n3b,
        "torque": R * n3b + R * 3 * n3b,
        "splat": n3b,
        "passB_fwd": 2 * he,
        "passA_stationary": n3b + he,
        "query": N_QUERY * 7 * 4 * 2,
        "resample": n3b + chunk * n3b,
    }
    # dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of the
    # pass C kernel of this launch shape (tile 5: planes staged by bulk
    # copies, 256 threads per CTA; tile 6: the same with 512 threads) over 32
    # rotations at 128^3, scaled to this launch's rotations: the traffic is
    # per rotation (each reads its own two spectra and writes its own four
    # fields); none for another launch shape
    captured = {5: 1.5717e9, 6: 1.5738e9}
    tc_now = ctx.tune_tiles(n)[1]
    traffic = ({"passC": captured[tc_now] * chunk / 32}
               if n == 128 and not tune_is_pencil(ctx, n) and tc_now in captured else {})
    hbm_peak, peak_kind = peaks()
    kernels = {}
    for k, (cnt, tot) in prof.items():
        avg = tot / cnt
        kernels[k] = {"launches": cnt, "avg_us": round(avg * 1e3, 2), "share": None,
                      "alg_GBps": round(alg.get(k, 0) / (avg * 1e-3) / 1e9, 1)}
    tot_all = sum(v[1] for v in prof.values()) or 1.0
    for k in kernels:
        kernels[k]["share"] = round(prof[k][1] / tot_all, 3)
    # the method's own bytes (the fields a launch writes; inputs amortised over
    # the batch): 16 N^3 per rotation for E + F, 12 N^3 for the torque's T;
    # a kernel that only moves intermediates of the design has none
    method = {"passC": chunk * 4 * n3b, "torque": R * 3 * n3b}
    dom = max(prof, key=lambda k: prof[k][1]) if prof else None
    roof = None
    if dom:
        dur = prof[dom][1] / prof[dom][0] * 1e-3
        achieved = method.get(dom, alg.get(dom, 0)) / dur / 1e9
        design = alg.get(dom, 0) / dur / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "bytes": "method: 16 N^3 of E+F written per rotation x rotations per launch",
                "alg_bytes_per_launch": method.get(dom, alg.get(dom, 0)),
                "achieved_design": round(design, 1), "frac_design": round(design / hbm_peak, 4),
                "design_bytes_per_launch": alg.get(dom, 0),
                "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                "traffic": traffic.get(dom),
                # the whole step against the method's floor: E + F + T written (28 N^3 per rotation)
                "step_achieved": round(28 * n**3 * value / world / 1e9, 1),
                "step_frac": round(28 * n**3 * value / world / 1e9 / hbm_peak, 4)}
    launches = sum(v[0] for v in prof.values())

    # ---- end to end through the public API from pinned host buffers
    hp = [torch.as_tensor(a, dtype=torch.float32).pin_memory() for a in (s1.pts, s1.sigma, s2.pts, s2.sigma)]
    tq_pin = torch.as_tensor(tq_h).pin_memory()
    res_pin = torch.empty((N_QUERY, 7), dtype=torch.float32).pin_memory()
    dbuf = [torch.empty_like(h, device=dev) for h in hp]
    tq_d = torch.empty_like(tq_pin, device=dev)

    def e2e_step():
        for d, h in zip(dbuf, hp):
            d.copy_(h, non_blocking=True)
        tq_d.copy_(tq_pin, non_blocking=True)
        ctx.density_build(n, dbuf[0], dbuf[1], out=g1)
        ctx.density_build(n, dbuf[2], dbuf[3], out=g2)
        p1.update(g1)
        p2.update(g2)
        fs.compute(p1, p2, quats)
        fs.query_batch(tq_d, out=qout)
        res_pin.copy_(qout, non_blocking=True)
        stream.synchronize()

    e2e_steps = max(2, args.steps // 2)
    e2e_step()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, world, dev)
    h2d = sum(h.numel() * 4 for h in hp) + tq_pin.numel() * 4 + quats.nbytes
    d2h = res_pin.numel() * 4

    # ---- pose-query latency (host call -> 7 floats back), 1 kHz-style random walk
    tw = synth.translation_walk(7 + rank, 2000)
    qw = synth.quaternion_walk(8 + rank, 2000)
    def query_walk():
        lat = []
        for i in range(2000):
            a = time.perf_counter()
            fs.query(tw[i], qw[i], k=4)
            lat.append((time.perf_counter() - a) * 1e6)
        return np.array(lat[100:])

    lat = query_walk()  # a kernel launch and a synchronisation per query
    lat_res = None
    try:  # the resident query kernel: no launch per query (the serving path)
        ctx.resident_queries(True)
        lat_res = query_walk()
    except hf.HFError:
        pass
    finally:
        ctx.resident_queries(False)

    # ---- the tuner's two-pipeline shape, when it chose it: the same step
    two_lanes = None
    if tune and tune.get("lanes_tuned") == 2:
        ctx.tune_lanes(n, 2)
        fs2 = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T)
        ctx.tune_lanes(n, 1)

        def step2():
            ctx.density_build(n, pts1, sig1, out=g1)
            ctx.density_build(n, pts2, sig2, out=g2)
            p1.update(g1)
            p2.update(g2)
            fs2.compute(p1, p2, quats)
            fs2.query_batch(tq, out=qout)

        for _ in range(args.warmup):
            step2()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step2()
        e1.record(stream)
        torch.cuda.synchronize()
        ms2 = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
        two_lanes = {"value": round(job_throughput(R, world, ms2 / 1e3), 1), "unit": UNIT,
                     "ms_per_step": round(ms2, 3), "note": "two pipelines alternating rotation chunks on two "
                     "streams (the tuner's choice); kernels overlap, so the roofline above uses one pipeline"}
        fs2.release()

    # ---- plain path: the same kernels, one rotation per launch
    plain = None
    if not args.no_plain and rank == 0:
        os.environ["HF_ROT_CHUNK"] = "1"
        os.environ["HF_LANES"] = "1"
        fs1 = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T)
        del os.environ["HF_ROT_CHUNK"]
        del os.environ["HF_LANES"]

        def plain_step():
            ctx.density_build(n, pts1, sig1, out=g1)
            ctx.density_build(n, pts2, sig2, out=g2)
            p1.update(g1)
            p2.update(g2)
            fs1.compute(p1, p2, quats)
            fs1.query_batch(tq, out=qout)

        plain_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plain_step()
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"value": round(R / (pms / 1e3), 1), "unit": UNIT, "ms_per_step": round(pms, 2),
                 "speedup_of_batched": round((R / (ms / 1e3)) / (R / (pms / 1e3)), 3)}
        fs1.release()

    # ---- CPU baseline (the oracle on this host's cores), rank 0, N = 1 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baselines(s1, s2, n, args.cpu_rotations)

    serving = batch = None
    if rank == 0 and world == 1 and (args.serve_seconds > 0 or args.batch_steps > 0 or args.precision_rotations > 0
                                     or args.spectral):
        del fs
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.batch_steps > 0:
        batch = run_batch(args, local_rank)
        torch.cuda.empty_cache()
    spectral = None
    if rank == 0 and world == 1 and args.spectral:
        spectral = run_next_rows(args, local_rank)
        torch.cuda.empty_cache()
    precision = None
    if rank == 0 and world == 1 and args.precision_rotations > 0:
        precision = run_precision(args, local_rank)
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.serve_seconds > 0:
        serving = run_serving(args, local_rank)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "host_issue_ms_per_step": round(host_ms, 3),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"c2 peg-in-hole skeletons, {n}^3 grid, 5000+5000 points, radii U(0.02,0.08), "
                                   f"{R} random rotations per rank, E+F+T fields, {N_QUERY} pose queries per step",
                       "grid": n, "rotations_per_rank": R, "launch_shape": tune, "parallelism": f"replicas x{world} (rotation batches)",
                       "l2": "working set > L2 (fields 60 GB per rank)"},
            "e2e": {"value": round(world * R / e2e_s, 1), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "query_latency_us": {"p50": round(float(np.percentile(lat, 50)), 1),
                                 "p99": round(float(np.percentile(lat, 99)), 1),
                                 "max": round(float(np.max(lat)), 1), "n": int(lat.size),
                                 "budget_us": 1000, "path": "a launch per query (hf_query)",
                                 "measured": "Python call to 7 floats back, idle device, 1 kHz-style pose walk",
                                 "resident_path": None if lat_res is None else {
                                     "p50": round(float(np.percentile(lat_res, 50)), 1),
                                     "p99": round(float(np.percentile(lat_res, 99)), 1),
                                     "max": round(float(np.max(lat_res)), 1)}},
            "paper_reported": {"product_and_inverse_fft_s_per_rotation": "up to 0.1", "grid_nodes": "1e6-1e7",
                               "hardware": "NVIDIA Tesla K20c (Kepler), cuFFT", "source": "Section 4.2, Fig. 6b"},
            "gpu_launches": int(launches),
            "roofline": roof,
            "kernels": kernels,
            "plain_path": plain,
            "two_pipelines": two_lanes,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            # bulk-copy waits that gave up in this run (each would have left its block's output invalid)
            "bulk_wait_timeouts": int(hf_binding.lib().hf_bulk_timeouts(0)),
            "batch": batch,
            "precision": precision,
            "next_rows": spectral,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)


# ------------------------------------------------------- uneven batch workload
BATCH_SLOTS = 8  # field sets per (size, rotations): 64 pairs' fields (250 GB) plus scratch exceed the device
# graph branches: 1 (builds in sequence inside the graph).  Measured on B300
# with 8 slots per size: 1 branch 50.4k rot/s, 3 branches 46.7k, 24 branches
# 47.5k -- concurrent 96^3/128^3 builds contend for SMs and L2
BATCH_LANES = 1


def run_batch(args, local_rank):
    """64 part pairs, grid sizes 64/96/128 (24/24/16), 1000-8000 points each,
    256 rotations per pair, E+F: launch shapes from the autotuner, the whole
    build recorded as one CUDA graph and replayed; the same builds issued pair
    by pair without the graph on one stream for comparison."""
    import tempfile

    import torch
    import paper_1711_05017_b300 as hf
    dev = torch.device("cuda", local_rank)
    specs = synth.c3_pairs(0)
    ctx = hf.Context(local_rank)
    flags = hf.HF_E | hf.HF_F
    tune = {}
    t0 = time.perf_counter()
    with tempfile.TemporaryDirectory() as d:
        for n in sorted(set(p.n for p in specs)):
            c, pen, rps = ctx.autotune(n, os.path.join(d, "tune.json"))
            tb, tc = ctx.tune_tiles(n)
            tune[n] = {"chunk": c, "pipeline": "pencil" if pen else "slab", "tile_b": tb, "tile_c": tc,
                       "lanes": ctx.tune_lanes(n), "rot_per_s": round(rps, 1)}
        with open(os.path.join(d, "tune.json")) as f:
            tune["cache"] = json.load(f)["tune"]
    tune_s = time.perf_counter() - t0
    pairs, quats = [], []
    for p in specs:
        cu = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)  # noqa: E731
        g1 = ctx.density_build(p.n, cu(p.s1.pts), cu(p.s1.sigma))
        g2 = ctx.density_build(p.n, cu(p.s2.pts), cu(p.s2.sigma))
        pairs.append((ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING)))
        quats.append(synth.random_quaternions(p.quat_seed, p.n_rot).astype(np.float32))
    R = [p.n_rot for p in specs]
    total = sum(R)
    b = hf.Batch(ctx, pairs, R, flags, slots_per_size=BATCH_SLOTS)
    for i, q in enumerate(quats):
        b.set_rotations(i, q)
    t0 = time.perf_counter()
    b.capture(BATCH_LANES)
    cap_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    steps, warm = args.batch_steps, 3
    for _ in range(warm):
        b.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        b.launch()
    e1.record(stream)
    torch.cuda.synchronize()
    g_ms = e0.elapsed_time(e1) / steps
    # the same builds pair by pair, no graph, one stream, into one set per (size, rotations)
    sets = {}
    for p in specs:
        if (p.n, p.n_rot) not in sets:
            sets[(p.n, p.n_rot)] = ctx.fieldset(p.n, p.n_rot, flags)

    def sequential():
        for p, pr, q in zip(specs, pairs, quats):
            sets[(p.n, p.n_rot)].compute(pr[0], pr[1], q)

    sequential()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(max(1, steps // 2)):
        sequential()
    e1.record(stream)
    torch.cuda.synchronize()
    s_ms = e0.elapsed_time(e1) / max(1, steps // 2)
    # the same batch as ONE launch of the work-queue kernel
    queue = None
    try:
        t0 = time.perf_counter()
        b.capture_queue(chunk=args.queue_chunk)
        qcap_s = time.perf_counter() - t0
        for _ in range(warm):
            b.launch()
        b.status()
        e0.record(stream)
        for _ in range(steps):
            b.launch()
        e1.record(stream)
        torch.cuda.synchronize()
        items, runs = b.status()
        q_ms = e0.elapsed_time(e1) / steps
        queue = {"value": round(total / (q_ms / 1e3), 1), "unit": UNIT, "ms_per_launch": round(q_ms, 2),
                 "kernel_launches_per_batch": 1, "work_items": items, "item_runs": runs,
                 "rotations_per_chunk": args.queue_chunk, "capture_s": round(qcap_s, 3), "launches": steps,
                 "vs_graph": round(g_ms / q_ms, 3)}
    except hf.HFError as ex:
        queue = {"error": str(ex)}
    out = {"workload": "64 part pairs, grids 64^3/96^3/128^3 (24/24/16), 1000-8000 skeleton points each, "
                       "256 random rotations per pair, E+F fields", "pairs": len(specs), "rotations": total,
           "one_launch_queue": queue,
           "graph": {"value": round(total / (g_ms / 1e3), 1), "unit": UNIT, "ms_per_launch": round(g_ms, 2),
                     "slots": b.slots(), "slots_per_size": BATCH_SLOTS, "lanes": BATCH_LANES or b.slots(), "capture_s": round(cap_s, 3),
                     "launches": steps},
           "sequential_no_graph": {"value": round(total / (s_ms / 1e3), 1), "unit": UNIT,
                                   "ms_per_pass": round(s_ms, 2)},
           "speedup_of_graph": round(s_ms / g_ms, 3), "autotune": tune, "autotune_s": round(tune_s, 1)}
    b.release()
    for v in sets.values():
        v.release()
    del pairs
    return out


# ------------------------------------------------------- precision variant
def run_precision(args, local_rank):
    """256^3, 20000 + 20000 skeleton points (radii U(0.01, 0.05)), 512
    rotations, E+F: the plain FP32 pipeline against the y stages as split
    BF16 / FP16 DFT-matrix GEMMs on the tensor cores.  Throughput per variant,
    the tensor-core kernel against the tensor peak, error against the FP32
    path on 2 rotations, and (--precision-oracle K) per-field error against
    the FP64 oracle on rotations 0..K-1 of the same rotation set, for parts
    splatted by the oracle from a 400-point subset of each part."""
    import torch
    import paper_1711_05017_b300 as hf
    from paper_1711_05017_b300 import _binding as B
    dev = torch.device("cuda", local_rank)
    n, R = 256, args.precision_rotations
    s1, s2 = synth.c4_pair(0)
    ctx = hf.Context(local_rank)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)  # noqa: E731
    g1 = ctx.density_build(n, cu(s1.pts), cu(s1.sigma))
    g2 = ctx.density_build(n, cu(s2.pts), cu(s2.sigma))
    p1, p2 = ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING)
    q = synth.random_quaternions(0, R).astype(np.float32)
    stream = torch.cuda.current_stream()
    B.lib().hf_tc_timeouts(1)
    variants = (("fp32", 0), ("split_bf16", hf.HF_PREC_SPLIT_BF16), ("split_f16", hf.HF_PREC_SPLIT_F16))
    out, ref2 = {}, None
    hbm_peak, _ = peaks()
    _, tc_peak, tc_kind = tensor_peak()
    for name, fl in variants:
        fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | fl)
        fs.compute(p1, p2, q)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        e0.record(stream)
        for _ in range(reps):
            fs.compute(p1, p2, q)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        prof = ctx.profile_read(reset=True)
        ctx.profile(False)
        f2 = np.stack([np.stack([fs.get(r, f).cpu().numpy().astype(np.float64) for f in range(4)]) for r in (0, 1)])
        if ref2 is None:
            ref2 = f2
        v = {"value": round(R / (ms / 1e3), 1), "unit": UNIT, "ms_per_build": round(ms, 2),
             "max_abs_err_vs_fp32_over_max": [float(np.abs(f2[:, f] - ref2[:, f]).max() / np.abs(ref2[:, f]).max())
                                              for f in range(4)],
             "kernels_avg_us": {k: round(t / c * 1e3, 1) for k, (c, t) in prof.items()}}
        if "y_tc" in prof:
            cnt, tot = prof["y_tc"]
            chunk = ctx.tune_get(n)[0]
            # tensor FLOPs per rotation: per 32-column tile 2 stages x 4 M
            # tiles x 2 K steps x (2 x 128 x 32 x 16) of DFT-matrix product,
            # over 1032 tiles, for 1 forward and 3 inverse transforms; the
            # split issues each 3 times (hi hi + hi lo + lo hi) -- the useful
            # flops are the DFT products once
            useful = 4 * 1032 * 16 * (2 * 128 * 32 * 16) * R * reps
            flops = 3 * useful
            ach = flops / (tot * 1e-3) / 1e12
            ach_useful = useful / (tot * 1e-3) / 1e12
            # HBM bytes: forward reads and writes one half spectrum, the
            # inverse reads S twice (S and Gy) and Gz once and writes three
            spec = n * n * (n // 2 + 1) * 8
            gbs = 8 * spec * R * reps / (tot * 1e-3) / 1e9
            v["y_tc"] = {"launches": cnt, "tensor": {"achieved": round(ach_useful, 1), "peak": tc_peak, "unit": "TFLOP/s",
                                                     "frac": round(ach_useful / tc_peak, 4), "peak_source": tc_kind,
                                                     "flops": "useful: the DFT-matrix products once",
                                                     "achieved_issued": round(ach, 1),
                                                     "frac_issued": round(ach / tc_peak, 4)},
                         "hbm": {"achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                                 "frac": round(gbs / hbm_peak, 4)}, "chunk": chunk}
        out[name] = v
        fs.release()
    out["tc_timeouts"] = B.lib().hf_tc_timeouts(0)
    if args.precision_oracle > 0:
        out["oracle_error"] = precision_oracle_error(ctx, hf, q[:args.precision_oracle], variants)
    del p1, p2
    return {"workload": f"256^3, 20000+20000 skeleton points (rings, segments, sheets; radii U(0.01,0.05)), "
                        f"{R} random rotations, E+F fields", "variants": out}


def tensor_peak():
    """(bf16 burst, bf16 sustained, which) from the measured peaks; FP16
    dense runs at the BF16 rate."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return m["bf16_tflops"], m["bf16_tflops_sustained"], "measured (bf16 sustained)"
    except (OSError, KeyError, ValueError):
        return 1800.0, 1400.0, "fallback (bf16 sustained)"


def precision_oracle_error(ctx, hf, q, variants, subset=400):
    """Per-field max-abs and relative-L2 error of each variant against the
    FP64 oracle on the rotations q: the parts are `subset`-point subsets of
    the 20000-point parts, splatted by the oracle (its plain O(P N^3) splat),
    the reference fields are the oracle's resample plus its library-DFT
    route (fields_lib, pocketfft in float64 on the host cores)."""
    import torch
    import oracle
    n = 256
    s1, s2 = synth.c4_pair(0)
    sel = np.random.default_rng(5).choice(len(s1.pts), subset, replace=False)
    t0 = time.perf_counter()
    r1 = oracle.splat(n, s1.pts[sel], s1.sigma[sel])
    r2 = oracle.splat(n, s2.pts[sel], s2.sigma[sel])
    t_splat = time.perf_counter() - t0
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    p1, p2 = ctx.part(cu(r1), hf.HF_STATIONARY), ctx.part(cu(r2), hf.HF_MOVING)
    r1f, r2f = r1.astype(np.float32).astype(np.float64), r2.astype(np.float32).astype(np.float64)
    K = len(q)
    sets = {}
    for name, fl in variants:
        fs = ctx.fieldset(n, K, hf.HF_E | hf.HF_F | fl)
        fs.compute(p1, p2, q)
        sets[name] = fs
    torch.cuda.synchronize()
    acc = {name: {"max_abs": np.zeros(4), "l2_num": np.zeros(4)} for name, _ in variants}
    ref_max, ref_l2 = np.zeros(4), np.zeros(4)
    t0 = time.perf_counter()
    for r in range(K):
        qq = q[r].astype(np.float64)
        qq /= np.linalg.norm(qq)
        Rm = oracle.quat_to_rot(qq).astype(np.float32).astype(np.float64)
        ref = np.stack(oracle.fields_lib(r1f, oracle.resample(r2f, Rm)))
        for f in range(4):
            ref_max[f] = max(ref_max[f], np.abs(ref[f]).max())
            ref_l2[f] += (ref[f] ** 2).sum()
        for name, fs in sets.items():
            for f in range(4):
                d = fs.get(r, f).cpu().numpy().astype(np.float64) - ref[f]
                acc[name]["max_abs"][f] = max(acc[name]["max_abs"][f], np.abs(d).max())
                acc[name]["l2_num"][f] += (d ** 2).sum()
    for fs in sets.values():
        fs.release()
    fields = ("E", "Fx", "Fy", "Fz")
    res = {"rotations": f"0..{K - 1}", "oracle_s": round(time.perf_counter() - t0, 1), "splat_s": round(t_splat, 1),
           "parts": f"{subset}-point subsets of the 20000-point parts, splatted by the oracle",
           "reference": "oracle resample + fields_lib (pocketfft float64), float32-rounded inputs"}
    for name in acc:
        res[name] = {fields[f]: {"max_abs_over_max": float(acc[name]["max_abs"][f] / ref_max[f]),
                                 "rel_l2": float(np.sqrt(acc[name]["l2_num"][f] / ref_l2[f]))} for f in range(4)}
    return res


# ------------------------------------------------- frequency-domain modes
def run_next_rows(args, local_rank):
    """The later rows on the c2 workload (128^3, 1024 rotations, E+F+T):
    rotation in the frequency domain (HF_SPECTRAL; tables padded os = 1 and 2)
    with its deviation from the spatial route; the analytic torque (HF_TA)
    against the least-squares one; single-pose queries from truncated
    spectra (|k~| <= K) at a 1 kHz-style random walk; and the mesh
    descriptor of a procedural peg and holed block."""
    import torch
    import paper_1711_05017_b300 as hf
    dev = torch.device("cuda", local_rank)
    n, R = 128, args.rotations
    s1, s2 = synth.c2_pair(0)
    ctx = hf.Context(local_rank)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)  # noqa: E731
    g1, g2 = ctx.density_build(n, cu(s1.pts), cu(s1.sigma)), ctx.density_build(n, cu(s2.pts), cu(s2.sigma))
    p1, p2 = ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING)
    ctx.autotune(n, args.tune_cache)
    q = rank_rotations(0, R)
    stream = torch.cuda.current_stream()
    out, ref = {}, None
    for name, fl, os_ in (("spatial", 0, 0), ("spectral_os1", hf.HF_SPECTRAL, 1), ("spectral_os2", hf.HF_SPECTRAL, 2)):
        if os_:
            p2.spectral(os_)
        fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T | fl)
        fs.compute(p1, p2, q)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            fs.compute(p1, p2, q)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 2
        f3 = np.stack([np.stack([fs.get(r, f).cpu().numpy().astype(np.float64) for f in range(4)]) for r in (0, 1)])
        if ref is None:
            ref = f3
        out[name] = {"value": round(R / (ms / 1e3), 1), "unit": UNIT, "ms_per_build": round(ms, 2),
                     "max_abs_dev_from_spatial_over_max": [
                         round(float(np.abs(f3[:, f] - ref[:, f]).max() / np.abs(ref[:, f]).max()), 6)
                         for f in range(4)]}
        fs.release()
    # analytic torque (HF_TA) against the least-squares differences (HF_T)
    p1.moments()
    ta = {}
    tref = None
    for name, fl in (("fd_least_squares", hf.HF_T), ("fd_least_squares_f64", hf.HF_T | hf.HF_TORQUE_F64),
                     ("fd_least_squares_compensated", hf.HF_T | hf.HF_TORQUE_C), ("analytic", hf.HF_TA)):
        fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | fl)
        fs.compute(p1, p2, q)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            fs.compute(p1, p2, q)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 2
        T = np.stack([fs.get(0, 4 + a).cpu().numpy().astype(np.float64) for a in range(3)])
        ta[name] = {"value": round(R / (ms / 1e3), 1), "unit": UNIT, "ms_per_build": round(ms, 2)}
        if tref is None:
            tref = T
        else:
            ta[name]["max_abs_dev_from_fd_over_max"] = [round(float(np.abs(T[a] - tref[a]).max() / np.abs(T[a]).max()), 8)
                                                        for a in range(3)]
        fs.release()
    out["torque"] = ta
    lp = {}
    tw, qw = synth.translation_walk(7, 2000), synth.quaternion_walk(8, 2000)
    for os_ in (1, 2):
        p2.spectral(os_)
        for K in (8, 16):
            lat = []
            for i in range(2000):
                a = time.perf_counter()
                hf.lowpass_query(p1, p2, tw[i], qw[i], K=K)
                lat.append((time.perf_counter() - a) * 1e6)
            lat = np.array(lat[100:])
            lp[f"os{os_}_K{K}"] = {"modes": (2 * K + 1) ** 3, "p50_us": round(float(np.percentile(lat, 50)), 1),
                                  "p99_us": round(float(np.percentile(lat, 99)), 1)}
    mesh = {}
    for seg in (32, 64):
        hole, peg = synth.peg_hole_pair(seg)
        ctx.density_mesh(n, *hole)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.density_mesh(n, *hole)
        ctx.density_mesh(n, *peg)
        torch.cuda.synchronize()
        mesh[f"segments_{seg}"] = {"triangles": int(len(hole[1]) + len(peg[1])), "grid": n,
                                   "seconds_both_parts": round(time.perf_counter() - t0, 3),
                                   "sigma": 0.5, "gamma_max": 0.05, "max_depth": 8}
    return {"workload": f"c2 peg-in-hole skeletons, 128^3, {R} rotations, E+F+T; procedural peg/hole meshes",
            "field_build": out, "lowpass_single_pose": lp, "mesh_descriptor": mesh,
            "cufft_comparison": run_cufft_comparison(ctx, p1, p2, g1, g2, n, dev)}


def _quat_to_rot(q):
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def run_cufft_comparison(ctx, p1, p2, g1, g2, n, dev, R=32, reps=5):
    """The E+F build of R rotations as cuFFT (torch.fft) would do it, timed
    beside this library's: resampled moving grids (made by the library's
    resample kernel, outside the timed region) -> batched R2C -> conjugate
    product with the stationary spectrum and the i pi k~ multipliers -> four
    C2R inverses.  A timing reference only: no cuFFT is on the library's path.
    The fields of both routes are compared first."""
    import torch
    import paper_1711_05017_b300 as hf
    q = rank_rotations(0, R)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F)
    fs.compute(p1, p2, q)
    grids = torch.stack([hf.resample(g2, _quat_to_rot(qq).astype(np.float32)) for qq in q])
    h3 = (2.0 / n) ** 3
    k = torch.fft.fftfreq(n, d=1.0 / n, device=dev)
    k[n // 2] = 0.0  # Nyquist multiplier 0
    kx = torch.fft.rfftfreq(n, d=1.0 / n, device=dev)
    kx[-1] = 0.0
    mult = [np.pi * kx.view(1, 1, 1, -1), np.pi * k.view(1, 1, -1, 1), np.pi * k.view(1, -1, 1, 1)]
    r1h = torch.fft.rfftn(g1)

    def cufft_build():
        S = r1h * torch.fft.rfftn(grids, dim=(1, 2, 3)).conj()
        E = torch.fft.irfftn(S, s=(n, n, n), dim=(1, 2, 3)) * h3
        F = [torch.fft.irfftn(S * (1j * m), s=(n, n, n), dim=(1, 2, 3)) * (-h3) for m in mult]
        return E, F

    E, F = cufft_build()
    dev_max = []
    for r in (0, R - 1):
        for f, a in enumerate([E[r], *[Fd[r] for Fd in F]]):
            b = fs.get(r, f)
            dev_max.append(round(float((a - b).abs().max() / b.abs().max()), 8))
    del E, F

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_cufft = timed(cufft_build)
    ms_ours = timed(lambda: fs.compute(p1, p2, q))
    return {"rotations": R, "grid": n, "cufft_ms_per_build": round(ms_cufft, 3),
            "cufft_rot_per_s": round(R / (ms_cufft / 1e3), 1), "ours_ms_per_build": round(ms_ours, 3),
            "ours_rot_per_s": round(R / (ms_ours / 1e3), 1), "speedup": round(ms_cufft / ms_ours, 2),
            "cufft_scope": "R2C + product + 4 C2R (resample excluded); ours: the whole E+F build",
            "max_abs_dev_over_max": dev_max}


# ------------------------------------------------------- serving workload
def run_serving(args, local_rank):
    """16 sessions (N from {64, 128, 256}), Poisson field-build requests
    (2/s per session, 64-512 rotations each, E+F+T), HBM budget 120 GB, a
    1 kHz pose-query random walk per session from native threads.  Requests
    whose set exceeds a third of the budget are built in rotation chunks
    admitted as memory frees.  Returns the summary dict."""
    import torch
    import paper_1711_05017_b300 as hf
    dev = torch.device("cuda", local_rank)
    sess = synth.c5_sessions(0, n_sessions=16, duration_s=args.serve_seconds)
    ctx = hf.Context(local_rank, hbm_budget_bytes=120 * (1 << 30))
    srv = hf.Server(ctx, max_inflight=4, query_lanes=16)
    sids, parts = [], []
    for s in sess:
        cu = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)  # noqa: E731
        g1 = ctx.density_build(s.n, cu(s.s1.pts), cu(s.s1.sigma))
        g2 = ctx.density_build(s.n, cu(s.s2.pts), cu(s.s2.sigma))
        p = (ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING))
        parts.append(p)
        sids.append(srv.open(*p))
    torch.cuda.synchronize()
    flags = hf.HF_E | hf.HF_F | hf.HF_T
    # warm-up: one 64-rotation build per session so that every session can answer queries
    first = [srv.submit(sid, synth.random_quaternions(900 + i, 64), flags) for i, sid in enumerate(sids)]
    srv.wait(first, timeout=600)
    for sid in sids:  # load the query kernels before the timed run (lazy module loading)
        try:
            srv.query(sid, [0.0, 0.0, 0.0], [1.0, 0.0, 0.0, 0.0])
        except hf.HFError:
            pass
    st0 = srv.stats()
    # arrivals merged over sessions
    events = sorted((t, i, int(r), int(qs))
                    for i, s in enumerate(sess) for t, r, qs in zip(s.arrivals, s.n_rot, s.quat_seeds))
    steps = int(args.serve_seconds * 1000)
    poses = np.stack([np.concatenate([synth.translation_walk(3000 + i, steps),
                                      synth.quaternion_walk(4000 + i, steps)], axis=1)
                      for i in range(len(sids))])
    drive = {}

    def driver():  # native threads, one per session, 1 kHz each (the call releases the GIL)
        drive["res"] = srv.drive_queries(sids, poses, rate_hz=1000.0, k=4)

    th = [threading.Thread(target=driver, daemon=True)]
    srv.query_latencies()  # drop the warm-up's
    srv.trace(0)
    srv.trace(1)
    cg0 = _cgroup_cpu_stat()
    t_start = time.perf_counter()
    for t in th:
        t.start()
    rids, rej = [], 0
    for t_ev, i, R, qs in events:
        wait = t_start + t_ev - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        try:
            rids.append((srv.submit(sids[i], synth.random_quaternions(qs, R), flags), sess[i].n, R))
        except hf.HFError:
            rej += 1
    for t in th:
        t.join()
    elapsed = time.perf_counter() - t_start
    st1 = srv.stats()
    lib_lat = srv.query_latencies()
    slow_q, slow_c = srv.trace(0), srv.trace(1)
    res = srv.wait([r[0] for r in rids], timeout=900)
    build_lat = [v[1] for v in res.values() if v[0] == "done"]
    chunked = [srv.request_chunks(r, R)[0] for r, _, R in rids if res[r][0] == "done"]
    st2 = srv.stats()
    answered, not_ready, late = drive["res"]
    lat = lib_lat if lib_lat.size else np.array([np.nan])

    def pct(a, p):
        return round(float(np.percentile(a, p)), 1)

    # the slowest queries, with what the scheduler was doing when they ran
    worst = []
    for row in slow_q[np.argsort(-slow_q[:, 1])[:5]] if len(slow_q) else []:
        t0q, us = row[0], row[1]
        over = [{"kind": ("create", "compute", "release")[int(c[2])], "start_ms": round(c[0], 2),
                 "us": round(c[1], 1)} for c in slow_c if c[0] <= t0q + us / 1e3 and c[0] + c[1] / 1e3 >= t0q]
        worst.append({"start_ms": round(t0q, 2), "us": round(us, 1), "mutex_us": round(row[2], 1),
                      "lane_wait_us": round(row[3], 1), "launch_us": round(row[4], 1), "sync_us": round(row[5], 1),
                      "session_n": sess[int(row[6])].n, "involuntary_csw": int(row[7]),
                      "voluntary_csw": int(row[8]), "overlapping_scheduler_calls": over[:4]})
    per_n = {}
    for sid, s in zip(sids, sess):
        a, nr = srv.session_counts(sid)
        d = per_n.setdefault(str(s.n), {"sessions": 0, "answered": 0, "not_ready": 0})
        d["sessions"] += 1
        d["answered"] += a
        d["not_ready"] += nr
    out = {
        "sessions": len(sids), "grid_sizes": sorted(set(s.n for s in sess)), "seconds": round(elapsed, 2),
        "queries_by_grid": per_n,
        "budget_gb": 120, "chunk_limit_gb": round(st2["chunk_bytes"] / (1 << 30), 1),
        "query_us": {"p50": pct(lat, 50), "p99": pct(lat, 99), "p99.9": pct(lat, 99.9),
                     "max": round(float(np.max(lat)), 1), "n": int(lat.size),
                     "over_1ms": int((lat > 1000).sum()),
                     "answered": int(answered), "not_ready": int(not_ready),
                     "started_late": int(late), "rate_hz_per_session": 1000,
                     "budget_us": 1000, "measured": "inside hf_server_query (entry to return)"},
        "builds": {"submitted": int(st2["submitted"] - st0["submitted"]), "completed": len(build_lat),
                   "rejected_at_submit": rej,
                   "superseded": int(st2["superseded"] - st0["superseded"]),
                   "failed": int(st2["failed"] - st0["failed"]),
                   "chunked": int(sum(c > 1 for c in chunked)),
                   "chunks_built": int(st2["chunks_completed"] - st0["chunks_completed"]),
                   "evicted_chunks": int(st2["evicted"] - st0["evicted"]),
                   "rotations_per_request": "U-integer[64, 512] at every N",
                   "latency_ms_p50": pct(build_lat, 50) if build_lat else None,
                   "latency_ms_p99": pct(build_lat, 99) if build_lat else None},
        "fields_per_s": round((st1["rotations_completed"] - st0["rotations_completed"]) / elapsed, 1),
        "memory_pool_gb": {"reserved_at_start": round(st0["pool_reserved_bytes"] / 2**30, 2),
                           "reserved_at_end": round(st1["pool_reserved_bytes"] / 2**30, 2),
                           "reserved_high": round(st1["pool_reserved_high"] / 2**30, 2)},
        "field_set_arena": {"gb": round(st1["arena_bytes"] / 2**30, 2),
                            "free_gb_at_end": round(st1["arena_free_bytes"] / 2**30, 2),
                            "largest_free_gb_at_end": round(st1["arena_largest_free"] / 2**30, 2),
                            "refusals": int(st2["arena_refusals"] - st0["arena_refusals"])},
        "hardware_queues": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8 (the default)"),
        "slowest_queries": worst,
        "slow_scheduler_calls": {"n": int(len(slow_c)),
                                 "max_us": round(float(slow_c[:, 1].max()), 1) if len(slow_c) else 0.0,
                                 "by_kind": {name: {"n": int((slow_c[:, 2] == k).sum()),
                                                    "max_us": round(float(slow_c[slow_c[:, 2] == k, 1].max()), 1),
                                                    "p50_us": round(float(np.median(slow_c[slow_c[:, 2] == k, 1])), 1)}
                                             for k, name in enumerate(("create", "compute", "release"))
                                             if len(slow_c) and (slow_c[:, 2] == k).any()}},
    }
    if len(slow_q):
        inv = slow_q[:, 7] > 0
        over = slow_q[:, 1] > 1000
        out["slow_query_causes"] = {
            "n_over_500us": int(len(slow_q)), "n_over_1ms": int(over.sum()),
            "with_involuntary_csw": int(inv.sum()), "over_1ms_with_involuntary_csw": int((inv & over).sum()),
            "launch_us_p50": round(float(np.median(slow_q[:, 4])), 1),
            "sync_us_p50": round(float(np.median(slow_q[:, 5])), 1),
            "over_1ms_launch_us_max": round(float(slow_q[over, 4].max()), 1) if over.any() else None,
            "over_1ms_sync_us_max": round(float(slow_q[over, 5].max()), 1) if over.any() else None}
    out["host_cpu"] = {"cpus_usable": len(os.sched_getaffinity(0)), "cgroup_cpu": _cgroup_cpu(cg0)}
    srv.close()
    del parts
    return out


def _cgroup_cpu_stat():
    """The process's cgroup CPU quota and throttling counters (cgroup v2 or
    v1), or None where neither is readable."""
    for stat, quota in (("/sys/fs/cgroup/cpu.stat", "/sys/fs/cgroup/cpu.max"),
                        ("/sys/fs/cgroup/cpu/cpu.stat", "/sys/fs/cgroup/cpu/cpu.cfs_quota_us")):
        try:
            with open(stat) as f:
                d = {k: int(v) for k, v in (ln.split() for ln in f if len(ln.split()) == 2)}
            with open(quota) as f:
                d["quota"] = f.read().strip()
            return d
        except (OSError, ValueError):
            continue
    return None


def _cgroup_cpu(before):
    """Throttling during the serving run: the counters' change since `before`."""
    after = _cgroup_cpu_stat()
    if not before or not after:
        return None
    keys = ("nr_periods", "nr_throttled", "throttled_usec", "throttled_time")
    return {"quota": after.get("quota"), **{k: after[k] - before[k] for k in keys if k in after and k in before}}


# ------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle (FP64, own FFT, OpenMP) on the host cores, same metric."""
    if rank != 0:
        return
    import oracle
    n = args.n
    s1, s2 = synth.c2_pair(0)
    q = synth.random_quaternions(0, max(1, args.steps + args.warmup))
    r1 = oracle.splat(n, s1.pts, s1.sigma)
    r2 = oracle.splat(n, s2.pts, s2.sigma)
    for i in range(args.warmup):
        oracle.fields(r1, oracle.resample(r2, oracle.quat_to_rot(q[i])))
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.fields(r1, oracle.resample(r2, oracle.quat_to_rot(q[args.warmup + i])))
    s = (time.perf_counter() - t0) / max(1, args.steps)
    v = 1.0 / s
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(s * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"c2 peg-in-hole skeletons, {n}^3 grid, one rotation per step (bounded sample "
                                   f"of the {N_ROT}-rotation batch), E+F fields", "grid": n},
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "one rotation per step: resample + energy/force by the oracle's own FFT"},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_spectral_only(args, local_rank):
    """Spectral (os 1) field builds of the c2 workload alone: a small, self-
    contained run of the frequency-domain route for kernel profiles."""
    import torch
    import paper_1711_05017_b300 as hf
    from paper_1711_05017_b300 import build

    build.build()
    torch.cuda.set_device(local_rank)
    n, R = args.n, args.spectral_only
    dev = torch.device("cuda", local_rank)
    s1, s2 = synth.c2_pair(0)
    ctx = hf.Context(local_rank)
    f32 = dict(dtype=torch.float32, device=dev)
    g1 = ctx.density_build(n, torch.as_tensor(s1.pts, **f32), torch.as_tensor(s1.sigma, **f32))
    g2 = ctx.density_build(n, torch.as_tensor(s2.pts, **f32), torch.as_tensor(s2.sigma, **f32))
    p1, p2 = ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING)
    p2.spectral(1)
    q = synth.random_quaternions(0, R).astype(np.float32)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_SPECTRAL)
    for _ in range(args.warmup):
        fs.compute(p1, p2, q)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        fs.compute(p1, p2, q)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    print(json.dumps({"metric": "spectral (os 1) E+F field build", "value": round(R / (ms / 1e3), 1),
                      "unit": "rotations/s", "rotations": R, "grid": n, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_build": round(ms, 3)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--rotations", type=int, default=N_ROT)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-rotations", type=int, default=16, help="rotations of the oracle CPU baseline")
    ap.add_argument("--no-tune", action="store_true", help="built-in launch shapes instead of the autotuner's")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file (read if it has this device and N)")
    ap.add_argument("--queue-chunk", type=int, default=32, help="rotations per work unit of the one-launch batch")
    ap.add_argument("--batch-steps", type=int, default=5,
                    help="graph launches of the 64-pair uneven batch (0 = skip)")
    ap.add_argument("--precision-rotations", type=int, default=512,
                    help="rotations of the 256^3 precision comparison (0 = skip)")
    ap.add_argument("--precision-oracle", type=int, default=16,
                    help="rotations (0..K-1) of the precision comparison checked against the FP64 oracle (0 = skip)")
    ap.add_argument("--spectral", type=int, default=1,
                    help="measure the later rows: frequency-domain modes, analytic torque, mesh descriptor (0 = skip)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the 16-session serving run (0 = skip)")
    ap.add_argument("--spectral-only", type=int, default=0, metavar="R",
                    help="profiling aid: only R-rotation spectral (os 1) field builds of the c2 workload, "
                         "warm-up plus --steps timed, one JSON line")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.spectral_only > 0:
        run_spectral_only(args, local_rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

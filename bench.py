"""Throughput of the ptychographic reconstruction hot path on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default): LSQML on a 256 x 256 detector, 10,000 scan positions
(100 x 100 raster, step 24 px, +-2 px seeded jitter), 2640 x 2640 object,
one probe mode, FP32 intensities with Poisson noise at 1e5 photons/frame.
A step is one iteration over all positions (the whole hot path: Fourier
step, object and probe overlap sums, LSQML step sizes, updates).  DM on the
same scan and the 16-bit intensity stores are reported beside it.

value   : patterns*iterations/s with all inputs resident in HBM;
e2e     : the same metric for a whole job through the C ABI from pinned host
          buffers (set_data + set_init + n iterations + get_object/get_probe);
roofline: the dominant kernel's algorithmic HBM bytes per launch over its
          CUDA-event duration, against the measured copy bandwidth;
cpu_baseline: the FP64 oracle on a bounded sub-scan of the same workload.

Under torchrun (N > 1) every rank reconstructs its own scan of the same shape
(independent replicas, weak scaling; no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "patterns·iter/s (DM/LSQML, 256² det, 10k pos) and time-to-ε vs plain FP32, 1 B300"
UNIT = "patterns*iter/s"
WORKLOAD = dict(M=256, K=1, grid=100, step=24, jitter=2, obj=2640, photons=1e5)
SUBPIXEL = 8   # 1/8-pixel position quantisation of the sub-pixel variants


def workload_desc(w=WORKLOAD):
    return (f"LSQML, {w['M']}x{w['M']} detector, {w['grid'] ** 2} positions ({w['grid']}x{w['grid']} raster, "
            f"step {w['step']} px, +-{w['jitter']} px jitter), {w['obj']}x{w['obj']} object, K={w['K']}, "
            f"Poisson {w['photons']:.0e} photons/frame")


def bench_config(world, w=WORKLOAD):
    """The workload both arms report (the reference arm times bounded
    samples of it, described in its cpu_baseline)."""
    M, K, J = w["M"], w["K"], w["grid"] ** 2
    return {"workload": workload_desc(w), "algorithm": "lsqml", "M": M, "K": K, "J": J,
            "object": [w["obj"], w["obj"]], "intensity_store": "f32",
            "l2": f"inputs larger than L2: {J * K * M * M * 8 / 1e9:.2g} GB of residuals and "
                  f"{J * M * M * 4 / 1e9:.2g} GB of amplitudes per iteration",
            "replicas": world}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def make_scan(seed, w=WORKLOAD):
    from paper_2202_03144_b300 import synth
    M, K = w["M"], w["K"]
    P = synth.make_probe(M, K, R=80.0, sigma=16.0, c=0.00125)
    pos = synth.raster_positions(w["grid"], w["grid"], w["step"], w["jitter"], w["jitter"], seed=2000 + seed)
    O = synth.make_object(w["obj"], w["obj"], seed=1000 + seed)
    P0 = synth.make_probe(M, K, R=88.0, sigma=16.0, c=0.00125)
    return P, O, pos, P0


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, dev):
        self.path = tempfile.mktemp(suffix=".csv")
        self.p = None
        if shutil.which("nvidia-smi"):
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # the timed region is short: let the sampler start before it begins
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.p.poll() is None:
                if os.path.exists(self.path) and os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.01)

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _block(P, O, pos, w, r0, c0, sub):
    """The sub x sub block of the raster with its first position at raster
    row r0, column c0, shifted to a cut of the object that holds it."""
    g = w["grid"]
    idx = np.array([(r0 + r) * g + (c0 + c) for r in range(sub) for c in range(sub)])
    pos_s = pos[idx]
    y0 = int(np.rint(pos_s[:, 0]).min())
    x0 = int(np.rint(pos_s[:, 1]).min())
    pos_s = pos_s - [y0, x0]
    ny = int(np.rint(pos_s[:, 0]).max()) + w["M"]
    nx = int(np.rint(pos_s[:, 1]).max()) + w["M"]
    return O[y0:y0 + ny, x0:x0 + nx].copy(), pos_s


def _oracle_worker(P, O_s, pos_s, P0, photons, steps, barrier, q):
    """One host core: the block's intensities from the oracle's forward
    model (not timed), then `steps` timed LSQML iterations of the unchanged
    FP64 oracle, each started together with the other workers."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    from oracle import ptycho_oracle as orc
    I_s = oracle_intensities(P, O_s, pos_s, photons, 5)
    O0 = np.ones(O_s.shape, complex)
    out = []
    for _ in range(steps):
        barrier.wait()
        t = time.perf_counter()
        orc.reconstruct("lsqml", O0, P0, pos_s, I_s, 1)
        out.append(time.perf_counter() - t)
    q.put(out)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_parallel(P, O, pos, P0, w=WORKLOAD, sub=12, steps=1, max_workers=64):
    """The FP64 oracle on the host's cores: one worker process per core
    (started with spawn: the parent may already hold a CUDA context), each
    on its own sub x sub block of the raster, the blocks' iterations started
    together.  Returns per step (positions, wall seconds = the slowest
    worker), the worker count and the host's core count."""
    import multiprocessing as mp
    cores = host_cores()
    nb = w["grid"] // sub
    n = max(1, min(cores, max_workers, nb * nb))
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(n), ctx.Queue()
    procs = []
    for i in range(n):
        O_s, pos_s = _block(P, O, pos, w, (i // nb) * sub, (i % nb) * sub, sub)
        p = ctx.Process(target=_oracle_worker, args=(P, O_s, pos_s, P0, w["photons"], steps, barrier, q))
        p.start()
        procs.append(p)
    res = [q.get() for _ in procs]
    for p in procs:
        p.join()
    per_step = [(n * sub * sub, max(r[s] for r in res)) for s in range(steps)]
    return per_step, n, cores


def cpu_baseline(P, O, pos, P0, w=WORKLOAD, sub=12):
    """FP64 oracle, one LSQML iteration per host core, each on its own block."""
    per_step, n, cores = oracle_parallel(P, O, pos, P0, w, sub=sub, steps=1)
    units, dt = per_step[0]
    return {"value": units / dt, "unit": UNIT, "cores": n, "kind": "oracle", "host_cores": cores,
            "sample": f"1 LSQML iteration of the FP64 numpy oracle on each of {n} {sub}x{sub}-position blocks of "
                      f"the raster ({units} positions, same M, probe and step), one process per core, all started "
                      f"together; {dt:.1f} s for the slowest block"}


def oracle_intensities(P, O, pos, photons, seed):
    from oracle import ptycho_oracle as orc
    from paper_2202_03144_b300 import synth
    I = orc.far_field_intensity(O, P, orc.round_positions(pos))
    I = I * photons / I.sum(axis=(1, 2)).mean()
    return synth.poisson(I, seed)


def rank_env():
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(dist, value, device="cuda"):
    """The largest of every rank's value (the job ends when the slowest rank
    does); the value itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, seconds):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / seconds


def run_reference(args):
    """Reference arm: the FP64 oracle, as it stands, on bounded samples of the
    workload, one process per host core."""
    _, rank, _ = rank_env()
    if rank != 0:
        return
    P, O, pos, P0 = make_scan(0)
    sub = 12
    per_step, n, cores = oracle_parallel(P, O, pos, P0, sub=sub, steps=args.warmup + args.steps)
    timed = per_step[args.warmup:]
    vals = [u / dt for u, dt in timed]
    v = statistics.median(vals)
    units = timed[0][0]
    ms = units / v * 1e3
    sample = (f"per step, 1 LSQML iteration of the FP64 numpy oracle on each of {n} {sub}x{sub}-position blocks "
              f"({units} positions), one process per host core, all started together")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": bench_config(args.gpus),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": n, "host_cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(api, torch, stream, n=64, iters=4, warm=2, seed=7, group_bytes=None):
    """Batched workload: n scans of unequal probe size and position count,
    one CUDA graph per iteration (members in L2-sized groups) vs every member
    at once and vs one member at a time."""
    from paper_2202_03144_b300 import synth
    members = synth.batch_members(n, seed=seed)
    side = max(max(m["obj_shape"]) for m in members)
    field = synth.make_object(side, side, seed=4242)
    probes = {}
    for M in sorted(set(m["M"] for m in members)):
        probes[M] = (synth.make_probe(M, 1, R=0.3125 * M, sigma=M / 16.0, c=0.02 * (64.0 / M) ** 2),
                     synth.make_probe(M, 1, R=0.34375 * M, sigma=M / 16.0, c=0.02 * (64.0 / M) ** 2))
    # cluster size and transform engine per M from the autotuners
    spec = [dict(M=m["M"], K=1, J=m["J"], obj_shape=m["obj_shape"], cluster=-1, fft_engine="auto") for m in members]
    gen = torch.Generator(device="cuda").manual_seed(99)
    with torch.cuda.stream(stream):
        b = api.Batch(spec, stream=stream.cuda_stream, group_bytes=group_bytes)
        for mem, m in zip(b.members, members):
            P, P0 = probes[m["M"]]
            O = field[:m["obj_shape"][0], :m["obj_shape"][1]]
            mem.set_positions(m["positions"])
            mem.set_init(O, P)
            I = torch.empty((m["J"], m["M"], m["M"]), dtype=torch.float32, device="cuda")
            mem.simulate(I)
            torch.cuda.synchronize()
            sc = m["photons"] / float(I.sum(dim=(1, 2)).mean())
            I = torch.poisson(I * sc, generator=gen)
            mem.set_data(I, m["positions"])
            mem.set_init(np.ones(m["obj_shape"], np.complex64), P0 * np.sqrt(sc))
            del I
        torch.cuda.synchronize()
        b.iterate("lsqml", warm)
        torch.cuda.synchronize()
        if group_bytes is None:  # the schedule (group budget or lanes) from the batch autotuner
            tuned_bytes, tuned_lanes, _ = b.autotune("lsqml", 1)
        else:
            tuned_bytes, tuned_lanes = group_bytes, 0
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.iterate("lsqml", iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_graph = e0.elapsed_time(e1)
        n_groups = max(b.groups()) + 1
        # every member at once (one group)
        b.set_group_bytes(0)
        b.iterate("lsqml", 1)
        e0.record(stream)
        b.iterate("lsqml", iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_all = e0.elapsed_time(e1)
        # one member after another (a job queue on one GPU)
        t0 = time.perf_counter()
        for mem in b.members:
            mem.iterate("lsqml", iters)
            mem.get_probe()  # synchronises the member
        ms_seq = (time.perf_counter() - t0) * 1e3
        kpi = b.kernels_per_iteration
        clusters = sorted({(m["M"], api.autotune(m["M"], 1)[0]) for m in members})
        engines = sorted({(m["M"], api.autotune_engine(m["M"], 1)[0]) for m in members})
        b.close()
    units = sum(m["J"] for m in members) * iters
    gb_mib = tuned_bytes / 2**20
    return {"value": units / (ms_graph / 1e3), "unit": UNIT, "groups": n_groups,
            "all_at_once_value": units / (ms_all / 1e3), "sequential_value": units / (ms_seq / 1e3),
            "members": n, "positions": sum(m["J"] for m in members), "iterations": iters,
            "kernels_per_graph": kpi, "autotuned_clusters": clusters, "autotuned_engines": engines,
            "autotuned_group_mib": gb_mib, "autotuned_lanes": tuned_lanes,
            "workload": f"{n} LSQML scans, probe sizes {{64,96,128,192,256}}, 100-4000 positions (Fermat "
                        "spirals, spacing 0.15 M), Poisson 1e4-1e6 photons/frame; one CUDA graph per iteration, "
                        + (f"members in {tuned_lanes} chains run side by side" if tuned_lanes else
                           f"members run in groups of at most {gb_mib:g} MiB working set")}


def time_to_eps(api, torch, stream, I, pos, P0s, w, n_ref=30, check=5):
    """Wall time and iterations for 16-bit amplitude storage to reach the
    Fourier error that plain FP32 LSQML reaches after n_ref iterations.  Every
    run is scored by the same FP32-stored context (its (O, P) copied over at
    each check), so the error is always measured against the FP32 data."""
    M, K, J = w["M"], w["K"], w["grid"] ** 2
    shape = (w["obj"], w["obj"])
    out = {}
    eps = None
    with torch.cuda.stream(stream):
        scorer = api.Reconstruction(M, K, J, shape, stream=stream.cuda_stream)
        scorer.set_data(I, pos)
        Ob = torch.empty(shape, dtype=torch.complex64, device="cuda")
        Pb = torch.empty((K, M, M), dtype=torch.complex64, device="cuda")
        runs = [("f32", {}), ("f16", dict(istore="f16")), ("bf16", dict(istore="bf16")),
                ("f32_residual16", dict(residual_store="f16")),
                ("f16_residual16", dict(istore="f16", residual_store="f16"))]
        for store, kw in runs:
            r = api.Reconstruction(M, K, J, shape, stream=stream.cuda_stream, **kw)
            r.set_data(I, pos)
            r.set_init(np.ones(shape, np.complex64), P0s)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, E = 0, None
            limit = n_ref if store == "f32" else 2 * n_ref
            while it < limit:
                r.iterate("lsqml", check)
                it += check
                r.get_object(Ob)
                r.get_probe(Pb)
                scorer.set_init(Ob, Pb)
                E = scorer.fourier_error()
                if eps is not None and E <= eps:
                    break
            dt = time.perf_counter() - t0
            r.close()
            if store == "f32":
                eps = E
            out[store] = {"iterations": it, "seconds": dt, "fourier_error": E, "reached": bool(E <= eps)}
        scorer.close()
    return {"eps": eps, "reference": f"plain FP32 LSQML after {n_ref} iterations from a flat object; errors "
                                     "measured against the FP32 data", "check_every": check,
            "variants": "amplitude storage f32 / f16 / bf16; *_residual16: LSQML residuals stored as FP16",
            **out}


def run_epie(api, torch, stream, iters=3, warm=1, subpixel=0):
    """ePIE (sequential by definition) on the 3-mode 128^2 spiral scan:
    positions*iterations/s of the persistent single-cluster sweep (on the
    widest compiled cluster: its latency per position bounds the sweep).
    subpixel = S: the same scan at fractional positions, 1/S-pixel shifts
    (one position at a time through the general kernels)."""
    from paper_2202_03144_b300 import synth
    d = synth.scan_config("modes128", seed=5)
    M, K, pos = d["M"], d["K"], d["positions"]
    if subpixel:
        pos = synth.fractional_positions(pos, seed=2005)
    shape = d["object"].shape
    with torch.cuda.stream(stream):
        r = api.Reconstruction(M, K, len(pos), shape, stream=stream.cuda_stream, seed=1, subpixel=subpixel)
        r.set_positions(pos)
        r.set_init(d["object"], d["probe"])
        I = torch.empty((len(pos), M, M), dtype=torch.float32, device="cuda")
        r.simulate(I)
        torch.cuda.synchronize()
        sc = d["photons"] / float(I.sum(dim=(1, 2)).mean())
        I = torch.poisson(I * sc, generator=torch.Generator(device="cuda").manual_seed(21))
        P0 = d["probe0"] * np.sqrt(float(I.sum(dim=(1, 2)).mean()) / (M * M) / np.sum(np.abs(d["probe0"]) ** 2))
        r.set_data(I, pos)
        r.set_init(d["object0"], P0)
        r.iterate("epie", warm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.iterate("epie", iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        cl = r.epie_cluster
        E = r.fourier_error()
        r.close()
    out = {"value": len(pos) * iters / (ms / 1e3), "unit": UNIT, "ms_per_iteration": ms / iters,
           "cluster": cl, "fourier_error": E,
           "workload": "ePIE, 1600-position Fermat spiral, 3-mode 128^2 probe, 1088^2 object, Poisson 1e5"}
    if subpixel:
        out["workload"] += f", fractional positions at 1/{subpixel} px"
    return out


def run_engines(api, torch, stream, grid=100, iters=5, warm=2):
    """The Fourier-pass engines on the 64^2 detector (the tensor-core DFT is
    compiled there): LSQML and DM on a 100 x 100 raster (step 6 px, +-2 px
    jitter, 10,000 positions), per-iteration time and the Fourier pass's
    CUDA-event time, FP32 FFT against the BF16 three-term tensor-core DFT."""
    from paper_2202_03144_b300 import synth
    M, K, J = 64, 1, grid * grid
    step = 6
    side = -(-(step * (grid - 1) + M + 8) // 16) * 16
    P = synth.make_probe(M, K, R=20.0, sigma=4.0, c=0.02)
    P0 = synth.make_probe(M, K, R=22.0, sigma=4.0, c=0.02)
    pos = synth.raster_positions(grid, grid, step, 2, 2, seed=2100)
    O = synth.make_object(side, side, seed=1100)
    out = {"workload": f"64x64 detector, {J} positions ({grid}x{grid} raster, step {step} px, +-2 px jitter), "
                       f"{side}x{side} object, K=1, Poisson 1e5 photons/frame"}
    with torch.cuda.stream(stream):
        sim = api.Reconstruction(M, K, J, (side, side), stream=stream.cuda_stream)
        sim.set_positions(pos)
        sim.set_init(O, P)
        I = torch.empty((J, M, M), dtype=torch.float32, device="cuda")
        sim.simulate(I)
        torch.cuda.synchronize()
        sim.close()
        sc = 1e5 / float(I.sum(dim=(1, 2)).mean())
        I = torch.poisson(I * sc, generator=torch.Generator(device="cuda").manual_seed(5))
        for eng in ("register", "tensor_bf16x3"):
            res = {}
            for alg, fam in (("lsqml", "fourier_chi"), ("dm", "fourier_dm")):
                r = api.Reconstruction(M, K, J, (side, side), stream=stream.cuda_stream, fft_engine=eng)
                r.set_data(I, pos)
                r.set_init(np.ones((side, side), np.complex64), P0 * np.sqrt(sc))
                r.iterate(alg, warm)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r.iterate(alg, iters)
                e1.record(stream)
                torch.cuda.synchronize()
                r.set_profiling(True)
                r.iterate(alg, 2)
                prof = r.get_profile()
                res[alg] = {"ms_per_iteration": e0.elapsed_time(e1) / iters,
                            "fourier_pass_ms": prof[fam]["ms"] / prof[fam]["launches"],
                            "fourier_error": r.fourier_error()}
                r.close()
            out[eng] = res
    return out


def run_training(api, torch, n_frames, batch=64):
    """Warm-start network training speed alone: n_frames simulated frames,
    one epoch at the given batch after a four-batch warm-up."""
    from paper_2202_03144_b300 import warmstart
    frames, targets, _ = warmstart.make_training_set(n_frames, seed=3, per_object=min(25000, n_frames))
    net = api.Net(seed=11, max_batch=256)
    warmstart.train(net, frames[:batch * 4], targets[:batch * 4], epochs=1, batch=batch)
    torch.cuda.synchronize()
    # the loss is read back (a host sync) only at the first and the last step
    losses, t = warmstart.train(net, frames, targets, epochs=1, batch=batch, lr=1e-3, log_every=1 << 30)
    net.close()
    return {"frames": n_frames, "batch": batch, "seconds": t, "frames_per_s": n_frames / t,
            "loss_first": losses[0][1], "loss_last": losses[-1][1]}


def run_warm_start(api, torch, stream, n_frames=200_000, epochs=1, n_ref=50, check=5):
    """Learned warm start on a 1600-position, 3-mode 128^2 scan: network
    training (one-off, reported apart), then iterations and wall time to the
    Fourier error the plain FP32 LSQML reaches from a flat object after n_ref
    iterations, for: flat start; warm start; warm start with FP16 storage."""
    from paper_2202_03144_b300 import synth, warmstart
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    frames, targets, _ = warmstart.make_training_set(n_frames, seed=3, per_object=25000)
    t_data = time.perf_counter() - t0
    net = api.Net(seed=11, max_batch=256)  # training uses batches of 64; inference up to 256
    losses, t_train = warmstart.train(net, frames, targets, epochs=epochs, batch=64, lr=1e-3, log_every=500)
    del frames, targets
    d = synth.scan_config("modes128", seed=5)
    M, K, pos = d["M"], d["K"], d["positions"]
    shape = d["object"].shape
    with torch.cuda.stream(stream):
        sim = api.Reconstruction(M, K, len(pos), shape, stream=stream.cuda_stream)
        sim.set_positions(pos)
        sim.set_init(d["object"], d["probe"])
        I = torch.empty((len(pos), M, M), dtype=torch.float32, device="cuda")
        sim.simulate(I)
        torch.cuda.synchronize()
        sim.close()
        sc = d["photons"] / float(I.sum(dim=(1, 2)).mean())
        I = torch.poisson(I * sc, generator=torch.Generator(device="cuda").manual_seed(17))
    P0 = d["probe0"] * np.sqrt(float(I.sum(dim=(1, 2)).mean()) / (M * M) / np.sum(np.abs(d["probe0"]) ** 2))
    scan = dict(M=M, K=K, positions=pos, object0=d["object0"], probe0=P0)
    res = warmstart.compare(net, scan, I, alg="lsqml", n_ref=n_ref, check=check, stream=stream.cuda_stream)
    # warm start + 16-bit amplitude storage, scored on the FP32 data
    with torch.cuda.stream(stream):
        scorer = api.Reconstruction(M, K, len(pos), shape, stream=stream.cuda_stream)
        scorer.set_data(I, pos)
        r = api.Reconstruction(M, K, len(pos), shape, stream=stream.cuda_stream, istore="f16")
        r.set_data(I, pos)
        r.set_init(scan["object0"], scan["probe0"])
        Ob = torch.empty(shape, dtype=torch.complex64, device="cuda")
        Pb = torch.empty((K, M, M), dtype=torch.complex64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.warm_start(r, net)
        it, E = 0, None
        while it < 2 * n_ref:
            r.iterate("lsqml", check)
            it += check
            r.get_object(Ob)
            r.get_probe(Pb)
            scorer.set_init(Ob, Pb)
            E = scorer.fourier_error()
            if E <= res["eps"]:
                break
        res["warm_f16"] = {"iterations": it, "seconds": time.perf_counter() - t0, "final_error": E,
                           "reached": bool(E <= res["eps"])}
        r.close()
        scorer.close()
    net.close()
    res["training"] = {"frames": n_frames, "epochs": epochs, "seconds": t_train, "data_seconds": t_data,
                       "frames_per_s": n_frames * epochs / t_train, "loss_first": losses[0][1],
                       "loss_last": losses[-1][1], "parameters": 1964690}
    res["workload"] = ("LSQML on 1600 Fermat-spiral positions (20 px mean spacing), 3-mode 128^2 probe, 1088^2 "
                       "object, Poisson 1e5; net trained on frames simulated from other seeded objects")
    # the one-off training spread over a number of scans of this kind; the
    # test objects come from the training generator (an in-distribution gain)
    saved = res["flat"]["seconds"] - res["warm"]["seconds"]
    n_scans = 100
    res["amortised"] = {"scans": n_scans, "training_seconds_per_scan": t_train / n_scans,
                        "warm_seconds_per_scan_with_training": res["warm"]["seconds"] + t_train / n_scans,
                        "flat_seconds_per_scan": res["flat"]["seconds"],
                        "break_even_scans": (t_train / saved) if saved > 0 else None,
                        "distribution": "in-distribution: test objects from the training generator"}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-iters", type=int, default=20)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--small", action="store_true", help="a 20x20-position scan (profiling runs)")
    ap.add_argument("--grid", type=int, default=0, help="raster side (positions = grid^2; profiling runs)")
    ap.add_argument("--cluster", type=int, default=0, help="FFT cluster size (0 = library default)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-eps", action="store_true", help="skip the time-to-epsilon runs")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm start")
    ap.add_argument("--warm-frames", type=int, default=200_000)
    ap.add_argument("--epie-only", action="store_true",
                    help="run only the ePIE sweeps of the 3-mode spiral scan, whole-pixel and sub-pixel (profiling runs)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the 64-scan batched workload and print its figures (profiling runs)")
    ap.add_argument("--engines-only", action="store_true",
                    help="run only the 64^2 Fourier-engine comparison on a --grid (default 100) raster (profiling runs)")
    ap.add_argument("--residual-store", default="f32", choices=["f32", "f16"],
                    help="LSQML residual storage of the headline and profile runs (profiling runs; --grid or --small)")
    ap.add_argument("--train-only", type=int, default=0, metavar="FRAMES",
                    help="only train the warm-start network on FRAMES frames at batch 64 (profiling runs)")
    args = ap.parse_args()
    if args.small:
        WORKLOAD["grid"] = 20
        WORKLOAD["obj"] = 736
    if args.grid:
        # corners reach 24 (grid - 1) + 4; plus the 256^2 window, rounded up to 16
        WORKLOAD["grid"] = args.grid
        WORKLOAD["obj"] = -(-(24 * args.grid + 236) // 16) * 16
    if args.impl == "reference":
        return run_reference(args)
    if args.residual_store != "f32" and not (args.small or args.grid):
        ap.error("--residual-store is for profiling runs (--grid or --small): the headline stores FP32 residuals")

    import torch
    from paper_2202_03144_b300 import api, synth

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if args.epie_only:
        stream = torch.cuda.Stream()
        ep = run_epie(api, torch, stream)
        ep["subpixel"] = run_epie(api, torch, stream, subpixel=SUBPIXEL)
        print(json.dumps(ep), flush=True)
        return
    if args.batch_only:
        stream = torch.cuda.Stream()
        print(json.dumps(run_batched(api, torch, stream)), flush=True)
        return
    if args.engines_only:
        stream = torch.cuda.Stream()
        print(json.dumps(run_engines(api, torch, stream, grid=args.grid or 100)), flush=True)
        return
    if args.train_only:
        print(json.dumps(run_training(api, torch, args.train_only)), flush=True)
        return
    w = WORKLOAD
    M, K, J = w["M"], w["K"], w["grid"] ** 2
    P, O, pos, P0 = make_scan(rank)
    stream = torch.cuda.Stream()
    # --- synthetic data on the device: forward model of the truth + shot noise
    with torch.cuda.stream(stream):
        sim = api.Reconstruction(M, K, J, (w["obj"], w["obj"]), stream=stream.cuda_stream)
        sim.set_positions(pos)
        sim.set_init(O, P)
        I = torch.empty((J, M, M), dtype=torch.float32, device="cuda")
        sim.simulate(I)
        stream.synchronize()
        sim.close()
        scale = w["photons"] / float(I.sum(dim=(1, 2)).mean())
        gen = torch.Generator(device="cuda").manual_seed(1234 + rank)
        I = torch.poisson(I * scale, generator=gen)
        P0s = P0 * np.sqrt(scale)
        # the same scan at fractional positions (1/8-pixel shifts of the probe)
        pos_sub = synth.fractional_positions(pos, seed=2002 + rank)
        sim = api.Reconstruction(M, K, J, (w["obj"], w["obj"]), stream=stream.cuda_stream, subpixel=SUBPIXEL)
        sim.set_positions(pos_sub)
        sim.set_init(O, P)
        I_sub = torch.empty((J, M, M), dtype=torch.float32, device="cuda")
        sim.simulate(I_sub)
        stream.synchronize()
        sim.close()
        I_sub = torch.poisson(I_sub * scale, generator=gen)
    stream.synchronize()

    def timed(alg, istore="f32", steps=args.steps, warm=args.warmup, profile=False, likelihood="amplitude",
              subpixel=0, block_positions=0, fractional_data=None, residual_store="f32"):
        with torch.cuda.stream(stream):
            r = api.Reconstruction(M, K, J, (w["obj"], w["obj"]), stream=stream.cuda_stream, istore=istore,
                                   cluster=args.cluster, likelihood=likelihood, subpixel=subpixel,
                                   block_positions=block_positions, residual_store=residual_store)
            if subpixel or fractional_data:
                r.set_data(I_sub, pos_sub)
            else:
                r.set_data(I, pos)
            r.set_init(np.ones((w["obj"], w["obj"]), np.complex64), P0s)
            r.iterate(alg, warm)
            stream.synchronize()
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            clk = Clocks(local) if not profile else None
            n0 = r.launch_count
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if profile:
                r.set_profiling(True)
            e0.record(stream)
            r.iterate(alg, steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            launches = r.launch_count - n0
            clocks = clk.stop() if clk else None
            prof = r.get_profile() if profile else None
            err = r.fourier_error()
            refine_ms = None
            if subpixel:  # one position-refinement call (residual pass, fit, re-binning), wall clock
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r.refine_positions(step=0.5)
                refine_ms = (time.perf_counter() - t0) * 1e3
            r.close()
        ms = max_over_ranks(dist, ms)
        return dict(ms=ms, launches=launches, clocks=clocks, prof=prof, err=err, refine_ms=refine_ms)

    main_run = timed("lsqml", residual_store=args.residual_store)
    dm_run = timed("dm")
    f16_run = timed("lsqml", istore="f16")
    bf16_run = timed("lsqml", istore="bf16")
    poisson_run = timed("lsqml", likelihood="poisson")
    r16_run = timed("lsqml", residual_store="f16")
    r16a16_run = timed("lsqml", istore="f16", residual_store="f16")
    sub_run = timed("lsqml", subpixel=SUBPIXEL)
    # the same fractional-position data under the whole-pixel model (positions rounded)
    sub_rounded = timed("lsqml", fractional_data=True)
    sub_dm_run = timed("dm", subpixel=SUBPIXEL)
    blk_run = timed("lsqml", block_positions=J // 4)
    prof_run = timed("lsqml", steps=3, warm=1, profile=True, residual_store=args.residual_store)

    def rate(run):
        return aggregate_rate(J * args.steps, world, run["ms"] / 1e3)

    value = rate(main_run)
    # --- roofline of the dominant kernel (live CUDA-event durations)
    prof = prof_run["prof"]
    top = max(prof.items(), key=lambda kv: kv[1]["ms"])
    hbm, peak_kind = peaks()
    total_ms = sum(v["ms"] for v in prof.values())
    ms_launch = top[1]["ms"] / top[1]["launches"]
    bytes_launch = top[1]["bytes"] / top[1]["launches"]
    hbm_achieved = bytes_launch / (ms_launch / 1e3) / 1e9
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                   "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["bytes"] else None}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    # DRAM traffic of the residual pass from an ncu capture of the same kernel
    # on a 2500-position cut (profiles/fourier_chi_det256_2500pos.md): bytes
    # per position, scaled to this launch's positions (amplitudes in,
    # residuals out: traffic grows in proportion).  Only for the kernel and
    # shape that capture measured (FP32 residuals).
    traffic = None
    if top[0] == "fourier_chi" and (M, K) == (256, 1) and not args.cluster and args.residual_store == "f32":
        traffic = 768.5e3 * J
    step_bytes = sum(v["bytes"] for v in prof.values())
    if top[0].startswith("fourier"):
        # The fused Fourier kernel is bound by FP32 arithmetic issue, not by
        # DRAM (ncu: 16% DRAM, 50% issue-active): report it against the FP32
        # rate measured on this device by the library's FMA microbenchmark
        # (independent FMA chains on every SM; SM clock sampled meanwhile),
        # counting the forward + inverse 2-D FFT of each (position, mode) at
        # 5 N log2 N FLOP (N = M^2).
        fft_flop = J * K * 2 * 5.0 * M * M * np.log2(float(M * M))
        clk = Clocks(local)
        runs = [api.fp32_fma_peak(stream.cuda_stream) for _ in range(20)]
        pclk = clk.stop()
        peak_fp32, _, sms = max(runs)
        mhz = pclk["sm_mhz"] if pclk else None
        ach = fft_flop / (ms_launch / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": top[0], "achieved": ach, "peak": peak_fp32, "unit": "TFLOP/s",
                "frac": ach / peak_fp32,
                "peak_kind": (f"measured: ptycho_fp32_fma_peak (independent FMA chains, 8 x 256 threads on each of "
                              f"{sms} SMs, 2 flop per FMA), best of 20 runs"
                              + (f" at a median SM clock of {mhz:.0f} MHz" if mhz else "")),
                "peak_unit_count": {"sms": sms, "fp32_lanes_per_sm": 128,
                                    "at_sampled_clock_tflops": (sms * 128 * 2 * mhz * 1e6 / 1e12) if mhz else None},
                "flop_per_launch": fft_flop, "ms_per_launch": ms_launch, "traffic": traffic,
                "traffic_source": "ncu capture of the 2500-position cut, scaled per position" if traffic else None,
                "hbm": {"achieved": hbm_achieved, "peak": hbm, "unit": "GB/s", "frac": hbm_achieved / hbm,
                        "peak_kind": peak_kind, "bytes_per_launch": bytes_launch},
                "share_of_step": top[1]["ms"] / total_ms, "kernels": kernels,
                "step_bytes_per_pattern": step_bytes / (prof[top[0]]["launches"] * J)}
    else:
        roof = {"bound": "hbm", "kernel": top[0], "achieved": hbm_achieved, "peak": hbm, "unit": "GB/s",
                "frac": hbm_achieved / hbm, "peak_kind": peak_kind, "bytes_per_launch": bytes_launch,
                "ms_per_launch": ms_launch, "traffic": None, "share_of_step": top[1]["ms"] / total_ms,
                "kernels": kernels, "step_bytes_per_pattern": step_bytes / (prof[top[0]]["launches"] * J)}
    # --- end to end through the ABI from pinned host buffers
    # inputs and outputs in pinned host memory, allocated once per job queue
    I_host = I.cpu().pin_memory()
    O0 = torch.ones((w["obj"], w["obj"]), dtype=torch.complex64).pin_memory()
    P0h = torch.from_numpy(P0s.astype(np.complex64)).pin_memory()
    O_out = torch.empty_like(O0).pin_memory()
    P_out = torch.empty_like(P0h).pin_memory()
    e2e_times = []
    with torch.cuda.stream(stream):
        r = api.Reconstruction(M, K, J, (w["obj"], w["obj"]), stream=stream.cuda_stream)
        for s in range(2 + args.steps // 5 + 1):
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            r.set_data(I_host, pos)
            r.set_init(O0, P0h)
            r.iterate("lsqml", args.e2e_iters)
            Oo = r.get_object(O_out)
            Po = r.get_probe(P_out)
            dt = time.perf_counter() - t0
            if s >= 2:
                e2e_times.append(dt)
        r.close()
    e2e_dt = max_over_ranks(dist, statistics.median(e2e_times))
    # the same job from raw 16-bit detector counts (ptycho_set_data_raw: the
    # frames are already detector-centred M x M, so the crop is the identity;
    # counts at 65535 would be masked as saturated)
    I_u16 = torch.clamp(I, 0, 65535).to(torch.int32).to(torch.uint16).cpu().pin_memory()
    n_sat = int((I >= 65535).sum())
    raw_times = []
    with torch.cuda.stream(stream):
        r = api.Reconstruction(M, K, J, (w["obj"], w["obj"]), stream=stream.cuda_stream)
        for s in range(2 + args.steps // 5 + 1):
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            r.set_data_raw(I_u16, pos, (M // 2, M // 2), saturation_bits=16)
            r.set_init(O0, P0h)
            r.iterate("lsqml", args.e2e_iters)
            r.get_object(O_out)
            r.get_probe(P_out)
            dt = time.perf_counter() - t0
            if s >= 2:
                raw_times.append(dt)
        r.close()
    raw_dt = max_over_ranks(dist, statistics.median(raw_times))
    # a job queue with two contexts on their own streams: while one context
    # iterates (asynchronously), the host uploads the next job into the
    # other, so the 55 GB/s host link runs under the GPU work; every step
    # still copies one job's frames in and one job's results out
    q_streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    q_ctx = [api.Reconstruction(M, K, J, (w["obj"], w["obj"]), stream=qs.cuda_stream) for qs in q_streams]
    q_times = []
    q_ctx[0].set_data(I_host, pos)
    q_ctx[0].set_init(O0, P0h)
    for s in range(2 + args.steps // 5 + 1):
        if dist:
            dist.barrier()
        cur, nxt = q_ctx[s % 2], q_ctx[(s + 1) % 2]
        t0 = time.perf_counter()
        cur.iterate("lsqml", args.e2e_iters)
        nxt.set_data(I_host, pos)
        nxt.set_init(O0, P0h)
        cur.get_object(O_out)
        cur.get_probe(P_out)
        dt = time.perf_counter() - t0
        if s >= 2:
            q_times.append(dt)
    for c in q_ctx:
        c.close()
    q_dt = max_over_ranks(dist, statistics.median(q_times))
    h2d = I_host.numel() * 4 + pos.size * 4 + O0.numel() * 8 + P0h.numel() * 8
    d2h = Oo.numel() * 8 + Po.numel() * 8
    e2e = {"value": aggregate_rate(J * args.e2e_iters, world, e2e_dt), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h),
           "step": f"one job: set_data + set_init from pinned host memory, {args.e2e_iters} LSQML iterations, "
                   f"get_object + get_probe into pinned host memory",
           "raw_u16": {"value": aggregate_rate(J * args.e2e_iters, world, raw_dt), "unit": UNIT,
                       "h2d_bytes_per_step": int(I_u16.numel() * 2 + pos.size * 4 + O0.numel() * 8 + P0h.numel() * 8),
                       "saturated_pixels": n_sat,
                       "step": "the same job with the frames as 16-bit detector counts (set_data_raw)"},
           "job_queue": {"value": aggregate_rate(J * args.e2e_iters, world, q_dt), "unit": UNIT,
                         "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                         "step": "two contexts alternating: one job's iterations run while the next job's "
                                 "frames and start are uploaded from pinned host memory; then the results of "
                                 "the finished job are read back"}}
    profiling_run = args.small or args.grid > 0
    batched = None if (args.no_batch or profiling_run) else run_batched(api, torch, stream)
    t2e = None if (args.no_eps or profiling_run) else time_to_eps(api, torch, stream, I, pos, P0s, w)
    del I
    epie = None if profiling_run else run_epie(api, torch, stream)
    if epie is not None:
        epie["subpixel"] = run_epie(api, torch, stream, subpixel=SUBPIXEL)
    warm = None if (args.no_warm or profiling_run) else run_warm_start(api, torch, stream, n_frames=args.warm_frames)
    engines = None if profiling_run else run_engines(api, torch, stream)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cb = None
    if not args.no_cpu:
        cb = cpu_baseline(P, O, pos, P0, w)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_run["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(bench_config(world, w), **({"residual_store": args.residual_store}
                                                   if args.residual_store != "f32" else {})),
        "by_variant": {
            "lsqml_f32": {"value": value, "fourier_error": main_run["err"]},
            "dm_f32": {"value": rate(dm_run), "fourier_error": dm_run["err"]},
            "lsqml_f16": {"value": rate(f16_run), "fourier_error": f16_run["err"]},
            "lsqml_poisson_f32": {"value": rate(poisson_run), "fourier_error": poisson_run["err"]},
            "lsqml_bf16": {"value": rate(bf16_run), "fourier_error": bf16_run["err"]},
            "lsqml_f32_residual16": {"value": rate(r16_run), "fourier_error": r16_run["err"],
                                     "note": "LSQML residuals stored as FP16 between the passes"},
            "lsqml_f16_residual16": {"value": rate(r16a16_run), "fourier_error": r16a16_run["err"],
                                     "note": "FP16 amplitudes and FP16 residuals"},
            f"lsqml_subpixel{SUBPIXEL}_f32": {"value": rate(sub_run), "fourier_error": sub_run["err"],
                                              "positions": "whole-pixel raster + uniform [0, 1) offsets",
                                              "fourier_error_rounded_positions": sub_rounded["err"],
                                              "refine_positions_ms": sub_run["refine_ms"]},
            f"dm_subpixel{SUBPIXEL}_f32": {"value": rate(sub_dm_run), "fourier_error": sub_dm_run["err"]},
            "lsqml_blocked_f32": {"value": rate(blk_run), "fourier_error": blk_run["err"],
                                  "block_positions": J // 4,
                                  "note": "residuals of a quarter of the positions resident; two Fourier passes"},
        },
        "batched": batched,
        "time_to_eps": t2e,
        "warm_start": warm,
        "fft_engines_64": engines,
        "epie": epie,
        "roofline": roof,
        "cpu_baseline": cb,
        "e2e": e2e,
        "gpu_launches": main_run["launches"],
        "clocks": main_run["clocks"],
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

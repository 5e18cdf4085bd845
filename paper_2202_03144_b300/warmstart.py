"""Learned warm start: training set, training loop and the time-to-epsilon
comparison against a flat start.

Everything numeric runs in the library's CUDA kernels through the C ABI
(forward model, network forward/backward, AdamW, stitching, reconstruction);
this module only orders the calls.  torch provides device memory, the
shuffling permutation and the Poisson draws of the synthetic training frames.

Training frames follow the 3-mode 128^2 workload: the probe of that workload,
synthetic objects drawn like the 256^2-object workload (smoothed amplitude in
[0.8, 1], smoothed phase in [-pi/2, pi/2]), uniformly random scan positions,
Poisson noise at ``photons`` per frame.  Targets are the amplitude and phase
of the central 64^2 patch of the true object at each position.
"""
from __future__ import annotations

import time

import numpy as np

from . import api, synth

M_NET = 128


def training_probe():
    return synth.make_probe(M_NET, 3, R=40.0, sigma=8.0, c=0.005)


def make_training_set(n_frames: int, seed: int = 0, photons: float = 1e5, per_object: int = 4096,
                      obj_side: int = 1088, stream=None):
    """(frames [N,128,128], targets [N,2,64,64]) float32 torch CUDA tensors."""
    import torch
    P = training_probe()
    frames = torch.empty((n_frames, M_NET, M_NET), dtype=torch.float32, device="cuda")
    targets = torch.empty((n_frames, 2, 64, 64), dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(seed)
    rng = np.random.default_rng(seed)
    done = 0
    k = 0
    scale = None
    while done < n_frames:
        J = min(per_object, n_frames - done)
        O = synth.make_object(obj_side, obj_side, seed=50000 + seed * 1000 + k)
        pos = rng.integers(0, obj_side - M_NET + 1, size=(J, 2)).astype(np.float64)
        with api.Reconstruction(M_NET, 3, J, (obj_side, obj_side), stream=stream) as r:
            r.set_positions(pos)
            r.set_init(O, P)
            I = frames[done:done + J]
            r.simulate(I)
            api.object_patches(r, targets[done:done + J])
            torch.cuda.synchronize()
        if scale is None:
            scale = photons / float(I.sum(dim=(1, 2)).mean())
        frames[done:done + J] = torch.poisson(I * scale, generator=gen)
        done += J
        k += 1
    return frames, targets, scale


def train(net: "api.Net", frames, targets, epochs: int = 1, batch: int = 64, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Minibatch AdamW over shuffled frames; learning rate decays by 10x
    (cosine) over the run.  Returns (losses every log_every steps, seconds)."""
    import torch
    n = frames.shape[0]
    steps = epochs * (n // batch)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = 0
    for _ in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            fb = frames.index_select(0, idx).contiguous()
            tb = targets.index_select(0, idx).contiguous()
            cur = lr * (0.1 + 0.9 * 0.5 * (1 + np.cos(np.pi * s / max(steps, 1))))
            want = log_every > 0 and (s % log_every == 0 or s == steps - 1)
            L = net.train_step(fb, tb, cur, want_loss=want)
            if want:
                losses.append((s, L))
            s += 1
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def iterations_to_eps(rec, alg: str, eps: float, limit: int, check: int = 5):
    """Iterate until the Fourier error is <= eps (checked every `check`
    iterations).  Returns (iterations, seconds, final error)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it = 0
    E = rec.fourier_error()
    while it < limit and E > eps:
        rec.iterate(alg, check)
        it += check
        E = rec.fourier_error()
    return it, time.perf_counter() - t0, E


def compare(net, scan: dict, I, alg: str = "lsqml", n_ref: int = 50, check: int = 5, stream=None):
    """Flat start vs warm start on one scan.  eps = the Fourier error the
    flat start reaches after n_ref iterations; the warm start's time includes
    its network inference and stitching."""
    import torch
    M, K = scan["M"], scan["K"]
    pos = scan["positions"]
    shape = scan["object0"].shape
    J = len(pos)
    res = {}
    with api.Reconstruction(M, K, J, shape, stream=stream) as r:
        r.set_data(I, pos)
        r.set_init(scan["object0"], scan["probe0"])
        E0_flat = r.fourier_error()
        # same checking cadence as the warm start, so both pay the same
        # error evaluations; eps is where the flat start ends
        it, t_flat, eps = iterations_to_eps(r, alg, -1.0, limit=n_ref, check=check)
    res["eps"] = eps
    res["flat"] = {"initial_error": E0_flat, "iterations": it, "seconds": t_flat}
    with api.Reconstruction(M, K, J, shape, stream=stream) as r:
        r.set_data(I, pos)
        r.set_init(scan["object0"], scan["probe0"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.warm_start(r, net)
        t_inf = time.perf_counter() - t0
        E0_warm = r.fourier_error()
        it, t_it, E = iterations_to_eps(r, alg, eps, limit=2 * n_ref, check=check)
    res["warm"] = {"initial_error": E0_warm, "iterations": it, "seconds": t_inf + t_it,
                   "inference_and_stitch_seconds": t_inf, "final_error": E, "reached": bool(E <= eps)}
    return res


def time_inference(n_warm: int = 4, n_predict: int = 3, seed: int = 11):
    """Wall time of the warm start (network inference + stitching) on the
    1600-position 3-mode 128^2 spiral scan, with an untrained network (the
    time does not depend on the weights), and of predictions of 256 frames.
    Returns (warm-start seconds per call, predict seconds per 256 frames)."""
    import torch
    d = synth.scan_config("modes128", seed=5)
    M, K, pos = d["M"], d["K"], d["positions"]
    shape = d["object"].shape
    with api.Reconstruction(M, K, len(pos), shape) as sim:
        sim.set_positions(pos)
        sim.set_init(d["object"], d["probe"])
        I = torch.empty((len(pos), M, M), dtype=torch.float32, device="cuda")
        sim.simulate(I)
        torch.cuda.synchronize()
    with api.Net(seed=seed, max_batch=256) as net, api.Reconstruction(M, K, len(pos), shape) as r:
        r.set_data(I, pos)
        r.set_init(d["object0"], d["probe0"])
        ws = []
        for _ in range(n_warm):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            api.warm_start(r, net)
            torch.cuda.synchronize()
            ws.append(time.perf_counter() - t0)
        out = torch.empty((256, 2, 64, 64), dtype=torch.float32, device="cuda")
        fr = I[:256].contiguous()
        pr = []
        for _ in range(n_predict):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            net.predict(fr, out)
            torch.cuda.synchronize()
            pr.append(time.perf_counter() - t0)
    return min(ws), min(pr)


if __name__ == "__main__":
    w, p = time_inference()
    print(f"warm start (1600 frames): {w * 1e3:.2f} ms; predict (256 frames): {p * 1e3:.3f} ms")

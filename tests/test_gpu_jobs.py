"""Contexts reused for one scan after another, and two contexts run as a job
queue on their own streams (one iterates while the host uploads the next
job into the other): every job's result equals that of a fresh context on
the same data, bit for bit.  set_data keeps its tile lists while they fit
and grows them when a denser scan needs more (a free would wait for the
whole device)."""
import numpy as np
import pytest

from gpu_cases import scan
from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api, synth

pytestmark = pytest.mark.gpu


def _fresh(c, n, shape, **kw):
    with api.Reconstruction(c["M"], c["K"], len(c["pos"]), shape, **kw) as r:
        r.set_data(c["I"].astype(np.float32), c["pos"])
        r.set_init(np.ones(shape, np.complex64), c["P0"])
        r.iterate("lsqml", n)
        return r.get_object(), r.get_probe()


def _scan_at(pos, M=32, shape=(160, 160), seed=0):
    """The oracle's data for given positions on a seeded object and probe."""
    P = synth.make_probe(M, 1, R=M / 4.0, sigma=M / 16.0, c=0.6 / M)
    O = synth.make_object(shape[0], shape[1], seed=seed + 2, smooth=2.0)
    pos = np.asarray(pos, np.float64)
    I = orc.far_field_intensity(O, P, orc.round_positions(pos))
    I = synth.poisson(I * 1e5 / I.sum(axis=(1, 2)).mean(), seed=seed + 3)
    return dict(M=M, K=1, pos=pos, I=I, P0=synth.noisy_probe(P, 0.1, seed=seed + 5))


def _tile_entries(pos, M=32, ty=32, tx=64):
    n = 0
    for y, x in np.rint(pos).astype(int):
        n += ((y + M - 1) // ty - y // ty + 1) * ((x + M - 1) // tx - x // tx + 1)
    return n


def test_reused_context_matches_fresh_ones_as_the_tile_lists_grow():
    """One context of fixed size takes three scans of the same position count
    in turn: patches inside single object tiles, patches across tile corners
    (more than twice the tile-list entries: the lists grow) and the first again."""
    M, J = 32, 16
    shape = (160, 160)
    g = np.arange(4)
    inside = np.stack(np.meshgrid(g * 32, g * 32 + 8, indexing="ij"), -1).reshape(-1, 2)[:J]
    across = np.stack(np.meshgrid(g * 32 + 16, (g % 2) * 64 + 40, indexing="ij"), -1).reshape(-1, 2)[:J]
    assert _tile_entries(across) > 2 * _tile_entries(inside)
    a, b = _scan_at(inside, seed=51), _scan_at(across, seed=52)
    with api.Reconstruction(M, 1, J, shape) as r:
        for c in (a, b, a):
            r.set_data(c["I"].astype(np.float32), c["pos"])
            r.set_init(np.ones(shape, np.complex64), c["P0"])
            r.iterate("lsqml", 3)
            O, P = r.get_object(), r.get_probe()
            Of, Pf = _fresh(c, 3, shape)
            assert np.array_equal(O, Of) and np.array_equal(P, Pf)


def test_two_context_job_queue_matches_fresh_contexts():
    torch = pytest.importorskip("torch")
    M = 64
    jobs = [scan(M, 1, grid=3, photons=1e5, seed=60 + i) for i in range(4)]
    shape = tuple(max(c["shape"][d] for c in jobs) for d in range(2))
    J = len(jobs[0]["pos"])
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ctx = [api.Reconstruction(M, 1, J, shape, stream=s.cuda_stream) for s in streams]
    try:
        def load(r, c):
            r.set_data(c["I"].astype(np.float32), c["pos"])
            r.set_init(np.ones(shape, np.complex64), c["P0"])

        load(ctx[0], jobs[0])
        got = []
        for i in range(len(jobs)):
            cur, nxt = ctx[i % 2], ctx[(i + 1) % 2]
            cur.iterate("lsqml", 4)                 # asynchronous
            if i + 1 < len(jobs):
                load(nxt, jobs[i + 1])              # while cur's iterations run
            got.append((cur.get_object(), cur.get_probe()))
    finally:
        for r in ctx:
            r.close()
    for c, (O, P) in zip(jobs, got):
        Of, Pf = _fresh(c, 4, shape)
        assert np.array_equal(O, Of) and np.array_equal(P, Pf)

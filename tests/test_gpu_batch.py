"""Batched reconstructions (one CUDA graph per iteration) and the autotuner.

Every member of a batch must end exactly where the same reconstruction run
alone ends (same kernels, same order inside each member: bit-identical), and
within the parity tolerance of the FP64 oracle."""
import numpy as np
import pytest

from gpu_cases import illuminated, scan
from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api
from util import align_global, rel_l2

pytestmark = pytest.mark.gpu

SHAPES = [(16, 1, 3), (32, 1, 4), (64, 1, 3), (96, 1, 2), (32, 3, 3), (192, 1, 2)]


def _cases():
    return [scan(M, K, grid=g, photons=1e5, seed=10 + i) for i, (M, K, g) in enumerate(SHAPES)]


@pytest.mark.parametrize("alg", ["dm", "lsqml"])
def test_batch_matches_single_and_oracle(alg):
    cases = _cases()
    n = 3
    members = [dict(M=c["M"], K=c["K"], J=len(c["pos"]), obj_shape=c["shape"], probe_start=1) for c in cases]
    with api.Batch(members) as b:
        for m, c in zip(b.members, cases):
            m.set_data(c["I"].astype(np.float32), c["pos"])
            m.set_init(c["O0"], c["P0"])
        b.iterate(alg, n)
        assert b.kernels_per_iteration > len(cases)
        got = [(m.get_object(), m.get_probe(), m.iteration) for m in b.members]
    for (Og, Pg, t), c in zip(got, cases):
        assert t == n
        with api.Reconstruction(c["M"], c["K"], len(c["pos"]), c["shape"], probe_start=1) as r:
            r.set_data(c["I"].astype(np.float32), c["pos"])
            r.set_init(c["O0"], c["P0"])
            r.iterate(alg, n)
            Os, Ps = r.get_object(), r.get_probe()
        assert np.array_equal(Og, Os) and np.array_equal(Pg, Ps), c["M"]
        Oc, Pc, _ = orc.reconstruct(alg, c["O0"], c["P0"], c["pos"], c["I"], n, probe_start=1)
        m = illuminated(c["P"], c["pos"], c["shape"])
        assert rel_l2(align_global(Og, Oc, m), Oc, m) < 1e-4 and rel_l2(Pg, Pc) < 1e-4, c["M"]


def test_batch_rejects_epie_and_missing_data():
    c = scan(32, 1, grid=2)
    with api.Batch([dict(M=32, K=1, J=len(c["pos"]), obj_shape=c["shape"])]) as b:
        with pytest.raises(api.PtychoError) as e:
            b.iterate("lsqml", 1)
        assert e.value.name == "STATE"
        b.members[0].set_data(c["I"].astype(np.float32), c["pos"])
        with pytest.raises(api.PtychoError) as e:
            b.iterate("epie", 1)
        assert e.value.name == "UNSUPPORTED"


def test_autotune_picks_a_compiled_cluster():
    best, ms = api.autotune(64, 1)
    assert best in (1, 2, 4) and ms > 0
    assert api.autotune(64, 1) == (best, ms)  # cached
    c = scan(64, 1, grid=2)
    with api.Reconstruction(64, 1, len(c["pos"]), c["shape"], cluster=-1) as r:
        assert r.cluster == best


def _bytes(c):
    M, K, J = c["M"], c["K"], len(c["pos"])
    return J * M * M * (8 * K + 4) + c["shape"][0] * c["shape"][1] * 24


@pytest.mark.parametrize("budget", [0, 1, 200_000, 1 << 30])
def test_batch_group_schedule_is_bit_identical(budget):
    """The group budget only reorders independent work: every schedule gives
    the results of the default one bit for bit; the plan follows the packing
    rule (a member at or above the budget alone, the rest packed largest
    first without exceeding it)."""
    cases = _cases()
    members = [dict(M=c["M"], K=c["K"], J=len(c["pos"]), obj_shape=c["shape"]) for c in cases]
    outs = []
    for gb in (None, budget):
        with api.Batch(members, group_bytes=gb) as b:
            for m, c in zip(b.members, cases):
                m.set_data(c["I"].astype(np.float32), c["pos"])
                m.set_init(c["O0"], c["P0"])
            b.iterate("lsqml", 2)
            outs.append([(m.get_object(), m.get_probe()) for m in b.members])
            groups = b.groups()
    for (O1, P1), (O2, P2) in zip(*outs):
        assert np.array_equal(O1, O2) and np.array_equal(P1, P2)
    w = [_bytes(c) for c in cases]
    ng = max(groups) + 1
    assert sorted(set(groups)) == list(range(ng))
    if budget <= 0:
        assert ng == 1
    for g in range(ng):
        idx = [i for i in range(len(cases)) if groups[i] == g]
        if budget > 0 and len(idx) > 1:
            assert sum(w[i] for i in idx) <= budget
            assert all(w[i] < budget for i in idx)
    if budget == 1:
        assert ng == len(cases)
    if budget == 1 << 30:
        assert ng == 1


@pytest.mark.parametrize("lanes", [1, 2, 3])
def test_batch_lane_schedule_is_bit_identical(lanes):
    """Lanes (chains of members run side by side, no barrier between chains)
    reorder independent work only: DM and LSQML give the group schedule's
    results bit for bit, DM's exit waves included.  Members go largest work
    first to the least-loaded chain, so the chains' work differs by at most
    one member's."""
    cases = _cases()
    members = [dict(M=c["M"], K=c["K"], J=len(c["pos"]), obj_shape=c["shape"]) for c in cases]
    for alg in ("lsqml", "dm"):
        outs = []
        for ln in (0, lanes):
            with api.Batch(members) as b:
                b.set_lanes(ln)
                assert b.lanes == ln
                for m, c in zip(b.members, cases):
                    m.set_data(c["I"].astype(np.float32), c["pos"])
                    m.set_init(c["O0"], c["P0"])
                b.iterate(alg, 2)
                outs.append([(m.get_object(), m.get_probe(), m.fourier_error()) for m in b.members])
                chain = b.groups()
        for (O1, P1, E1), (O2, P2, E2) in zip(*outs):
            assert np.array_equal(O1, O2) and np.array_equal(P1, P2) and E1 == E2
        assert max(chain) + 1 == min(lanes, len(cases))
        work = [len(c["pos"]) * c["K"] * c["M"] ** 2 * (np.log2(c["M"]) + 6) for c in cases]
        load = [sum(w for w, l in zip(work, chain) if l == k) for k in range(max(chain) + 1)]
        assert max(load) - min(load) <= max(work) * (1 + 1e-12)


def test_batch_autotune_keeps_the_fastest_budget_and_the_results():
    """The group-budget autotuner times real iterations under each distinct
    partition and keeps the fastest; the members end exactly where the same
    number of iterations under a fixed budget ends (the schedule only
    reorders independent work)."""
    cases = _cases()
    members = [dict(M=c["M"], K=c["K"], J=len(c["pos"]), obj_shape=c["shape"]) for c in cases]
    with api.Batch(members) as b:
        for m, c in zip(b.members, cases):
            m.set_data(c["I"].astype(np.float32), c["pos"])
            m.set_init(c["O0"], c["P0"])
        gb, lanes, ms = b.autotune("lsqml", 1)
        assert gb in (0, 64 << 20, 128 << 20, 256 << 20, 512 << 20, 1 << 30, 2 << 30, 4 << 30) and ms > 0
        assert lanes in (0, 2, 4, 8, 16, 32) and b.lanes == lanes
        n = b.members[0].iteration
        assert n >= 2 and all(m.iteration == n for m in b.members)
        tuned = [(m.get_object(), m.get_probe()) for m in b.members]
    with api.Batch(members, group_bytes=1) as b:
        for m, c in zip(b.members, cases):
            m.set_data(c["I"].astype(np.float32), c["pos"])
            m.set_init(c["O0"], c["P0"])
        b.iterate("lsqml", n)
        ref = [(m.get_object(), m.get_probe()) for m in b.members]
    for (O1, P1), (O2, P2) in zip(tuned, ref):
        assert np.array_equal(O1, O2) and np.array_equal(P1, P2)


def test_batch_members_with_poisson_and_mode_orthogonalisation():
    """Per-member options reach the captured graph: Poisson-likelihood LSQML
    and orthogonalised 3-mode probes give the results of the same members run
    alone, bit for bit."""
    cases = [scan(32, 3, grid=3, photons=1e5, seed=21), scan(64, 1, grid=3, photons=1e5, seed=22)]
    opts = [dict(probe_ortho=1, likelihood="poisson"), dict(likelihood="poisson")]
    members = [dict(M=c["M"], K=c["K"], J=len(c["pos"]), obj_shape=c["shape"], **o) for c, o in zip(cases, opts)]
    with api.Batch(members) as b:
        for m, c in zip(b.members, cases):
            m.set_data(c["I"].astype(np.float32), c["pos"])
            m.set_init(c["O0"], c["P0"])
        b.iterate("lsqml", 3)
        got = [(m.get_object(), m.get_probe()) for m in b.members]
    for (Og, Pg), c, o in zip(got, cases, opts):
        with api.Reconstruction(c["M"], c["K"], len(c["pos"]), c["shape"], **o) as r:
            r.set_data(c["I"].astype(np.float32), c["pos"])
            r.set_init(c["O0"], c["P0"])
            r.iterate("lsqml", 3)
            assert np.array_equal(Og, r.get_object()) and np.array_equal(Pg, r.get_probe())


@pytest.mark.parametrize("alg", ["dm", "lsqml"])
def test_batch_members_with_subpixel_positions(alg):
    """Sub-pixel members (shifted-probe tables, the DM probe solve) inside the
    captured graph: bit-identical to the members run alone, beside an
    integer-position member."""
    from gpu_cases import subpixel_scan
    cases = [subpixel_scan(32, 2, 8, grid=3, photons=1e5, seed=31), subpixel_scan(64, 1, 4, grid=3, photons=1e5, seed=32),
             scan(32, 1, grid=3, photons=1e5, seed=33)]
    opts = [dict(subpixel=8), dict(subpixel=4), dict()]
    members = [dict(M=c["M"], K=c["K"], J=len(c["pos"]), obj_shape=c["shape"], **o) for c, o in zip(cases, opts)]
    with api.Batch(members) as b:
        for m, c in zip(b.members, cases):
            m.set_data(c["I"].astype(np.float32), c["pos"])
            m.set_init(c["O0"], c["P0"])
        b.iterate(alg, 3)
        got = [(m.get_object(), m.get_probe()) for m in b.members]
    for (Og, Pg), c, o in zip(got, cases, opts):
        with api.Reconstruction(c["M"], c["K"], len(c["pos"]), c["shape"], **o) as r:
            r.set_data(c["I"].astype(np.float32), c["pos"])
            r.set_init(c["O0"], c["P0"])
            r.iterate(alg, 3)
            assert np.array_equal(Og, r.get_object()) and np.array_equal(Pg, r.get_probe())


def test_batch_full_workload_sampled():
    """The benchmark's 64-member batch (probe sizes 64-256, 100-4000
    positions each, autotuned clusters, grouped graph): three sampled members
    end bit for bit where they end alone, and the smallest member -- its
    frames from the oracle's forward model -- matches the oracle to 1e-4.
    Starts are random objects (a flat start makes the first projection
    ill-conditioned; see test_gpu_configs)."""
    torch = pytest.importorskip("torch")
    from paper_2202_03144_b300 import synth
    members = synth.batch_members(64, seed=7)
    side = max(max(m["obj_shape"]) for m in members)
    field = synth.make_object(side, side, seed=4242)
    field0 = synth.make_object(side, side, seed=4343)
    probes = {M: synth.make_probe(M, 1, R=0.3125 * M, sigma=M / 16.0, c=0.02 * (64.0 / M) ** 2)
              for M in sorted(set(m["M"] for m in members))}
    small = int(np.argmin([m["J"] * m["M"] ** 2 for m in members]))
    big = next(i for i, m in enumerate(members) if m["M"] == 256)
    mid = next(i for i, m in enumerate(members) if m["M"] == 96)
    spec = [dict(M=m["M"], K=1, J=m["J"], obj_shape=m["obj_shape"], cluster=-1) for m in members]
    gen = torch.Generator(device="cuda").manual_seed(99)
    data, starts, clusters = [], [], []
    with api.Batch(spec) as b:
        for i, (mem, m) in enumerate(zip(b.members, members)):
            P = probes[m["M"]]
            ny, nx = m["obj_shape"]
            if i == small:  # the member checked against the oracle: oracle frames
                I = orc.far_field_intensity(field[:ny, :nx], P, orc.round_positions(m["positions"]))
                sc = m["photons"] / I.sum(axis=(1, 2)).mean()
                I = synth.poisson(I * sc, seed=5).astype(np.float32)
            else:
                mem.set_positions(m["positions"])
                mem.set_init(field[:ny, :nx], P)
                It = torch.empty((m["J"], m["M"], m["M"]), dtype=torch.float32, device="cuda")
                mem.simulate(It)
                torch.cuda.synchronize()
                sc = m["photons"] / float(It.sum(dim=(1, 2)).mean())
                I = torch.poisson(It * sc, generator=gen).cpu().numpy()
                del It
            data.append(I)
            starts.append((field0[:ny, :nx], synth.noisy_probe(P * np.sqrt(sc), 0.1, seed=i)))
            clusters.append(mem.cluster)
            mem.set_data(I, m["positions"])
            mem.set_init(*starts[-1])
        b.iterate("lsqml", 2)
        got = {i: (b.members[i].get_object(), b.members[i].get_probe()) for i in (small, big, mid)}
    for i in (small, big, mid):
        m = members[i]
        with api.Reconstruction(m["M"], 1, m["J"], m["obj_shape"], cluster=clusters[i]) as r:
            r.set_data(data[i], m["positions"])
            r.set_init(*starts[i])
            r.iterate("lsqml", 2)
            assert np.array_equal(got[i][0], r.get_object()) and np.array_equal(got[i][1], r.get_probe()), i
    m = members[small]
    Oc, Pc, _ = orc.reconstruct("lsqml", starts[small][0], starts[small][1], m["positions"],
                                data[small].astype(np.float64), 2)
    mask = illuminated(probes[m["M"]], m["positions"], m["obj_shape"])
    Og, Pg = got[small]
    assert rel_l2(align_global(Og, Oc, mask), Oc, mask) < 1e-4 and rel_l2(Pg, Pc) < 1e-4

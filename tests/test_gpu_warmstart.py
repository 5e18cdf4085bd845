"""What the trained warm-start network gains over the plain method.

A network trained briefly (49,152 simulated frames, 3 epochs) on objects drawn
like the synthetic workloads, then used on a held-out scan (new object seed,
400-position Fermat spiral, 3-mode 128^2 probe, Poisson noise): its stitched
patches must start LSQML at a lower Fourier error than the flat object and
reach the error the flat start reaches after 30 iterations in fewer
iterations.  The intensities of the held-out scan come from the FP64 oracle's
forward model."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2202_03144_b300 import api, synth, warmstart

pytestmark = pytest.mark.gpu


def _held_out_scan(seed=123, J=400):
    M, K = 128, 3
    P = warmstart.training_probe()
    pos = synth.spiral_positions(J, 20.0, (0.0, 0.0))
    pos = pos - pos.min(0) + 8
    ny, nx = synth.object_shape_for(pos, M, margin=8, multiple=16)
    O = synth.make_object(ny, nx, seed=seed)
    I = orc.far_field_intensity(O, P, orc.round_positions(pos))
    I = synth.poisson(I * 1e5 / I.sum(axis=(1, 2)).mean(), seed=seed + 1)
    P0 = synth.make_probe(M, K, R=44.0, sigma=8.0, c=0.005)
    # the initial probe carries the data's power (Parseval: frame sum / M^2)
    P0 = P0 * np.sqrt(I.sum(axis=(1, 2)).mean() / (M * M) / np.sum(np.abs(P0) ** 2))
    return dict(M=M, K=K, positions=pos, object0=synth.flat_object(ny, nx), probe0=P0), I


def test_warm_start_beats_flat_start():
    torch = pytest.importorskip("torch")
    frames, targets, _ = warmstart.make_training_set(49152, seed=3, per_object=12288)
    with api.Net(seed=11, max_batch=64) as net:
        losses, secs = warmstart.train(net, frames, targets, epochs=3, batch=64, lr=1e-3, log_every=100)
        assert losses[-1][1] < 0.5 * losses[0][1], losses
        scan, I = _held_out_scan()
        It = torch.from_numpy(I.astype(np.float32)).cuda()
        res = warmstart.compare(net, scan, It, alg="lsqml", n_ref=30, check=5)
    print(res)
    assert res["warm"]["initial_error"] < res["flat"]["initial_error"], res
    assert res["warm"]["reached"] and res["warm"]["iterations"] < res["flat"]["iterations"], res

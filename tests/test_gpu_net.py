"""Warm-start network on the GPU against the FP64 oracle.

Two checks of the same kernels:
* verification mode (FP32 activation storage) against the unrounded oracle on
  the same BF16 weights: only FP32-vs-FP64 summation differs -> relative L2
  <= 1e-4 per output and per parameter tensor;
* the method (BF16 activations) against the oracle that rounds its input and
  hidden activations to BF16 as well.  Those roundings decide ReLU masks and
  ~1e-6 summation differences flip a share of them: perturbing the oracle's
  own pre-activations by 1e-6 relative noise moves its per-tensor gradients by
  up to 6%, so the tolerance there is 8e-2 (gradients) and 2e-2 (output, loss).
"""
import numpy as np
import pytest

from oracle import net_oracle as orc_net
from paper_2202_03144_b300 import api

pytestmark = pytest.mark.gpu


def _batch(B, seed):
    rng = np.random.default_rng(seed)
    I = np.exp(rng.uniform(0, 7, (B, 128, 128))).astype(np.float32) - 1.0
    t = (0.5 * rng.standard_normal((B, 2, 64, 64))).astype(np.float32)
    return I, t


def _oracle_params(p):
    q = np.asarray(p, np.float64).copy()
    for (wo, bo), (ci, co, *_) in zip(orc_net.layout()[0], orc_net.LAYERS):
        q[wo:wo + co * ci * 9] = orc_net.bf16_round(p[wo:wo + co * ci * 9])
    return q


def _compare(f32, tol_out, tol_grad):
    torch = pytest.importorskip("torch")
    I, t = _batch(2, 1)
    with api.Net(seed=3, max_batch=4, f32_activations=f32) as net:
        p = net.get_params()
        assert p.size == orc_net.layout()[1]
        It, tt = torch.from_numpy(I).cuda(), torch.from_numpy(t).cuda()
        out = torch.empty((2, 2, 64, 64), dtype=torch.float32, device="cuda")
        net.predict(It, out)
        torch.cuda.synchronize()
        L, g = net.gradients(It, tt)
        L2, g2 = net.gradients(It, tt)
    assert L == L2 and np.array_equal(g, g2), "gradients not deterministic"
    q = _oracle_params(p)
    ref_out, _ = orc_net.forward(q, I, act_bf16=not f32)
    o = out.cpu().numpy()
    assert np.linalg.norm(o - ref_out) / np.linalg.norm(ref_out) < tol_out
    Lr, gr = orc_net.loss_and_grads(q, I, t, act_bf16=not f32)
    assert abs(L - Lr) / Lr < tol_out
    errs = []
    for l, ((wo, bo), (ci, co, *_)) in enumerate(zip(orc_net.layout()[0], orc_net.LAYERS)):
        for kind, (a, b) in (("w", (wo, wo + co * ci * 9)), ("b", (bo, bo + co))):
            errs.append((l, kind, float(np.linalg.norm(g[a:b] - gr[a:b]) / max(np.linalg.norm(gr[a:b]), 1e-30))))
    print("per-tensor relative gradient error:", errs)
    assert all(e < tol_grad for _, _, e in errs), errs


def test_kernels_match_oracle_with_fp32_activations():
    _compare(True, 1e-4, 1e-4)


def test_bf16_method_matches_bf16_oracle():
    _compare(False, 2e-2, 8e-2)


def test_training_reduces_loss_on_a_fixed_batch():
    torch = pytest.importorskip("torch")
    I, _ = _batch(8, 2)
    # a learnable target: the centre of the (log) frame, in both channels
    c = (np.log1p(I[:, 32:96, 32:96]) / 10.0).astype(np.float32)
    t = np.stack([c, -c], axis=1)
    It, tt = torch.from_numpy(I).cuda(), torch.from_numpy(t).cuda()
    with api.Net(seed=5, max_batch=8) as net:
        L0 = net.train_step(It, tt, 1e-3, want_loss=True)
        for _ in range(30):
            L = net.train_step(It, tt, 1e-3, want_loss=True)
    assert L < 0.5 * L0, (L0, L)


def test_set_params_roundtrip_and_errors():
    with api.Net(seed=7, max_batch=2) as net:
        p = net.get_params()
        p2 = p * 0.5
        net.set_params(p2)
        assert np.array_equal(net.get_params(), p2.astype(np.float32))
        bad = p.copy()
        bad[3] = np.nan
        with pytest.raises(api.PtychoError) as e:
            net.set_params(bad)
        assert e.value.name == "NONFINITE"


def test_tensor_core_forward_matches_cuda_cores():
    """Forward convolutions as tcgen05 implicit GEMMs (the default) against the
    CUDA-core kernels on identical BF16 weights and frames; only the FP32
    summation order differs (then BF16-rounded per layer): 1e-2."""
    torch = pytest.importorskip("torch")
    I, _ = _batch(8, 4)
    It = torch.from_numpy(I).cuda()
    outs = []
    for cc in (False, True):
        with api.Net(seed=9, max_batch=8, cuda_cores=cc) as net:
            o = torch.empty((8, 2, 64, 64), dtype=torch.float32, device="cuda")
            net.predict(It, o)
            net.predict(It, o)  # second call: reused tensor memory and barriers
            torch.cuda.synchronize()
            outs.append(o.cpu().numpy())
    e = np.linalg.norm(outs[0] - outs[1]) / np.linalg.norm(outs[1])
    print("tensor-core vs CUDA-core forward:", e)
    assert e < 1e-2


def test_inference_forward_follows_parameter_updates():
    """The inference forward (channel-last tensor-core convolutions with a
    cached tap-major copy of the weights) tracks every parameter change:
    after a training step and after set_params its predictions match a
    CUDA-core network holding the same parameters (1e-2, summation order)."""
    torch = pytest.importorskip("torch")
    I, t = _batch(4, 6)
    It, tt = torch.from_numpy(I).cuda(), torch.from_numpy(t).cuda()

    def rel(a, b):
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))

    with api.Net(seed=21, max_batch=4) as net, api.Net(seed=0, max_batch=4, cuda_cores=True) as ref:
        o = torch.empty((4, 2, 64, 64), dtype=torch.float32, device="cuda")
        r = torch.empty_like(o)
        net.predict(It, o)  # builds the cached weights
        net.train_step(It, tt, 1e-2)
        ref.set_params(net.get_params())
        net.predict(It, o)
        ref.predict(It, r)
        torch.cuda.synchronize()
        assert rel(o, r) < 1e-2
        p2 = (net.get_params() * 0.7).astype(np.float32)
        net.set_params(p2)
        ref.set_params(p2)
        net.predict(It, o)
        ref.predict(It, r)
        torch.cuda.synchronize()
        assert rel(o, r) < 1e-2


@pytest.mark.parametrize("B", [64, 37], ids=["batch64", "batch37"])
def test_tensor_core_gradients_match_cuda_cores_at_training_batches(B):
    """The tensor-core backward (tap-major gathers, parity-class stride-2 data
    gradients, pixel-split weight gradients summed in order) at the training
    batch and at a ragged one, against the CUDA-core backward on identical
    BF16 weights and frames.  The two forwards sum in different orders before
    each BF16 rounding, so ReLU masks flip between them as between the method
    and the oracle: the same 8e-2 per gradient tensor, 2e-2 on the loss.
    Repeated calls agree bit for bit."""
    torch = pytest.importorskip("torch")
    I, t = _batch(B, 40 + B)
    It, tt = torch.from_numpy(I).cuda(), torch.from_numpy(t).cuda()
    res = []
    for cc in (False, True):
        with api.Net(seed=13, max_batch=B, cuda_cores=cc) as net:
            L, g = net.gradients(It, tt)
            if not cc:
                L2, g2 = net.gradients(It, tt)
                assert L == L2 and np.array_equal(g, g2), "tensor-core gradients not deterministic"
            res.append((L, g))
    (Lt, gt), (Lc, gc) = res
    assert abs(Lt - Lc) / Lc < 2e-2
    errs = []
    for l, ((wo, bo), (ci, co, *_)) in enumerate(zip(orc_net.layout()[0], orc_net.LAYERS)):
        for kind, (a, b) in (("w", (wo, wo + co * ci * 9)), ("b", (bo, bo + co))):
            errs.append((l, kind, float(np.linalg.norm(gt[a:b] - gc[a:b]) / max(np.linalg.norm(gc[a:b]), 1e-30))))
    print(f"batch {B}: tensor-core vs CUDA-core gradients, worst", max(errs, key=lambda e: e[2]))
    assert all(e < 8e-2 for _, _, e in errs), errs

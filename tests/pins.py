"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each ``pin_*`` takes the oracle module as an argument and raises
AssertionError if the oracle disagrees with a definition, an identity, a
closed form or brute force.  ``test_oracle_pins.py`` runs them on the real
oracle; ``test_oracle_mutations.py`` plants plausible mistakes in a copy of
the oracle and checks that some pin catches each one.
"""
from __future__ import annotations

import cmath
import math
import os

import numpy as np
from scipy import optimize

from util import small_scan

RNG = np.random.default_rng(12345)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _crandn(*shape, rng=None):
    rng = rng or RNG
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _dft2_bruteforce(x: np.ndarray) -> np.ndarray:
    """X[ky,kx] = sum_{y,x} x[y,x] exp(-2 pi i (ky y + kx x)/M), by explicit sums."""
    M = x.shape[0]
    N = x.shape[1]
    X = np.zeros((M, N), dtype=complex)
    for ky in range(M):
        for kx in range(N):
            s = 0j
            for yy in range(M):
                for xx in range(N):
                    s += x[yy, xx] * cmath.exp(-2j * math.pi * (ky * yy / M + kx * xx / N))
            X[ky, kx] = s
    return X


# --------------------------------------------------------------------- FFT

def pin_fft_bruteforce(orc):
    for M in (2, 3, 4, 6, 8, 12):
        x = _crandn(M, M)
        X = orc.fft2(x)
        ref = _dft2_bruteforce(x)
        assert np.allclose(X, ref, atol=1e-12 * M * M, rtol=0), f"fft2 != DFT at M={M}"
        assert np.allclose(orc.ifft2(ref), x, atol=1e-12, rtol=0), f"ifft2 not the inverse at M={M}"


def pin_parseval(orc):
    for M in (4, 16, 64):
        x = _crandn(3, M, M)
        X = orc.fft2(x)
        assert abs(np.sum(np.abs(X) ** 2) - M * M * np.sum(np.abs(x) ** 2)) < 1e-9 * M * M * np.sum(np.abs(x) ** 2)
        assert np.allclose(orc.ifft2(orc.fft2(x)), x, atol=1e-12)


# ----------------------------------------------------------- forward model

def pin_forward_bruteforce(orc):
    """I_j(q) = sum_k |DFT(P_k O_j)|^2 with the zero frequency at (M/2, M/2),
    by explicit loops over a 4x4 probe, 8x8 object, 2 positions, 2 modes."""
    M, K = 4, 2
    P = _crandn(K, M, M)
    O = _crandn(8, 8)
    pos = np.array([[0, 1], [3, 4]])
    I = orc.far_field_intensity(O, P, pos)
    for j, (y, x) in enumerate(pos):
        ref = np.zeros((M, M))
        for k in range(K):
            ex = np.array([[P[k, u, v] * O[y + u, x + v] for v in range(M)] for u in range(M)])
            X = _dft2_bruteforce(ex)
            for ky in range(M):
                for kx in range(M):
                    ref[(ky + M // 2) % M, (kx + M // 2) % M] += abs(X[ky, kx]) ** 2
        assert np.allclose(I[j], ref, rtol=1e-12, atol=1e-12 * ref.max()), f"forward model frame {j}"


def pin_mode_mixing_invariance(orc):
    """Incoherent modes: a unitary mixing of the K modes leaves I unchanged."""
    P, O, pos = small_scan(M=8, K=3, grid=2, step=3)
    pos = orc.round_positions(pos)
    Q, _ = np.linalg.qr(_crandn(3, 3))
    Pm = np.einsum("kl,luv->kuv", Q, P)
    I1 = orc.far_field_intensity(O, P, pos)
    I2 = orc.far_field_intensity(O, Pm, pos)
    assert np.allclose(I1, I2, rtol=1e-10, atol=1e-10 * I1.max())


def pin_gather_scatter_adjoint(orc):
    """<S x, y> = <x, G y> for random complex patches and object."""
    M = 5
    pos = np.array([[0, 0], [2, 3], [4, 1], [2, 3]])
    shape = (9, 9)
    x = _crandn(len(pos), M, M)
    y = _crandn(*shape)
    lhs = np.vdot(orc.scatter_add(shape, pos, x), y)
    rhs = np.vdot(x, orc.gather(y, pos, M))
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    cover = orc.scatter_add(shape, pos, np.ones((len(pos), M, M)))
    ref = np.zeros(shape)
    for (py, px) in pos:
        for u in range(M):
            for v in range(M):
                ref[py + u, px + v] += 1
    assert np.array_equal(cover, ref)


def pin_rounding(orc):
    p = orc.round_positions(np.array([[2.5, 3.5], [0.4999, 1.5000001], [-0.5, 7.0]]))
    assert p.tolist() == [[2, 4], [0, 2], [0, 7]]


# -------------------------------------------------------------- projection

def pin_projection(orc):
    J, K, M = 3, 2, 8
    Psi = _crandn(J, K, M, M) * 3.0
    I = np.abs(RNG.standard_normal((J, M, M))) * 10.0
    I[0, 1, 2] = -1.0          # masked
    Psi[1, :, 3, 3] = 0.0       # A = 0 -> projected to 0
    Q = orc.project(Psi, I)
    A2 = np.sum(np.abs(Q) ** 2, axis=1)
    m = (I >= 0)
    m[1, 3, 3] = False
    assert np.allclose(np.sqrt(A2[m]), np.sqrt(I[m]), rtol=1e-12), "modulus != sqrt(I)"
    # phases and mode ratios unchanged where the modulus is positive
    nz = np.abs(Psi) > 0
    assert np.allclose(np.angle(Q[nz & np.broadcast_to(m[:, None], Q.shape)]),
                       np.angle(Psi[nz & np.broadcast_to(m[:, None], Q.shape)]), atol=1e-12)
    assert np.allclose(Q[0, :, 1, 2], Psi[0, :, 1, 2]), "masked pixel changed"
    assert np.all(Q[1, :, 3, 3] == 0)
    assert np.allclose(orc.project(Q, I), Q, rtol=1e-12, atol=1e-12), "projection not idempotent"


def pin_fourier_error(orc):
    P, O, pos = small_scan(M=16, K=2)
    pos = orc.round_positions(pos)
    I = orc.far_field_intensity(O, P, pos)
    assert orc.fourier_error(O, P, pos, I) < 1e-24
    c = 1.7
    E = orc.fourier_error(O, P, pos, c * c * I)
    assert abs(E - (1 - c) ** 2 / c ** 2) < 1e-12, "scaled data: E != (1-c)^2/c^2"
    Im = c * c * I.copy()
    Im[:, ::2, :] = -1.0        # mask half the rows: the ratio is unchanged
    assert abs(orc.fourier_error(O, P, pos, Im) - (1 - c) ** 2 / c ** 2) < 1e-12


# ------------------------------------------------------------ fixed points

def _truth_case(orc, K=2):
    P, O, pos = small_scan(M=16, K=K)
    pos = orc.round_positions(pos)
    I = orc.far_field_intensity(O, P, pos)
    return P, O, pos, I


def pin_fixed_points(orc):
    P, O, pos, I = _truth_case(orc)
    O1, P1 = orc.epie_iteration(O, P, pos, I, t=0, seed=5)
    assert np.allclose(O1, O, atol=1e-12) and np.allclose(P1, P, atol=1e-12), "ePIE moved off the truth"
    psi = orc.dm_init(O, P, pos)
    O2, P2, psi2 = orc.dm_iteration(O, P, psi, pos, I, t=0)
    assert np.allclose(O2, O, atol=1e-12) and np.allclose(P2, P, atol=1e-12), "DM moved O/P off the truth"
    assert np.allclose(psi2, psi, atol=1e-12), "DM moved psi off the truth"
    O3, P3 = orc.lsqml_iteration(O, P, pos, I, t=0)
    assert np.allclose(O3, O, atol=1e-12) and np.allclose(P3, P, atol=1e-12), "LSQML moved off the truth"


def _er_step(patch, I_centred):
    """Error-reduction step written with polar form: keep the phase, impose sqrt(I)."""
    F = np.fft.fft2(patch)
    amp = np.sqrt(np.fft.ifftshift(I_centred))
    return np.fft.ifft2(amp * np.exp(1j * np.angle(F)))


def pin_epie_er_special_case(orc):
    """J=1, K=1, P = 1, alpha = 1, probe fixed: the patch becomes F^-1 Pi F(patch)."""
    M = 8
    O = _crandn(12, 12)
    P = np.ones((1, M, M), dtype=complex)
    pos = np.array([[2, 3]])
    I = np.abs(_crandn(1, M, M)) ** 2
    O1, P1 = orc.epie_iteration(O, P, pos, I, t=0, probe_start=10)
    ref = O.copy()
    ref[2:10, 3:11] = _er_step(O[2:10, 3:11], I[0])
    assert np.allclose(O1, ref, atol=1e-12), "ePIE object step != error reduction"
    assert np.array_equal(P1, P)
    # symmetric case for the probe: O = 1 on the patch, probe updated
    O = np.ones((12, 12), dtype=complex)
    Pr = _crandn(1, M, M)
    O2, P2 = orc.epie_iteration(O, Pr, pos, I, t=0, probe_start=0)
    assert np.allclose(P2[0], _er_step(Pr[0], I[0]), atol=1e-12), "ePIE probe step != error reduction"


def pin_epie_gradient(orc):
    """The ePIE object/probe corrections are steepest-descent steps of
    f = 1/2 sum_k ||z_k - P_k O_j||^2 (z fixed) with steps alpha/max|P|^2, beta/max|O_j|^2."""
    M, K = 6, 2
    O = _crandn(8, 8)
    P = _crandn(K, M, M)
    pos = np.array([[1, 2]])
    I = np.abs(_crandn(1, M, M)) ** 2
    alpha, beta = 0.7, 0.3
    O1, P1 = orc.epie_iteration(O, P, pos, I, t=0, alpha=alpha, beta=beta)
    Oj = O[1:7, 2:8]
    # target exit waves: the mode-summed modulus replaced by sqrt(I), phases and mode ratios kept
    F = np.fft.fft2(P * Oj)
    A = np.sqrt(np.sum(np.abs(F) ** 2, axis=0))
    z = np.fft.ifft2(F * np.fft.ifftshift(np.sqrt(I[0]))[None] / A[None])

    def f(Ov, Pv):
        return 0.5 * np.sum(np.abs(z - Pv * Ov[None]) ** 2)

    h = 1e-6
    gO = np.zeros_like(Oj)
    for u in range(M):
        for v in range(M):
            e = np.zeros_like(Oj)
            e[u, v] = h
            gr = (f(Oj + e, P) - f(Oj - e, P)) / (2 * h)
            gi = (f(Oj + 1j * e, P) - f(Oj - 1j * e, P)) / (2 * h)
            gO[u, v] = gr + 1j * gi
    pmax = np.max(np.sum(np.abs(P) ** 2, axis=0))
    assert np.allclose(O1[1:7, 2:8] - Oj, -alpha / pmax * gO, atol=1e-6), "ePIE object step direction"
    gP = np.zeros_like(P)
    for k in range(K):
        for u in range(M):
            for v in range(M):
                e = np.zeros_like(P)
                e[k, u, v] = h
                gr = (f(Oj, P + e) - f(Oj, P - e)) / (2 * h)
                gi = (f(Oj, P + 1j * e) - f(Oj, P - 1j * e)) / (2 * h)
                gP[k, u, v] = gr + 1j * gi
    omax = np.max(np.abs(Oj) ** 2)
    assert np.allclose(P1 - P, -beta / omax * gP, atol=1e-6), "ePIE probe step direction"


def pin_epie_order(orc):
    golden = [l for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if not l.startswith("#")]
    g = orc.splitmix64_stream(0)
    assert next(g) == int(golden[0], 16), "SplitMix64 seed-0 test vector"
    assert orc.epie_order(0, 3, 7).tolist() == list(range(7))
    for t in range(4):
        o = orc.epie_order(99, t, 50)
        assert sorted(o.tolist()) == list(range(50))
    assert orc.epie_order(99, 0, 50).tolist() != orc.epie_order(99, 1, 50).tolist()


# --------------------------------------------------------------------- DM

def _ls_directional_derivative(g, X, rng):
    """Max over a few random directions of |dg/ds| at s = 0 (central differences)."""
    h = 1e-6
    worst = 0.0
    for _ in range(4):
        eta = _crandn(*X.shape, rng=rng)
        d = (g(X + h * eta) - g(X - h * eta)) / (2 * h)
        worst = max(worst, abs(d))
    return worst


def pin_dm_overlap_least_squares(orc):
    """O_new minimises sum ||psi - P O_j||^2 + d_O ||O - O_old||^2; then P_new minimises
    sum ||psi - P O_new,j||^2 + d_P ||P - P_old||^2 (d = reg max den, den by brute force)."""
    rng = np.random.default_rng(7)
    P, O, pos = small_scan(M=8, K=2, grid=3, step=3)
    pos = orc.round_positions(pos)
    psi = _crandn(len(pos), 2, 8, 8, rng=rng)
    reg = 0.05
    On, Pn = orc.dm_overlap_update(O, P, psi, pos, reg, True)
    M = 8
    denO = np.zeros(O.shape)
    for (y, x) in pos:
        denO[y:y + M, x:x + M] += np.sum(np.abs(P) ** 2, axis=0)
    dO = reg * denO.max()

    def gO(Ov):
        s = sum(np.sum(np.abs(psi[j] - P * Ov[y:y + M, x:x + M][None]) ** 2) for j, (y, x) in enumerate(pos))
        return s + dO * np.sum(np.abs(Ov - O) ** 2)

    base = _ls_directional_derivative(gO, O, rng)
    assert _ls_directional_derivative(gO, On, rng) < 1e-6 * base, "DM object update not the LS minimiser"
    denP = sum(np.abs(On[y:y + M, x:x + M]) ** 2 for (y, x) in pos)
    dP = reg * denP.max()

    def gP(Pv):
        s = sum(np.sum(np.abs(psi[j] - Pv * On[y:y + M, x:x + M][None]) ** 2) for j, (y, x) in enumerate(pos))
        return s + dP * np.sum(np.abs(Pv - P) ** 2)

    base = _ls_directional_derivative(gP, P, rng)
    assert _ls_directional_derivative(gP, Pn, rng) < 1e-6 * base, "DM probe update not the LS minimiser"


def pin_dm_all_masked(orc):
    """With every detector pixel masked the Fourier constraint is the identity,
    so one DM iteration returns the overlap projection: psi_new = P_new O_new,j."""
    rng = np.random.default_rng(3)
    P, O, pos = small_scan(M=8, K=2, grid=3, step=3)
    pos = orc.round_positions(pos)
    psi = _crandn(len(pos), 2, 8, 8, rng=rng)
    I = -np.ones((len(pos), 8, 8))
    On, Pn, psin = orc.dm_iteration(O, P, psi, pos, I, t=0, reg=0.01)
    assert np.allclose(psin, orc.exit_waves(On, Pn, pos), atol=1e-12), "DM with identity Fourier step"


# ------------------------------------------------------------------ LSQML

def pin_lsqml_step_sizes(orc):
    """alpha_j minimises ||chi_j - aO a_j - aP b_j||^2 + lam (aO^2 + aP^2), found by BFGS."""
    rng = np.random.default_rng(5)
    P, O, pos = small_scan(M=8, K=2, grid=2, step=4)
    pos = orc.round_positions(pos)
    J = len(pos)
    chi = _crandn(J, 2, 8, 8, rng=rng)
    dO = _crandn(*O.shape, rng=rng)
    dP = _crandn(2, 8, 8, rng=rng)
    aO, aP = orc.lsqml_step_sizes(O, P, chi, pos, dO, dP)
    for j, (y, x) in enumerate(pos):
        a = P * dO[y:y + 8, x:x + 8][None]
        b = O[y:y + 8, x:x + 8][None] * dP
        lam = 1e-6 * (np.sum(np.abs(a) ** 2) + np.sum(np.abs(b) ** 2)) / 2

        def q(v):
            return np.sum(np.abs(chi[j] - v[0] * a - v[1] * b) ** 2) + lam * (v[0] ** 2 + v[1] ** 2)

        res = optimize.minimize(q, np.zeros(2), method="BFGS", options=dict(gtol=1e-12))
        assert np.allclose([aO[j], aP[j]], res.x, rtol=1e-5, atol=1e-7), f"step sizes of position {j}"


def pin_lsqml_er_special_case(orc):
    """J=1, K=1, P = 1, probe fixed, beta = 1: the patch moves to the error-reduction
    step up to the lambda and reg terms (relative 1e-6)."""
    M = 8
    O = _crandn(12, 12)
    P = np.ones((1, M, M), dtype=complex)
    pos = np.array([[2, 3]])
    I = np.abs(_crandn(1, M, M)) ** 2
    O1, P1 = orc.lsqml_iteration(O, P, pos, I, t=0, beta=1.0, probe_start=5)
    ref = O.copy()
    ref[2:10, 3:11] = _er_step(O[2:10, 3:11], I[0])
    assert np.allclose(O1, ref, rtol=0, atol=2e-6 * np.abs(ref).max()), "LSQML with P = 1 != error reduction"
    assert np.array_equal(P1, P)


def pin_lsqml_all_masked(orc):
    P, O, pos = small_scan(M=8, K=2, grid=3, step=3)
    pos = orc.round_positions(pos)
    I = -np.ones((len(pos), 8, 8))
    O1, P1 = orc.lsqml_iteration(O, P, pos, I, t=0)
    assert np.allclose(O1, O, atol=1e-14) and np.allclose(P1, P, atol=1e-14)


def pin_lsqml_directions(orc):
    """dO and dP are steepest-descent directions of 1/2 sum ||chi - delta(P O_j)||^2 at zero
    change, scaled by the denominators: dO * wO = -grad_O, dP * wP = -grad_P."""
    rng = np.random.default_rng(9)
    M = 6
    P, O, pos = small_scan(M=M, K=2, grid=2, step=3)
    pos = orc.round_positions(pos)
    chi = _crandn(len(pos), 2, M, M, rng=rng)
    dO, dP, wO, wP = orc.lsqml_directions(O, P, chi, pos, 1e-3, True)

    def f(Ov, Pv):
        return 0.5 * sum(np.sum(np.abs(chi[j] + P * O[y:y + M, x:x + M][None] - Pv * Ov[y:y + M, x:x + M][None]) ** 2)
                         for j, (y, x) in enumerate(pos))

    h = 1e-6
    # object gradient on a few pixels
    for (u, v) in [(pos[0][0] + 1, pos[0][1] + 2), (pos[-1][0] + 3, pos[-1][1] + 3)]:
        e = np.zeros_like(O)
        e[u, v] = h
        g = ((f(O + e, P) - f(O - e, P)) + 1j * (f(O + 1j * e, P) - f(O - 1j * e, P))) / (2 * h)
        assert abs(dO[u, v] * wO[u, v] + g) < 1e-6 * (1 + abs(g)), "LSQML object direction"
    for (k, u, v) in [(0, 1, 1), (1, 4, 2)]:
        e = np.zeros_like(P)
        e[k, u, v] = h
        g = ((f(O, P + e) - f(O, P - e)) + 1j * (f(O, P + 1j * e) - f(O, P - 1j * e))) / (2 * h)
        assert abs(dP[k, u, v] * wP[u, v] + g) < 1e-6 * (1 + abs(g)), "LSQML probe direction"


def pin_poisson_newton_step(orc):
    """Per pixel, the Poisson correction is one Newton step of the pixel's
    negative log-likelihood l(s) = a(s) - I log a(s), a(s) = (1 + s)^2 A^2,
    along its steepest-descent direction: with s* = -l'(0) / l''(0) from
    central differences of l, correction = s* Psi_k (sum over modes in A^2);
    and s* has the sign of -dl/ds (a descent step).  Masked pixels: none."""
    rng = np.random.default_rng(12)
    M, K = 4, 2
    Psi = _crandn(2, K, M, M, rng=rng)
    I = rng.poisson(3.0 * np.sum(np.abs(Psi) ** 2, axis=1) * rng.uniform(0.2, 5.0, (2, M, M))).astype(float)
    I[0, 1, 2] = -1.0  # masked
    I[1, 0, 0] = 0.0   # zero counts
    corr = orc.poisson_correction(Psi, I)
    h = 1e-4
    for (j, u, v) in [(0, 0, 0), (0, 1, 2), (0, 3, 1), (1, 0, 0), (1, 2, 3)]:
        A2 = float(np.sum(np.abs(Psi[j, :, u, v]) ** 2))
        if I[j, u, v] < 0:
            assert np.allclose(corr[j, :, u, v], 0.0)
            continue
        l = lambda s_: (1 + s_) ** 2 * A2 - I[j, u, v] * np.log((1 + s_) ** 2 * A2)
        d1 = (l(h) - l(-h)) / (2 * h)
        d2 = (l(h) - 2 * l(0.0) + l(-h)) / h ** 2
        s_star = -d1 / d2
        assert np.allclose(corr[j, :, u, v], s_star * Psi[j, :, u, v], rtol=1e-6, atol=1e-9), "Poisson Newton step"
        assert s_star * d1 <= 0.0
    assert np.allclose(orc.poisson_correction(Psi, -np.ones_like(I)), 0.0)


def pin_lsqml_poisson(orc):
    """Poisson LSQML: the object direction is a descent direction of the
    Poisson negative log-likelihood (directional derivative from central
    differences of :func:`poisson_nll` is negative), and noise-free data is a
    fixed point."""
    M = 6
    P, O, pos = small_scan(M=M, K=2, grid=2, step=3)
    pos = orc.round_positions(pos)
    rng = np.random.default_rng(4)
    I = orc.far_field_intensity(O * (1 + 0.1 * _crandn(*O.shape, rng=rng)), P, pos)
    I[0, 2, 2] = -1.0
    chi = orc.fourier_residual(O, P, pos, I, likelihood="poisson")
    dO, _, _, _ = orc.lsqml_directions(O, P, chi, pos, 1e-3, False)
    h = 1e-7
    f = lambda Ov: orc.poisson_nll(Ov, P, pos, I)
    slope = (f(O + h * dO) - f(O - h * dO)) / (2 * h)
    assert slope < 0.0, "Poisson LSQML object direction is not a descent direction"
    P0, O0, pos0, I0 = _truth_case(orc)
    O1, P1 = orc.lsqml_iteration(O0, P0, pos0, I0, t=0, likelihood="poisson")
    assert np.allclose(O1, O0, atol=1e-12) and np.allclose(P1, P0, atol=1e-12), "Poisson LSQML moved off the truth"


def pin_mode_orthogonalisation(orc):
    """Orthogonalised modes: mutually orthogonal, powers decreasing, the
    largest power equal to the maximum of ||sum_l c_l P_l||^2 over unit
    vectors c (checked against random unit vectors, never exceeded and
    attained by the first mode), the sum of powers unchanged, every
    diffraction pattern unchanged, idempotent, and the phase convention
    (largest entry of each column of V real positive) met."""
    rng = np.random.default_rng(17)
    M, K = 8, 3
    P = _crandn(K, M, M, rng=rng) * np.array([3.0, 1.5, 1.0])[:, None, None]
    Q, V = orc.orthogonalize_modes(P)
    flat = Q.reshape(K, -1)
    G = np.conj(flat) @ flat.T
    pw = np.real(np.diag(G))
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 1e-10 * pw.max(), "modes not orthogonal"
    assert np.all(np.diff(pw) < 0), "powers not decreasing"
    assert abs(pw.sum() - np.sum(np.abs(P) ** 2)) < 1e-10 * pw.sum()
    c = _crandn(4000, K, rng=rng)
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    comb = np.einsum("nk,kxy->nxy", c, P)
    best = np.max(np.sum(np.abs(comb) ** 2, axis=(1, 2)))
    assert best <= pw[0] * (1 + 1e-12) and best > 0.9 * pw[0]
    assert np.allclose(np.sum(np.abs(Q) ** 2, axis=0), np.sum(np.abs(P) ** 2, axis=0), atol=1e-10)
    O = 1.0 + 0.3 * _crandn(12, 12, rng=rng)
    pos = np.array([[0, 0], [2, 3], [4, 1]])
    assert np.allclose(orc.far_field_intensity(O, Q, pos), orc.far_field_intensity(O, P, pos), rtol=1e-10)
    Q2, V2 = orc.orthogonalize_modes(Q)
    assert np.allclose(Q2, Q, atol=1e-10) and np.allclose(V2, np.eye(K), atol=1e-10), "not idempotent"
    for m in range(K):
        i = int(np.argmax(np.abs(V[:, m])))
        assert abs(V[i, m].imag) < 1e-12 and V[i, m].real > 0


def pin_dm_mode_orthogonalisation_keeps_truth(orc):
    """DM with orthogonalisation on noise-free data whose true modes are a
    non-orthogonal mixture: the object stays at the truth and every
    diffraction pattern and the per-pixel mode power stay fixed (the exit
    waves are mixed with the probe)."""
    rng = np.random.default_rng(23)
    P, O, pos = small_scan(M=16, K=2, grid=3, step=6)
    pos = orc.round_positions(pos)
    U, _ = np.linalg.qr(_crandn(2, 2, rng=rng))
    Pm = orc.mix_modes(P, U) * np.array([1.0, 1.0])[:, None, None]
    Pm[1] += 0.3 * Pm[0]  # no longer orthogonal
    I = orc.far_field_intensity(O, Pm, pos)
    O1, P1, psi1 = orc.reconstruct("dm", O, Pm, pos, I, 3, probe_ortho=True)
    assert np.allclose(O1, O, atol=1e-9), "DM with orthogonalisation moved the object"
    assert np.allclose(orc.far_field_intensity(O1, P1, pos), I, rtol=1e-8)
    assert np.allclose(np.sum(np.abs(P1) ** 2, axis=0), np.sum(np.abs(Pm) ** 2, axis=0), atol=1e-9)


def pin_preprocess(orc):
    """Detector preprocessing: a plain crop around the centre (identity for a
    centred M x M frame), a quarter turn moves the pixel right of the zero
    frequency to the one above it, two turns are the point reflection about
    the zero frequency on the periodic grid, four are the identity; pixels
    outside the raw frame, negative ones and saturated ones (>= 2^bits - 1)
    are masked; values below the threshold become 0."""
    rng = np.random.default_rng(5)
    M, h = 8, 4
    raw = rng.uniform(1.0, 100.0, (2, M, M))
    assert np.array_equal(orc.preprocess_frames(raw, (h, h), M), raw)
    assert np.array_equal(orc.preprocess_frames(raw, (h, h), M, rot90=4), raw)
    y, x = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    assert np.array_equal(orc.preprocess_frames(raw, (h, h), M, rot90=2), raw[:, (2 * h - y) % M, (2 * h - x) % M])
    spot = np.zeros((1, M, M))
    spot[0, h, h + 1] = 7.0
    q = orc.preprocess_frames(spot, (h, h), M, rot90=1)
    assert q[0, h - 1, h] == 7.0 and np.count_nonzero(q) == 1, "quarter turn direction"
    big = rng.uniform(1.0, 100.0, (1, 20, 24))
    c = orc.preprocess_frames(big, (9.0, 13.0), M)
    assert np.array_equal(c, big[:, 9 - h:9 + h, 13 - h:13 + h])
    edge = orc.preprocess_frames(big, (2.0, 22.0), M)
    assert np.all(edge[0, :2, :] == -1.0) and np.all(edge[0, :, -2:] == -1.0) and np.all(edge[0, 2:, :-2] > 0)
    sat = raw.copy()
    sat[0, 1, 1] = 4095.0
    sat[0, 2, 2] = 4094.0
    sat[1, 3, 3] = -5.0
    p_ = orc.preprocess_frames(sat, (h, h), M, saturation_bits=12, threshold=10.0)
    assert p_[0, 1, 1] == -1.0 and p_[0, 2, 2] == 4094.0 and p_[1, 3, 3] == -1.0
    low = (sat >= 0) & (sat < 10.0)
    assert np.all(p_[low] == 0.0) and np.all(p_[(sat >= 10.0) & (sat < 4095)] == sat[(sat >= 10.0) & (sat < 4095)])



# ------------------------------------------------------- sub-pixel positions

def pin_subpixel_positions(orc):
    """Quantisation to 1/S pixel and the split into corner + shift in
    [-1/2, 1/2), on hand-worked values (S = 8 unless stated)."""
    raw = np.array([[10.3, -0.3], [10.5, 3.0625], [10.45, 3.1875], [7.0, 6.9375]])
    p, d = orc.subpixel_positions(raw, 8)
    # 10.3 -> q 82 -> (10, +1/4); -0.3 -> q -2 -> (0, -1/4); 10.5 -> q 84 -> (11, -1/2);
    # 3.0625 -> 24.5 -> q 24 (half to even) -> (3, 0); 10.45 -> 83.6 -> q 84 -> (11, -1/2);
    # 3.1875 -> 25.5 -> q 26 -> (3, +1/4); 7 -> (7, 0); 6.9375 -> 55.5 -> q 56 -> (7, 0)
    assert p.tolist() == [[10, 0], [11, 3], [11, 3], [7, 7]]
    assert d.tolist() == [[0.25, -0.25], [-0.5, 0.0], [-0.5, 0.25], [0.0, 0.0]]
    p2, d2 = orc.subpixel_positions(np.array([[1.25, 1.75]]), 2)   # q = 2 (half to even), 4
    assert p2.tolist() == [[1, 2]] and d2.tolist() == [[0.0, 0.0]]
    rng = np.random.default_rng(21)
    for S in (2, 4, 16):
        r = rng.uniform(0, 50, (40, 2))
        p, d = orc.subpixel_positions(r, S)
        assert ((d >= -0.5) & (d < 0.5)).all()
        assert np.all(np.abs(p + d - r) <= 0.5 / S + 1e-12)


def _bandlimited(rng, M, nmax, n_terms=5):
    """Coefficients and frequencies of a sum of complex exponentials
    exp(2 pi i (ny y + nx x) / M) with |ny|, |nx| <= nmax."""
    freqs = rng.integers(-nmax, nmax + 1, (n_terms, 2))
    coef = _crandn(n_terms, rng=rng)
    return coef, freqs


def _eval_bandlimited(coef, freqs, M, y, x):
    return sum(c * np.exp(2j * np.pi * (fy * y + fx * x) / M) for c, (fy, fx) in zip(coef, freqs))


def pin_fourier_shift(orc):
    """T_delta: integer shifts are circular shifts (np.roll), a band-limited
    periodic function is translated exactly ((T f)(u) = f(u - delta), by
    direct evaluation), T_a T_b = T_(a+b), and T_-delta is the adjoint."""
    rng = np.random.default_rng(22)
    M = 12
    X = _crandn(2, M, M, rng=rng)
    for dy, dx in [(1, 0), (0, 1), (-2, 3)]:
        assert np.allclose(orc.shift_probe(X, dy, dx), np.roll(X, (dy, dx), axis=(-2, -1)), atol=1e-12)
    coef, freqs = _bandlimited(rng, M, M // 2 - 1)
    yy, xx = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    f = _eval_bandlimited(coef, freqs, M, yy, xx)
    for dy, dx in [(0.25, -0.5), (-0.375, 0.125), (0.4, 0.3)]:
        ref = _eval_bandlimited(coef, freqs, M, yy - dy, xx - dx)
        assert np.allclose(orc.shift_probe(f, dy, dx), ref, atol=1e-11 * np.abs(ref).max()), "band-limited translation"
    a = orc.shift_probe(orc.shift_probe(X, 0.25, -0.125), -0.5, 0.375)
    assert np.allclose(a, orc.shift_probe(X, -0.25, 0.25), atol=1e-12)
    Y = _crandn(2, M, M, rng=rng)
    lhs = np.vdot(orc.shift_probe(X, 0.3, -0.2), Y)
    rhs = np.vdot(X, orc.shift_probe(Y, -0.3, 0.2))
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def pin_subpixel_forward(orc):
    """A probe and an M-periodic object, both band-limited so that their
    product has no frequency at or beyond M/2: the pattern of the probe at the
    sub-pixel position y equals, by translation invariance of |F|, the pattern
    of the unshifted probe over the object evaluated at y + u (direct
    evaluation of the object's exponentials at non-integer points), with a
    brute-force DFT."""
    rng = np.random.default_rng(23)
    M, K, S = 8, 2, 8
    pc = [_bandlimited(rng, M, 1, 4) for _ in range(K)]
    oc, of = _bandlimited(rng, M, 1, 5)
    yy, xx = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    P = np.stack([_eval_bandlimited(c, f, M, yy, xx) for c, f in pc])
    ny = nx = 20
    gy, gx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    O = _eval_bandlimited(oc, of, M, gy, gx)
    raw = np.array([[2.25, 3.625], [5.5, 1.875], [9.0, 10.125]])   # on the 1/8 grid
    pos, delta = orc.subpixel_positions(raw, S)
    I = orc.far_field_intensity(O, P, pos, delta)
    for j, (y, x) in enumerate(raw):
        ref = np.zeros((M, M))
        Oj = _eval_bandlimited(oc, of, M, y + yy, x + xx)
        for k in range(K):
            X = _dft2_bruteforce(P[k] * Oj)
            ref += np.abs(np.fft.fftshift(X)) ** 2
        assert np.allclose(I[j], ref, rtol=1e-10, atol=1e-10 * ref.max()), f"sub-pixel pattern {j}"


def _subpixel_case(orc, M=8, K=2, S=8, seed=24):
    rng = np.random.default_rng(seed)
    P, O, pos = small_scan(M=M, K=K, grid=2, step=3)
    raw = pos + rng.uniform(-0.5, 0.5, pos.shape)
    raw = np.clip(raw, 0.0, None)
    p, d = orc.subpixel_positions(raw, S)
    assert (p >= 0).all() and (p + M <= np.array(O.shape)).all()
    return P, O, raw, p, d, rng


def pin_subpixel_gradients(orc):
    """Sub-pixel LSQML directions are the scaled steepest-descent directions of
    1/2 sum_j ||chi_j - delta((T_j P) O_j)||^2 (central differences), den_O is
    sum_j S_j[sum_k |T_j P_k|^2] by explicit loops, and the DM object update
    minimises sum ||psi - (T_j P) O_j||^2 + d_O ||O - O_old||^2."""
    P, O, raw, pos, delta, rng = _subpixel_case(orc)
    M = P.shape[-1]
    J = len(pos)
    Pj = [orc.shift_probe(P, dy, dx) for dy, dx in delta]
    chi = _crandn(J, 2, M, M, rng=rng)
    dO, dP, wO, wP = orc.lsqml_directions(O, P, chi, pos, 1e-3, True, delta)
    den = np.zeros(O.shape)
    for j, (y, x) in enumerate(pos):
        den[y:y + M, x:x + M] += np.sum(np.abs(Pj[j]) ** 2, axis=0)
    assert np.allclose(wO, den + 1e-3 * den.max(), rtol=1e-12), "sub-pixel den_O"

    def f(Ov, Pv):
        return 0.5 * sum(np.sum(np.abs(chi[j] + Pj[j] * O[y:y + M, x:x + M][None]
                                       - orc.shift_probe(Pv, *delta[j]) * Ov[y:y + M, x:x + M][None]) ** 2)
                         for j, (y, x) in enumerate(pos))

    h = 1e-6
    for (u, v) in [(pos[0][0] + 1, pos[0][1] + 2), (pos[-1][0] + 3, pos[-1][1] + 3)]:
        e = np.zeros_like(O)
        e[u, v] = h
        g = ((f(O + e, P) - f(O - e, P)) + 1j * (f(O + 1j * e, P) - f(O - 1j * e, P))) / (2 * h)
        assert abs(dO[u, v] * wO[u, v] + g) < 1e-6 * (1 + abs(g)), "sub-pixel object direction"
    for (k, u, v) in [(0, 1, 1), (1, 4, 2), (0, 7, 6)]:
        e = np.zeros_like(P)
        e[k, u, v] = h
        g = ((f(O, P + e) - f(O, P - e)) + 1j * (f(O, P + 1j * e) - f(O, P - 1j * e))) / (2 * h)
        assert abs(dP[k, u, v] * wP[u, v] + g) < 1e-6 * (1 + abs(g)), "sub-pixel probe direction"
    psi = _crandn(J, 2, M, M, rng=rng)
    reg = 0.05
    On, _ = orc.dm_overlap_update(O, P, psi, pos, reg, False, delta)
    dreg = reg * den.max()

    def gO(Ov):
        s = sum(np.sum(np.abs(psi[j] - Pj[j] * Ov[y:y + M, x:x + M][None]) ** 2) for j, (y, x) in enumerate(pos))
        return s + dreg * np.sum(np.abs(Ov - O) ** 2)

    base = _ls_directional_derivative(gO, O, rng)
    assert _ls_directional_derivative(gO, On, rng) < 1e-6 * base, "sub-pixel DM object update not the LS minimiser"


def pin_subpixel_dm_probe_solve(orc):
    """The sub-pixel DM probe update: run to convergence (60 conjugate-gradient
    iterations) it minimises sum ||psi_j - (T_j P) O_j||^2 + d_P ||P - P_old||^2
    (central differences along random directions, the shift from explicit
    loops over positions); the normal operator is Hermitian positive; the
    default iteration count already leaves a smaller normal-equation residual
    than the diagonal (unshifted-denominator) update."""
    P, O, raw, pos, delta, rng = _subpixel_case(orc, seed=27)
    M = P.shape[-1]
    J = len(pos)
    psi = _crandn(J, 2, M, M, rng=rng)
    reg = 0.05
    den = sum(np.abs(O[y:y + M, x:x + M]) ** 2 for (y, x) in pos)
    d = reg * den.max()

    def g(Pv):
        s = sum(np.sum(np.abs(psi[j] - orc.shift_probe(Pv, *delta[j]) * O[y:y + M, x:x + M][None]) ** 2)
                for j, (y, x) in enumerate(pos))
        return s + d * np.sum(np.abs(Pv - P) ** 2)

    Pn = orc.dm_probe_solve(O, P, psi, pos, reg, delta, n_cg=60)
    base = _ls_directional_derivative(g, P, rng)
    assert _ls_directional_derivative(g, Pn, rng) < 1e-6 * base, "sub-pixel DM probe solve not the LS minimiser"
    X, Y = _crandn(2, M, M, rng=rng), _crandn(2, M, M, rng=rng)
    BX, BY = orc.probe_normal_operator(O, pos, delta, X), orc.probe_normal_operator(O, pos, delta, Y)
    assert abs(np.vdot(Y, BX) - np.vdot(BY, X)) < 1e-12 * abs(np.vdot(Y, BX)) and np.vdot(X, BX).real > 0

    def residual(Pv):
        rhs = sum(orc.shift_probe(np.conj(O[y:y + M, x:x + M])[None] * psi[j], -delta[j][0], -delta[j][1])
                  for j, (y, x) in enumerate(pos)) + d * P
        return np.linalg.norm(orc.probe_normal_operator(O, pos, delta, Pv) + d * Pv - rhs)

    num = sum(orc.shift_probe(np.conj(O[y:y + M, x:x + M])[None] * psi[j], -delta[j][0], -delta[j][1])
              for j, (y, x) in enumerate(pos))
    diag = (num + d * P) / (den + d)[None]
    assert residual(orc.dm_probe_solve(O, P, psi, pos, reg, delta)) < residual(diag)
    # n conjugate-gradient steps = the A-norm-optimal point of the real Krylov
    # space P + span{z0, (W^-1 A) z0, ...} (Hestenes & Stiefel), found here by
    # a Galerkin solve over an explicit basis; A = B + d, W = den + d
    A = lambda V: orc.probe_normal_operator(O, pos, delta, V) + d * V
    r0 = num + d * P - A(P)
    basis = [r0 / (den + d)[None]]
    for n in (1, 2, 3):
        V = basis[:n]
        G = np.array([[np.real(np.vdot(a, A(b))) for b in V] for a in V])
        y = np.linalg.solve(G, np.array([np.real(np.vdot(a, r0)) for a in V]))
        ref = P + sum(c * v for c, v in zip(y, V))
        got = orc.dm_probe_solve(O, P, psi, pos, reg, delta, n_cg=n)
        assert np.linalg.norm(got - ref) < 1e-8 * np.linalg.norm(ref), f"CG step {n} is not Krylov-optimal"
        basis.append(A(basis[-1]) / (den + d)[None])


def pin_subpixel_step_sizes(orc):
    """Sub-pixel step sizes minimise ||chi_j - aO a_j - aP b_j||^2 + lam |alpha|^2
    with a_j = (T_j P) dO_j and b_j = O_j (T_j dP) (BFGS)."""
    P, O, raw, pos, delta, rng = _subpixel_case(orc, seed=25)
    M = P.shape[-1]
    J = len(pos)
    chi = _crandn(J, 2, M, M, rng=rng)
    dO = _crandn(*O.shape, rng=rng)
    dP = _crandn(2, M, M, rng=rng)
    aO, aP = orc.lsqml_step_sizes(O, P, chi, pos, dO, dP, delta)
    for j, (y, x) in enumerate(pos):
        a = orc.shift_probe(P, *delta[j]) * dO[y:y + M, x:x + M][None]
        b = O[y:y + M, x:x + M][None] * orc.shift_probe(dP, *delta[j])
        lam = 1e-6 * (np.sum(np.abs(a) ** 2) + np.sum(np.abs(b) ** 2)) / 2

        def q(v):
            return np.sum(np.abs(chi[j] - v[0] * a - v[1] * b) ** 2) + lam * (v[0] ** 2 + v[1] ** 2)

        res = optimize.minimize(q, np.zeros(2), method="BFGS", options=dict(gtol=1e-12))
        assert np.allclose([aO[j], aP[j]], res.x, rtol=1e-5, atol=1e-7), f"sub-pixel step sizes of position {j}"


def pin_subpixel_fixed_point_and_reduction(orc):
    """Noise-free data simulated at sub-pixel positions is a fixed point of
    sub-pixel LSQML, and of DM while the probe is fixed (the object update is
    then exact least squares and psi = (T_j P) O_j is unchanged); positions
    that fall on integers give exactly the integer path (the shift by zero is
    the identity)."""
    P, O, raw, pos, delta, rng = _subpixel_case(orc, M=16, seed=26)
    I = orc.far_field_intensity(O, P, pos, delta)
    O1, P1, _ = orc.reconstruct("lsqml", O, P, raw, I, 1, subpixel=8)
    assert np.allclose(O1, O, atol=1e-12) and np.allclose(P1, P, atol=1e-12), "sub-pixel LSQML moved off the truth"
    psi = orc.dm_init(O, P, pos, delta)
    O2, P2, psi2 = orc.reconstruct("dm", O, P, raw, I, 1, psi=psi, probe_start=5, subpixel=8)
    assert np.allclose(O2, O, atol=1e-12) and np.allclose(psi2, psi, atol=1e-12), "sub-pixel DM moved off the truth"
    O3, P3, psi3 = orc.reconstruct("dm", O, P, raw, I, 1, psi=psi, subpixel=8)
    assert np.allclose(O3, O, atol=1e-12) and np.allclose(P3, P, atol=1e-12) and np.allclose(psi3, psi, atol=1e-12), \
        "sub-pixel DM (probe updated) moved off the truth"
    O4, P4, _ = orc.reconstruct("epie", O, P, raw, I, 1, seed=3, subpixel=8)
    assert np.allclose(O4, O, atol=1e-12) and np.allclose(P4, P, atol=1e-12), "sub-pixel ePIE moved off the truth"
    ip = pos.astype(float)
    I2 = orc.far_field_intensity(O, P, pos)
    O0 = np.ones_like(O)
    for alg in ("dm", "lsqml"):
        a = orc.reconstruct(alg, O0, P * 1.1, ip, I2, 2, subpixel=8)
        b = orc.reconstruct(alg, O0, P * 1.1, ip, I2, 2)
        assert np.allclose(a[0], b[0], atol=1e-12) and np.allclose(a[1], b[1], atol=1e-12), f"{alg}: zero shift"


def pin_position_refinement(orc):
    """Position correction: the object gradient is the central difference by
    explicit loops; the shift s_j minimises ||chi_j - s_y a_y - s_x a_x||^2 +
    lam |s|^2 (BFGS); s_y a_y + s_x a_x is the first-order change of the
    far-field intensity when the object moves by s under the probe (Taylor
    check against a continuous Fourier shift of a smooth object); and from the
    true object and probe, refinement walks perturbed positions back towards
    the truth (rms error monotone, below half after five steps)."""
    rng = np.random.default_rng(41)
    O = _crandn(7, 9, rng=rng)
    gy, gx = orc.object_gradient(O)
    for (y, x) in [(0, 0), (3, 4), (6, 8), (0, 5), (6, 0)]:
        ref_y = (O[min(y + 1, 6), x] - O[max(y - 1, 0), x]) / 2
        ref_x = (O[y, min(x + 1, 8)] - O[y, max(x - 1, 0)]) / 2
        assert abs(gy[y, x] - ref_y) < 1e-14 and abs(gx[y, x] - ref_x) < 1e-14, "object gradient"
    M, S = 16, 16
    P, O, pos = small_scan(M=M, K=2, grid=3, step=5)
    pos = np.rint(pos).astype(float) + 1.0
    true = np.round((pos + rng.uniform(0, 1, pos.shape)) * S) / S
    corner, delta = orc.subpixel_positions(true, S)
    chi = _crandn(len(pos), 2, M, M, rng=rng)
    s = orc.position_correction(O, P, corner, delta, chi)
    gy, gx = orc.object_gradient(O)
    for j, (y, x) in enumerate(corner):
        Pj = orc.shift_probe(P, *delta[j])
        ay, ax = Pj * gy[y:y + M, x:x + M][None], Pj * gx[y:y + M, x:x + M][None]
        lam = 1e-6 * (np.sum(np.abs(ay) ** 2) + np.sum(np.abs(ax) ** 2)) / 2
        # the regularised real least-squares problem, stacked for lstsq
        A = np.stack([np.concatenate([ay.real.ravel(), ay.imag.ravel()]),
                      np.concatenate([ax.real.ravel(), ax.imag.ravel()])], axis=1)
        A = np.vstack([A, np.sqrt(lam) * np.eye(2)])
        b = np.concatenate([chi[j].real.ravel(), chi[j].imag.ravel(), np.zeros(2)])
        ref = np.linalg.lstsq(A, b, rcond=None)[0]
        assert np.allclose(s[j], ref, rtol=1e-9, atol=1e-12), f"position correction of {j}"
    # Taylor: moving the (smooth, band-limited) object by h under the probe
    coef, freqs = _bandlimited(rng, 64, 3, 6)
    yy, xx = np.meshgrid(np.arange(40), np.arange(40), indexing="ij")
    Ob = 1.0 + 0.2 * _eval_bandlimited(coef, freqs, 64, yy, xx)
    gyb, gxb = orc.object_gradient(Ob)
    y0, x0 = 10, 12
    Pk = P[0]
    for (hy, hx) in [(1e-3, 0.0), (0.0, 1e-3), (7e-4, -5e-4)]:
        moved = 1.0 + 0.2 * _eval_bandlimited(coef, freqs, 64, y0 + hy + yy[:M, :M], x0 + hx + xx[:M, :M])
        I1 = np.abs(orc.fft2(Pk * moved)) ** 2
        lin = Pk * (Ob[y0:y0 + M, x0:x0 + M] + hy * gyb[y0:y0 + M, x0:x0 + M] + hx * gxb[y0:y0 + M, x0:x0 + M])
        I0 = np.abs(orc.fft2(Pk * Ob[y0:y0 + M, x0:x0 + M])) ** 2
        dI, dI_lin = I1 - I0, np.abs(orc.fft2(lin)) ** 2 - I0
        assert np.linalg.norm(dI - dI_lin) < 2e-2 * np.linalg.norm(dI), "first-order intensity change"
    I = orc.far_field_intensity(O, P, corner, delta)
    cur = true + np.round(rng.uniform(-0.3, 0.3, pos.shape) * S) / S
    errs = [np.sqrt(np.mean((cur - true) ** 2))]
    for _ in range(5):
        cur = orc.refine_positions(O, P, cur, I, S)
        errs.append(np.sqrt(np.mean((cur - true) ** 2)))
    assert all(b < a for a, b in zip(errs, errs[1:])) and errs[-1] < 0.5 * errs[0], errs


def pin_subpixel_epie(orc):
    """Sub-pixel ePIE: its object and probe corrections are steepest-descent
    steps of f = 1/2 sum_k ||z_k - (T_delta P_k) O_j||^2 (z the projected
    target, fixed), with steps alpha / max sum |T_delta P|^2 and
    beta / max |O_j|^2 (central differences through the shift); with a
    constant probe (T_delta 1 = 1) the patch moves to the error-reduction
    step whatever the shift."""
    rng = np.random.default_rng(28)
    M, K = 6, 2
    O = _crandn(8, 8, rng=rng)
    P = _crandn(K, M, M, rng=rng)
    raw = np.array([[1.25, 1.625]])
    pos, delta = orc.subpixel_positions(raw, 8)
    y, x = pos[0]
    I = np.abs(_crandn(1, M, M, rng=rng)) ** 2
    alpha, beta = 0.7, 0.3
    O1, P1, _ = orc.reconstruct("epie", O, P, raw, I, 1, epie_alpha=alpha, epie_beta=beta, subpixel=8)
    Oj = O[y:y + M, x:x + M]
    Pj = orc.shift_probe(P, *delta[0])
    F = np.fft.fft2(Pj * Oj)
    A = np.sqrt(np.sum(np.abs(F) ** 2, axis=0))
    z = np.fft.ifft2(F * np.fft.ifftshift(np.sqrt(I[0]))[None] / A[None])

    def f(Ov, Pv):
        return 0.5 * np.sum(np.abs(z - orc.shift_probe(Pv, *delta[0]) * Ov[None]) ** 2)

    h = 1e-6
    gO = np.zeros_like(Oj)
    for u in range(M):
        for v in range(M):
            e = np.zeros_like(Oj)
            e[u, v] = h
            gO[u, v] = (f(Oj + e, P) - f(Oj - e, P)) / (2 * h) + 1j * (f(Oj + 1j * e, P) - f(Oj - 1j * e, P)) / (2 * h)
    pmax = np.max(np.sum(np.abs(Pj) ** 2, axis=0))
    assert np.allclose(O1[y:y + M, x:x + M] - Oj, -alpha / pmax * gO, atol=1e-6), "sub-pixel ePIE object step"
    gP = np.zeros_like(P)
    for k in range(K):
        for u in range(M):
            for v in range(M):
                e = np.zeros_like(P)
                e[k, u, v] = h
                gP[k, u, v] = ((f(Oj, P + e) - f(Oj, P - e)) + 1j * (f(Oj, P + 1j * e) - f(Oj, P - 1j * e))) / (2 * h)
    omax = np.max(np.abs(Oj) ** 2)
    assert np.allclose(P1 - P, -beta / omax * gP, atol=1e-6), "sub-pixel ePIE probe step"
    M = 8
    O = _crandn(12, 12, rng=rng)
    P1c = np.ones((1, M, M), dtype=complex)
    raw = np.array([[2.375, 3.125]])
    (yy, xx), = orc.subpixel_positions(raw, 8)[0]
    I = np.abs(_crandn(1, M, M, rng=rng)) ** 2
    O2, _, _ = orc.reconstruct("epie", O, P1c, raw, I, 1, probe_start=5, subpixel=8)
    ref = O.copy()
    ref[yy:yy + M, xx:xx + M] = _er_step(O[yy:yy + M, xx:xx + M], I[0])
    assert np.allclose(O2, ref, atol=1e-12 * np.abs(ref).max()), "sub-pixel ePIE with P = 1 != error reduction"


ALL_PINS = [
    pin_fft_bruteforce, pin_parseval, pin_forward_bruteforce, pin_mode_mixing_invariance,
    pin_gather_scatter_adjoint, pin_rounding, pin_projection, pin_fourier_error,
    pin_fixed_points, pin_epie_er_special_case, pin_epie_gradient, pin_epie_order,
    pin_dm_overlap_least_squares, pin_dm_all_masked, pin_lsqml_step_sizes,
    pin_lsqml_er_special_case, pin_lsqml_all_masked, pin_lsqml_directions,
    pin_poisson_newton_step, pin_lsqml_poisson, pin_mode_orthogonalisation,
    pin_dm_mode_orthogonalisation_keeps_truth, pin_preprocess, pin_subpixel_positions,
    pin_fourier_shift, pin_subpixel_forward, pin_subpixel_gradients, pin_subpixel_dm_probe_solve,
    pin_subpixel_step_sizes, pin_position_refinement, pin_subpixel_epie,
    pin_subpixel_fixed_point_and_reduction,
]

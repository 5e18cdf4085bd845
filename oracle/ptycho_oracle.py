"""FP64 CPU oracle of the ptychographic reconstruction hot path.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The library
itself (``paper_2202_03144_b300``) never calls it and has no CPU fallback.

What it computes, and where it comes from
-----------------------------------------
The ptychopy paper (Yue et al., arXiv 2202.03144) names the method and its
three reconstruction algorithms but prints no formulas:

* the far-field forward model -- an exit wave (probe times object patch),
  whose Fourier transform's squared modulus is the measured diffraction
  pattern -- and the batched transforms of all the diffraction patterns
  are stated in Sec. 2.3 (Data reconstruction back end module);
* ePIE (Maiden & Rodenburg 2009), DM (Thibault et al. 2009, 2008) and LSQML
  (Thibault & Menzel 2013; Odstrcil et al. 2018) are named in the Abstract,
  Sec. 1 and Sec. 2.3; the multi-mode probe and the iteration after which
  the probe is updated are GUI parameters in Sec. 2.2.

The update rules below are therefore the standard published forms of those
cited algorithms, written out from their mathematics; every constant that the
paper does not fix (tau, reg, lambda, beta, the ePIE order) is a documented
reading of this library, identical on the CUDA side.

Conventions (shared with the C ABI):

* O: object [Ny, Nx] complex; P: probe modes [K, M, M] complex;
* positions: (y, x) of each patch's top-left corner, rounded half-to-even;
* F: unnormalised 2-D DFT (numpy ``fft2``); F^-1 = numpy ``ifft2`` (1/M^2);
* I: measured intensities [J, M, M], detector-centred (zero frequency at
  pixel (M/2, M/2)); a negative value marks a masked pixel.

Only library primitives used: ``numpy.fft.fft2/ifft2`` for the DFT and
elementwise numpy.  No blocking, fusion or reordering beyond the algorithms'
own steps.  Every function is pinned by the CPU tests in ``tests/``
(brute-force DFT, Parseval, adjointness, projection idempotence, fixed
points, reductions to an error-reduction step, least-squares optimality).
"""
from __future__ import annotations

import numpy as np

TAU = 1e-30          # modulus floor of the projection (FP64)
MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------------------
# Fourier transform and geometry (Sec. 2.3: far-field diffraction, FFTs)
# ---------------------------------------------------------------------------

def fft2(x: np.ndarray) -> np.ndarray:
    """Unnormalised forward 2-D DFT over the last two axes."""
    return np.fft.fft2(x, axes=(-2, -1))


def ifft2(x: np.ndarray) -> np.ndarray:
    """Inverse 2-D DFT over the last two axes, normalised by 1/M^2."""
    return np.fft.ifft2(x, axes=(-2, -1))


def round_positions(positions: np.ndarray) -> np.ndarray:
    """Integer top-left corners: round half to even."""
    return np.rint(np.asarray(positions, dtype=np.float64)).astype(np.int64)


def subpixel_positions(positions: np.ndarray, S: int) -> tuple[np.ndarray, np.ndarray]:
    """Positions quantised to 1/S pixel (S even), split into integer corners
    and sub-pixel shifts: q = rint(S y) (half to even), corner
    p = floor((q + S/2) / S), shift delta = q / S - p in [-1/2, 1/2).
    Returns (p [J, 2] integers, delta [J, 2] floats)."""
    if S < 2 or S % 2:
        raise ValueError("S must be an even integer >= 2")
    q = np.rint(S * np.asarray(positions, dtype=np.float64)).astype(np.int64)
    p = np.floor_divide(q + S // 2, S)
    return p, (q - S * p) / S


def shift_probe(P: np.ndarray, dy: float, dx: float) -> np.ndarray:
    """T_delta P: the probe (last two axes, M x M) translated by (dy, dx)
    pixels by the Fourier shift theorem, so (T P)(u) = P(u - delta) for a
    band-limited periodic P:
        F(T P)(f) = F(P)(f) exp(-2 pi i (f_y dy + f_x dx)),
    f = k / M for k < M/2 and (k - M) / M otherwise (numpy ``fftfreq``).
    T is unitary and T_delta^H = T_-delta."""
    M = P.shape[-1]
    f = np.fft.fftfreq(M)
    ph = np.exp(-2j * np.pi * (f[:, None] * dy + f[None, :] * dx))
    return ifft2(fft2(P) * ph)


def position_probes(P: np.ndarray, delta: np.ndarray | None) -> np.ndarray:
    """The probe each position sees: P[None] for integer positions (delta
    None), else P_j = T_delta_j P, shape [J, K, M, M]."""
    if delta is None:
        return P[None]
    return np.stack([shift_probe(P, dy, dx) for dy, dx in delta])


def check_positions(pos: np.ndarray, M: int, ny: int, nx: int) -> None:
    if pos.ndim != 2 or pos.shape[1] != 2:
        raise ValueError("positions must be [J, 2]")
    if (pos < 0).any() or (pos[:, 0] + M > ny).any() or (pos[:, 1] + M > nx).any():
        raise ValueError("a patch falls outside the object")


def gather(O: np.ndarray, pos: np.ndarray, M: int) -> np.ndarray:
    """Object patches O_j = O[y_j:y_j+M, x_j:x_j+M], shape [J, M, M]."""
    return np.stack([O[y:y + M, x:x + M] for y, x in pos])


def scatter_add(shape: tuple, pos: np.ndarray, patches: np.ndarray) -> np.ndarray:
    """Sum_j S_j[patches_j]: the adjoint of :func:`gather`, summed in j order."""
    M = patches.shape[-1]
    acc = np.zeros(shape, dtype=patches.dtype)
    for j, (y, x) in enumerate(pos):
        acc[y:y + M, x:x + M] += patches[j]
    return acc


def exit_waves(O: np.ndarray, P: np.ndarray, pos: np.ndarray, delta=None) -> np.ndarray:
    """psi_{j,k} = P_k * O_j (sub-pixel: (T_delta_j P_k) * O_j), shape [J, K, M, M]."""
    M = P.shape[-1]
    return position_probes(P, delta) * gather(O, pos, M)[:, None, :, :]


def far_field_intensity(O: np.ndarray, P: np.ndarray, pos: np.ndarray, delta=None) -> np.ndarray:
    """Detector-centred I_j = fftshift(sum_k |F(P_k O_j)|^2), shape [J, M, M]."""
    Psi = fft2(exit_waves(O, P, pos, delta))
    I = np.sum(np.abs(Psi) ** 2, axis=1)
    return np.fft.fftshift(I, axes=(-2, -1))


def to_fft_order(I: np.ndarray) -> np.ndarray:
    """Move the zero frequency of detector-centred frames back to pixel (0, 0)."""
    return np.fft.ifftshift(I, axes=(-2, -1))


# ---------------------------------------------------------------------------
# Modulus projection and Fourier error
# ---------------------------------------------------------------------------

def project(Psi: np.ndarray, I_fft: np.ndarray, tau: float = TAU) -> np.ndarray:
    """Replace the mode-summed Fourier modulus by sqrt(I).

    Psi: [J, K, M, M] far fields; I_fft: [J, M, M] intensities in FFT order.
    A = sqrt(sum_k |Psi_k|^2).  Where I < 0 (masked) Psi is returned
    unchanged; where A <= tau the result is 0; elsewhere Psi_k sqrt(I) / A.
    """
    A = np.sqrt(np.sum(np.abs(Psi) ** 2, axis=1))
    masked = I_fft < 0
    sqrtI = np.sqrt(np.where(masked, 0.0, I_fft))
    safe_A = np.where(A > tau, A, 1.0)
    ratio = np.where(A > tau, sqrtI / safe_A, 0.0)
    out = Psi * ratio[:, None, :, :]
    return np.where(masked[:, None, :, :], Psi, out)


def fourier_error(O: np.ndarray, P: np.ndarray, pos: np.ndarray, I: np.ndarray, delta=None) -> float:
    """E = sum m (A - sqrt I)^2 / sum m I over all frames and unmasked pixels,
    from a fresh forward pass at the current (O, P)."""
    I_fft = to_fft_order(I)
    A = np.sqrt(np.sum(np.abs(fft2(exit_waves(O, P, pos, delta))) ** 2, axis=1))
    m = I_fft >= 0
    sqrtI = np.sqrt(np.where(m, I_fft, 0.0))
    num = float(np.sum(np.where(m, (A - sqrtI) ** 2, 0.0)))
    den = float(np.sum(np.where(m, I_fft, 0.0)))
    return num / den if den > 0 else 0.0


def poisson_correction(Psi: np.ndarray, I_fft: np.ndarray) -> np.ndarray:
    """Detector-plane correction of the Poisson likelihood (maximum-likelihood
    exit-wave update for photon counts; Odstrcil et al. 2018).

    With A^2 = sum_k |Psi_k|^2 the pixel's negative log-likelihood is
    A^2 - I log A^2; its steepest-descent direction in Psi_k is
    g = (I / A^2 - 1) Psi_k, unbounded where the model is far weaker than the
    counts.  One Newton step along g from the current value, per pixel, scales
    it by A^2 / (A^2 + I), giving

        (I - A^2) / (I + A^2) * Psi_k,

    a factor in [-1, 1] that equals the amplitude projection's
    sqrt(I)/A - 1 to first order near a fit.  Masked pixels (I < 0) and
    pixels with I + A^2 = 0 get no correction."""
    A2 = np.sum(np.abs(Psi) ** 2, axis=1)
    masked = I_fft < 0
    Iu = np.where(masked, 0.0, I_fft)
    den = Iu + A2
    f = np.where(masked | (den <= 0), 0.0, (Iu - A2) / np.where(den > 0, den, 1.0))
    return Psi * f[:, None, :, :]


def poisson_nll(O: np.ndarray, P: np.ndarray, pos: np.ndarray, I: np.ndarray, delta=None) -> float:
    """sum over unmasked pixels of A^2 - I log A^2 at the current (O, P)."""
    I_fft = to_fft_order(I)
    A2 = np.sum(np.abs(fft2(exit_waves(O, P, pos, delta))) ** 2, axis=1)
    m = I_fft >= 0
    return float(np.sum(np.where(m, A2 - np.where(m, I_fft, 0.0) * np.log(np.where(m, A2, 1.0)), 0.0)))


def fourier_residual(O: np.ndarray, P: np.ndarray, pos: np.ndarray, I: np.ndarray,
                     likelihood: str = "amplitude", delta=None) -> np.ndarray:
    """Exit-wave residual chi_{j,k}, shape [J, K, M, M].

    amplitude (Gaussian noise on sqrt I): chi = F^-1 Pi(F(P_k O_j)) - P_k O_j;
    poisson: chi = F^-1 [(I - A^2) / (I + A^2) F(P_k O_j)], the per-pixel
    Newton step of the Poisson negative log-likelihood along its gradient
    (:func:`poisson_correction`)."""
    phi = exit_waves(O, P, pos, delta)
    if likelihood == "amplitude":
        return ifft2(project(fft2(phi), to_fft_order(I))) - phi
    if likelihood == "poisson":
        return ifft2(poisson_correction(fft2(phi), to_fft_order(I)))
    raise ValueError(likelihood)


# ---------------------------------------------------------------------------
# ePIE  (Maiden & Rodenburg 2009; multi-mode form of Thibault & Menzel 2013)
# ---------------------------------------------------------------------------

def splitmix64_stream(state: int):
    """Counter-based 64-bit generator (Steele, Lea & Flood's SplitMix64)."""
    while True:
        state = (state + 0x9E3779B97F4A7C15) & MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        yield z ^ (z >> 31)


def epie_order(seed: int, t: int, J: int) -> np.ndarray:
    """Visiting order of iteration t: identity for seed 0, else a
    Fisher-Yates (Durstenfeld) shuffle drawn from SplitMix64(seed XOR t)."""
    order = list(range(J))
    if seed == 0:
        return np.asarray(order, dtype=np.int64)
    g = splitmix64_stream((seed ^ t) & MASK64)
    for i in range(J - 1, 0, -1):
        r = next(g) % (i + 1)
        order[i], order[r] = order[r], order[i]
    return np.asarray(order, dtype=np.int64)


def epie_position_update(O, P, y, x, I_fft_j, alpha, beta, update_probe, shift=None):
    """One ePIE step at the patch with top-left (y, x); updates O and P in place.

    psi_k = P_k O_j; Delta_k = F^-1 Pi(F psi)_k - psi_k;
    O_j += alpha sum_k conj(P_k) Delta_k / max_u sum_k |P_k(u)|^2;
    P_k += beta conj(O_j_old) Delta_k / max_u |O_j_old(u)|^2  (if update_probe),
    both from the values held before this step.

    Sub-pixel position (shift = delta_j): the position sees P_j = T_delta P
    (:func:`shift_probe`), which takes P's place in the exit wave, the object
    step and its maximum; the probe step is taken in that frame and moved back
    by the adjoint shift, P_k += beta T_-delta[conj(O_j_old) Delta_k] / max
    |O_j_old|^2 (the steepest-descent step in P of the same objective).
    """
    M = P.shape[-1]
    Oj = O[y:y + M, x:x + M].copy()
    Pj = P if shift is None else shift_probe(P, shift[0], shift[1])
    psi = Pj * Oj[None]
    Delta = ifft2(project(fft2(psi)[None], I_fft_j[None])[0]) - psi
    pmax = float(np.max(np.sum(np.abs(Pj) ** 2, axis=0)))
    omax = float(np.max(np.abs(Oj) ** 2))
    if pmax > 0:
        O[y:y + M, x:x + M] = Oj + alpha * np.sum(np.conj(Pj) * Delta, axis=0) / pmax
    if update_probe and omax > 0:
        step = np.conj(Oj)[None] * Delta
        if shift is not None:
            step = shift_probe(step, -shift[0], -shift[1])
        P[...] = P + beta * step / omax


def epie_iteration(O, P, pos, I, t, seed=0, alpha=1.0, beta=1.0, probe_start=0, delta=None):
    """One ePIE sweep (iteration index t) over all positions; returns new (O, P)."""
    O = O.astype(np.complex128).copy()
    P = P.astype(np.complex128).copy()
    I_fft = to_fft_order(I)
    for j in epie_order(seed, t, len(pos)):
        y, x = pos[j]
        epie_position_update(O, P, y, x, I_fft[j], alpha, beta, t >= probe_start,
                             None if delta is None else delta[j])
    return O, P


# ---------------------------------------------------------------------------
# Overlap quantities shared by DM and LSQML
# ---------------------------------------------------------------------------

def object_denominator(P: np.ndarray, pos: np.ndarray, shape: tuple, delta=None) -> np.ndarray:
    """den_O = sum_j S_j[sum_k |P_jk|^2] (real, object-sized); P_j is the probe
    position j sees (:func:`position_probes`)."""
    w = np.sum(np.abs(position_probes(P, delta)) ** 2, axis=1)
    return scatter_add(shape, pos, np.broadcast_to(w, (len(pos),) + w.shape[1:]).astype(np.float64))


def object_numerator(P: np.ndarray, X: np.ndarray, pos: np.ndarray, shape: tuple,
                     weights: np.ndarray | None = None, delta=None) -> np.ndarray:
    """sum_j w_j S_j[sum_k conj(P_jk) X_{j,k}] (object-sized)."""
    c = np.sum(np.conj(position_probes(P, delta)) * X, axis=1)
    if weights is not None:
        c = c * np.asarray(weights, dtype=np.float64)[:, None, None]
    return scatter_add(shape, pos, c)


def probe_numerator(O: np.ndarray, X: np.ndarray, pos: np.ndarray,
                    weights: np.ndarray | None = None, delta=None) -> np.ndarray:
    """sum_j w_j conj(O_j) X_{j,k}, shape [K, M, M].  Sub-pixel positions:
    sum_j w_j T_-delta_j[conj(O_j) X_{j,k}], the adjoint of P -> T_delta_j P
    applied to each term (summed in j order)."""
    M = X.shape[-1]
    Oc = np.conj(gather(O, pos, M))[:, None]
    t = Oc * X
    if weights is not None:
        t = t * np.asarray(weights, dtype=np.float64)[:, None, None, None]
    if delta is not None:
        t = np.stack([shift_probe(t[j], -dy, -dx) for j, (dy, dx) in enumerate(delta)])
    return np.sum(t, axis=0)


def probe_denominator(O: np.ndarray, pos: np.ndarray, M: int) -> np.ndarray:
    """den_P = sum_j |O_j|^2, shape [M, M].  With sub-pixel positions the same
    unshifted sum serves as the diagonal scaling of the LSQML probe direction
    and as the preconditioner of the DM probe solve: the exact normal operator
    sum_j T_j^H |O_j|^2 T_j is not diagonal, and |O_j|^2 varies little over a
    fraction of a pixel."""
    return np.sum(np.abs(gather(O, pos, M)) ** 2, axis=0)


# ---------------------------------------------------------------------------
# DM  (difference map; Thibault et al. 2009 / 2008)
# ---------------------------------------------------------------------------

DM_PROBE_CG = 4     # conjugate-gradient iterations of the sub-pixel DM probe solve


def probe_normal_operator(O: np.ndarray, pos: np.ndarray, delta: np.ndarray, X: np.ndarray) -> np.ndarray:
    """B X = sum_j T_-delta_j[|O_j|^2 T_delta_j X]: the normal operator of
    P -> {(T_delta_j P) O_j}, applied to probe-shaped X [K, M, M] (summed in j
    order)."""
    M = X.shape[-1]
    D = np.abs(gather(O, pos, M)) ** 2
    out = np.zeros_like(X, dtype=np.complex128)
    for j, (dy, dx) in enumerate(delta):
        out += shift_probe(D[j][None] * shift_probe(X, dy, dx), -dy, -dx)
    return out


def dm_probe_solve(O, P, psi, pos, reg, delta, n_cg=DM_PROBE_CG):
    """Sub-pixel DM probe update: the least-squares problem
        min_P sum_j ||psi_j - (T_delta_j P) O_j||^2 + d_P ||P - P_old||^2
    has the normal equations (B + d_P) P = sum_j T_-delta_j[conj(O_j) psi_j]
    + d_P P_old (B: :func:`probe_normal_operator`), no longer diagonal.  They
    are solved by n_cg iterations of preconditioned conjugate gradients from
    P_old, with the diagonal preconditioner den_P + d_P (den_P =
    sum_j |O_j|^2, d_P = reg max den_P) and Re<.,.> over all modes and pixels:
        r = rhs - (B + d) X,  z = r / (den + d),  p = z;
        repeat: q = (B + d) p, a = <r,z>/<p,q>, X += a p, r -= a q,
                z = r / (den + d), b = <r,z>_new/<r,z>_old, p = z + b p.
    A zero <p,q> or <r,z> ends the updates (a = 0, b = 0).  Without the exact
    solve the overlap step is not a projection and the difference map drifts
    off (the diagonal form with the shifted numerator diverges)."""
    M = P.shape[-1]
    den = probe_denominator(O, pos, M)
    d = reg * float(den.max())
    w = (den + d)[None]
    X = P.copy()
    r = probe_numerator(O, psi, pos, delta=delta) - probe_normal_operator(O, pos, delta, X)
    z = r / w
    p = z.copy()
    rz = float(np.real(np.vdot(r, z)))
    for _ in range(n_cg):
        q = probe_normal_operator(O, pos, delta, p) + d * p
        pq = float(np.real(np.vdot(p, q)))
        a = rz / pq if pq > 0 else 0.0
        X = X + a * p
        r = r - a * q
        z = r / w
        rz_new = float(np.real(np.vdot(r, z)))
        b = rz_new / rz if rz > 0 else 0.0
        p = z + b * p
        rz = rz_new
    return X


def dm_init(O: np.ndarray, P: np.ndarray, pos: np.ndarray, delta=None) -> np.ndarray:
    """Initial exit-wave state psi = P_k O_j."""
    return exit_waves(O, P, pos, delta)


def dm_overlap_update(O, P, psi, pos, reg, update_probe, delta=None):
    """Overlap projection: object then probe least-squares update from psi.

    O <- (sum_j S_j[sum_k conj(P_k) psi_jk] + d_O O) / (den_O + d_O),
    then, with the new O, P_k <- (sum_j conj(O_j) psi_jk + d_P P_k) / (den_P + d_P),
    d = reg * max(den).  Sub-pixel positions: P_k -> P_jk in the object
    update (exact), and the probe update solves its (non-diagonal) normal
    equations by conjugate gradients (:func:`dm_probe_solve`).
    """
    M = P.shape[-1]
    den_O = object_denominator(P, pos, O.shape, delta)
    num_O = object_numerator(P, psi, pos, O.shape, delta=delta)
    d_O = reg * float(den_O.max())
    O = (num_O + d_O * O) / (den_O + d_O)
    if update_probe and delta is not None:
        P = dm_probe_solve(O, P, psi, pos, reg, delta)
    elif update_probe:
        den_P = probe_denominator(O, pos, M)
        num_P = probe_numerator(O, psi, pos)
        d_P = reg * float(den_P.max())
        P = (num_P + d_P * P) / (den_P[None] + d_P)
    return O, P


def dm_iteration(O, P, psi, pos, I, t, reg=1e-3, probe_start=0, delta=None):
    """One DM iteration (index t); returns new (O, P, psi).

    1-2. overlap update of O, then of P (when t >= probe_start);
    3.   phi = P_k O_j;  psi <- psi + F^-1 Pi(F(2 phi - psi)) - phi.
    """
    O, P = dm_overlap_update(O.astype(np.complex128), P.astype(np.complex128), psi, pos,
                             reg, t >= probe_start, delta)
    phi = exit_waves(O, P, pos, delta)
    psi = psi + ifft2(project(fft2(2.0 * phi - psi), to_fft_order(I))) - phi
    return O, P, psi


# ---------------------------------------------------------------------------
# LSQML  (Odstrcil et al. 2018, amplitude likelihood, whole batch)
# ---------------------------------------------------------------------------

def lsqml_directions(O, P, chi, pos, reg, update_probe, delta=None):
    """Steepest-descent directions and their normalising denominators.

    dO = sum_j S_j[sum_k conj(P_k) chi_jk] / (den_O + d_O);
    dP_k = sum_j conj(O_j) chi_jk / (den_P + d_P)   (zero if the probe is fixed).
    Returns (dO, dP, den_O + d_O, den_P + d_P or None).
    """
    M = P.shape[-1]
    den_O = object_denominator(P, pos, O.shape, delta)
    d_O = reg * float(den_O.max())
    wO = den_O + d_O
    dO = object_numerator(P, chi, pos, O.shape, delta=delta) / wO
    if update_probe:
        den_P = probe_denominator(O, pos, M)
        d_P = reg * float(den_P.max())
        wP = den_P + d_P
        dP = probe_numerator(O, chi, pos, delta=delta) / wP[None]
    else:
        wP = None
        dP = np.zeros_like(P)
    return dO, dP, wO, wP


def lsqml_solve_2x2(A11: float, A12: float, A22: float, r1: float, r2: float) -> tuple[float, float]:
    """Solve ([[A11, A12], [A12, A22]] + lam I) alpha = r, lam = 1e-6 (A11 + A22) / 2;
    alpha = 0 when the trace vanishes."""
    tr = A11 + A22
    if not tr > 0.0:
        return 0.0, 0.0
    lam = 1e-6 * tr / 2.0
    a, b, d = A11 + lam, A12, A22 + lam
    det = a * d - b * b
    return (d * r1 - b * r2) / det, (a * r2 - b * r1) / det


def lsqml_step_sizes(O, P, chi, pos, dO, dP, delta=None):
    """Per-position (alpha_O, alpha_P): least squares fit of chi_j by
    alpha_O a_j + alpha_P b_j with a_jk = P_jk dO_j and b_jk = O_j dP_jk
    (P_j, dP_j: the probe and its direction as position j sees them)."""
    M = P.shape[-1]
    Oj = gather(O, pos, M)
    dOj = gather(dO, pos, M)
    Pj = position_probes(P, delta)     # [1 or J, K, M, M]
    dPj = position_probes(dP, delta)
    aO = np.empty(len(pos))
    aP = np.empty(len(pos))
    for j in range(len(pos)):
        i = 0 if delta is None else j
        a = Pj[i] * dOj[j][None]
        b = Oj[j][None] * dPj[i]
        A11 = float(np.sum(np.abs(a) ** 2))
        A12 = float(np.real(np.sum(np.conj(a) * b)))
        A22 = float(np.sum(np.abs(b) ** 2))
        r1 = float(np.real(np.sum(np.conj(a) * chi[j])))
        r2 = float(np.real(np.sum(np.conj(b) * chi[j])))
        aO[j], aP[j] = lsqml_solve_2x2(A11, A12, A22, r1, r2)
    return aO, aP


def lsqml_iteration(O, P, pos, I, t, reg=1e-3, beta=0.9, probe_start=0, return_steps=False,
                    likelihood="amplitude", delta=None):
    """One LSQML iteration (index t); returns new (O, P) [and (alpha_O, alpha_P)].

    1. chi_jk = F^-1 Pi(F(P_k O_j)) - P_k O_j (amplitude likelihood) or the
       Poisson correction F^-1[(I - A^2)/(I + A^2) F(P_k O_j)] (see
       :func:`fourier_residual`);
    2. directions dO, dP (see :func:`lsqml_directions`);
    3. per-position step sizes (see :func:`lsqml_step_sizes`);
    4. O <- O + beta sum_j S_j[alpha_O,j sum_k conj(P_k) chi_jk] / (den_O + d_O),
       P_k <- P_k + beta sum_j alpha_P,j conj(O_j) chi_jk / (den_P + d_P),
       both from the values held at the start of the iteration.
    Sub-pixel positions (delta): every P_k O_j is (T_delta_j P_k) O_j and the
    probe sums take the adjoint shift (:func:`probe_numerator`).
    """
    O = O.astype(np.complex128)
    P = P.astype(np.complex128)
    upd = t >= probe_start
    chi = fourier_residual(O, P, pos, I, likelihood, delta)
    dO, dP, wO, wP = lsqml_directions(O, P, chi, pos, reg, upd, delta)
    aO, aP = lsqml_step_sizes(O, P, chi, pos, dO, dP, delta)
    O_new = O + beta * object_numerator(P, chi, pos, O.shape, weights=aO, delta=delta) / wO
    if upd:
        P_new = P + beta * probe_numerator(O, chi, pos, weights=aP, delta=delta) / wP[None]
    else:
        P_new = P.copy()
    if return_steps:
        return O_new, P_new, (aO, aP)
    return O_new, P_new


# ---------------------------------------------------------------------------
# Position refinement (sub-pixel positions; the position-correction step of
# Odstrcil et al. 2018, cited for LSQML in Sec. 1)
# ---------------------------------------------------------------------------

def object_gradient(O: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Central differences (d/dy, d/dx) of the object,
    (O(y + 1, x) - O(y - 1, x)) / 2 and likewise in x, an index past the edge
    taken as the edge pixel."""
    Op = np.pad(O, 1, mode="edge")
    return (Op[2:, 1:-1] - Op[:-2, 1:-1]) / 2.0, (Op[1:-1, 2:] - Op[1:-1, :-2]) / 2.0


def position_correction(O, P, pos, delta, chi):
    """Per-position shift (dy, dx) that best explains the exit-wave residual.
    The exit wave of the probe at r is P(u) O(r + u) in its own window; moving
    r by s changes it by s_y a_y + s_x a_x to first order with
    a_y = P_jk d_yO_j (the illuminated object's gradient, central differences:
    :func:`object_gradient`; P_j the probe position j sees).  (In the window
    of the integer corner the same move also translates the whole exit wave,
    which changes no far-field modulus and so cannot be fitted.)  s minimises
    ||chi_j - s_y a_y - s_x a_x||^2 over all modes and pixels; the 2x2 normal
    equations are solved as the LSQML step sizes are (:func:`lsqml_solve_2x2`,
    FP64).  Returns [J, 2]."""
    M = P.shape[-1]
    gy, gx = object_gradient(O)
    Gy, Gx = gather(gy, pos, M), gather(gx, pos, M)
    Pj = position_probes(P, delta)
    out = np.empty((len(pos), 2))
    for j in range(len(pos)):
        Pk = Pj[0 if delta is None else j]
        ay = Pk * Gy[j][None]
        ax = Pk * Gx[j][None]
        A11 = float(np.sum(np.abs(ay) ** 2))
        A12 = float(np.real(np.sum(np.conj(ay) * ax)))
        A22 = float(np.sum(np.abs(ax) ** 2))
        r1 = float(np.real(np.sum(np.conj(ay) * chi[j])))
        r2 = float(np.real(np.sum(np.conj(ax) * chi[j])))
        out[j] = lsqml_solve_2x2(A11, A12, A22, r1, r2)
    return out


def refine_positions(O, P, positions, I, S, step=1.0, max_shift=0.5, likelihood="amplitude"):
    """One position-refinement step at the current (O, P): the residual chi of
    a fresh Fourier pass (:func:`fourier_residual`) at the positions quantised
    to 1/S pixel, the correction of :func:`position_correction`, each
    component clipped to [-max_shift, max_shift] pixels and scaled by step.
    Returns the new (unquantised) positions."""
    pos, delta = subpixel_positions(positions, S)
    chi = fourier_residual(O, P, pos, I, likelihood, delta)
    d = position_correction(O, P, pos, delta, chi)
    return np.asarray(positions, dtype=np.float64) + step * np.clip(d, -max_shift, max_shift)


# ---------------------------------------------------------------------------
# Detector preprocessing (Sec. 2.2: centre, crop size, saturation bit depth,
# noise threshold and rotation of the diffraction patterns)
# ---------------------------------------------------------------------------

def preprocess_frames(raw: np.ndarray, center: tuple, M: int, saturation_bits: int = 0,
                      threshold: float = 0.0, rot90: int = 0) -> np.ndarray:
    """Detector-centred M x M intensities from raw frames [J, H, W].

    Output pixel (y, x) has offset d = (y - M/2, x - M/2) from the zero
    frequency.  It reads the raw pixel center + R^-k d, where R turns an
    offset a quarter turn counter-clockwise, (a, b) -> (-b, a), k = rot90, and
    offsets wrap into [-M/2, M/2) (the DFT grid is periodic).  center is
    rounded half-to-even.  A raw pixel outside the frame, negative, or (with
    saturation_bits > 0) at or above 2^bits - 1 is masked (-1); a value below
    threshold (> 0) becomes 0 (noise removal)."""
    raw = np.asarray(raw, dtype=np.float64)
    J, H, W = raw.shape
    cy, cx = (int(v) for v in np.rint(np.asarray(center, dtype=np.float64)))
    h = M // 2
    dy, dx = np.meshgrid(np.arange(M) - h, np.arange(M) - h, indexing="ij")
    sy, sx = dy, dx
    for _ in range(rot90 % 4):  # apply R^-1: (a, b) -> (b, -a)
        sy, sx = sx, -sy
    sy = np.mod(sy + h, M) - h
    sx = np.mod(sx + h, M) - h
    ry, rx = cy + sy, cx + sx
    inside = (ry >= 0) & (ry < H) & (rx >= 0) & (rx < W)
    v = raw[:, np.clip(ry, 0, H - 1), np.clip(rx, 0, W - 1)]
    masked = ~inside[None] | (v < 0)
    if saturation_bits > 0:
        masked |= v >= float(2 ** saturation_bits - 1)
    if threshold > 0:
        v = np.where(v < threshold, 0.0, v)
    return np.where(masked, -1.0, v)


# ---------------------------------------------------------------------------
# Probe-mode orthogonalisation (Thibault & Menzel 2013, cited in Sec. 1)
# ---------------------------------------------------------------------------

def mode_basis(P: np.ndarray) -> np.ndarray:
    """Unitary V [K, K] whose columns are the eigenvectors of the modes' Gram
    matrix G[l, k] = <P_l, P_k> = sum_u conj(P_l(u)) P_k(u), ordered by
    decreasing eigenvalue (mode power); each column's phase is fixed so that
    its entry of largest modulus (the first one on a tie) is real positive."""
    K = P.shape[0]
    flat = P.reshape(K, -1)
    G = np.conj(flat) @ flat.T
    lam, V = np.linalg.eigh(G)
    V = V[:, np.argsort(-lam, kind="stable")]
    for m in range(K):
        i = int(np.argmax(np.abs(V[:, m])))
        V[:, m] *= np.conj(V[i, m]) / abs(V[i, m])
    return V


def mix_modes(X: np.ndarray, V: np.ndarray, axis: int = 0) -> np.ndarray:
    """X'_m = sum_l V[l, m] X_l along the mode axis."""
    return np.moveaxis(np.tensordot(V, np.moveaxis(X, axis, 0), axes=([0], [0])), 0, axis)


def orthogonalize_modes(P: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Orthogonal probe modes P'_m = sum_l V[l, m] P_l (see :func:`mode_basis`):
    <P'_m, P'_n> = 0 for m != n, powers ||P'_m||^2 the eigenvalues of G in
    decreasing order, and sum_m |P'_m(u)|^2 = sum_l |P_l(u)|^2 at every pixel
    (a unitary mixing leaves every diffraction pattern unchanged).  Returns
    (P', V)."""
    V = mode_basis(P)
    return mix_modes(P, V), V


# ---------------------------------------------------------------------------
# Driver used by tests and the CPU baseline
# ---------------------------------------------------------------------------

def reconstruct(alg: str, O, P, positions, I, n_iter, t0=0, psi=None, seed=0, reg=1e-3,
                epie_alpha=1.0, epie_beta=1.0, lsqml_beta=0.9, probe_start=0, likelihood="amplitude",
                probe_ortho=False, subpixel=0):
    """Run n_iter iterations of 'epie', 'dm' or 'lsqml' starting at index t0.

    probe_ortho: after every iteration that updated the probe, orthogonalise
    its modes (:func:`orthogonalize_modes`); DM's exit waves are mixed with
    the same unitary so that psi_jk stays P_k O_j-shaped.

    subpixel: S > 0 quantises the positions to 1/S pixel and shifts the probe
    by each position's sub-pixel part (:func:`subpixel_positions`).

    Returns (O, P, psi) -- psi is the DM state (None for the others)."""
    delta = None
    if subpixel:
        pos, delta = subpixel_positions(positions, subpixel)
    else:
        pos = round_positions(positions)
    O = np.asarray(O, dtype=np.complex128)
    P = np.asarray(P, dtype=np.complex128)
    check_positions(pos, P.shape[-1], *O.shape)
    for t in range(t0, t0 + n_iter):
        if alg == "epie":
            O, P = epie_iteration(O, P, pos, I, t, seed, epie_alpha, epie_beta, probe_start, delta)
        elif alg == "dm":
            if psi is None:
                psi = dm_init(O, P, pos, delta)
            O, P, psi = dm_iteration(O, P, psi, pos, I, t, reg, probe_start, delta)
        elif alg == "lsqml":
            O, P = lsqml_iteration(O, P, pos, I, t, reg, lsqml_beta, probe_start, likelihood=likelihood,
                                   delta=delta)
        else:
            raise ValueError(alg)
        if probe_ortho and t >= probe_start and P.shape[0] > 1:
            P, V = orthogonalize_modes(P)
            if alg == "dm":
                psi = mix_modes(psi, V, axis=1)
    return O, P, psi

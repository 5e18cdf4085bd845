"""The pins have teeth: plant a plausible mistake in a copy of the oracle's
source (a dropped term, a wrong sign, a missing conjugate, a transposed index)
and check that at least one pin fails on it.  CPU only; the real oracle is
never modified."""
import importlib.util
import inspect
import types

import pytest

import pins
from oracle import ptycho_oracle as orc

SRC = inspect.getsource(orc)

MUTATIONS = {
    "no_sqrt_in_projection": ("sqrtI = np.sqrt(np.where(masked, 0.0, I_fft))",
                              "sqrtI = np.where(masked, 0.0, I_fft)"),
    "conj_probe_in_exit_wave": ("return position_probes(P, delta) * gather(O, pos, M)[:, None, :, :]",
                                "return np.conj(position_probes(P, delta)) * gather(O, pos, M)[:, None, :, :]"),
    "no_fftshift_in_forward": ("return np.fft.fftshift(I, axes=(-2, -1))", "return I"),
    "ifft_as_forward": ("return np.fft.fft2(x, axes=(-2, -1))",
                        "return np.fft.ifft2(x, axes=(-2, -1)) * (x.shape[-1] * x.shape[-2])"),
    "scatter_transposed": ("acc[y:y + M, x:x + M] += patches[j]", "acc[x:x + M, y:y + M] += patches[j]"),
    "object_numerator_no_conj": ("c = np.sum(np.conj(position_probes(P, delta)) * X, axis=1)",
                                 "c = np.sum(position_probes(P, delta) * X, axis=1)"),
    "probe_numerator_no_conj": ("Oc = np.conj(gather(O, pos, M))[:, None]", "Oc = gather(O, pos, M)[:, None]"),
    "dm_reflection_swapped": ("project(fft2(2.0 * phi - psi)", "project(fft2(2.0 * psi - phi)"),
    "dm_wrong_sign_phi": ("psi = psi + ifft2(project(fft2(2.0 * phi - psi), to_fft_order(I))) - phi",
                          "psi = psi + ifft2(project(fft2(2.0 * phi - psi), to_fft_order(I))) + phi"),
    "dm_drop_prox_term": ("O = (num_O + d_O * O) / (den_O + d_O)", "O = num_O / (den_O + d_O)"),
    "lsqml_solve_sign": ("return (d * r1 - b * r2) / det, (a * r2 - b * r1) / det",
                         "return (d * r1 + b * r2) / det, (a * r2 - b * r1) / det"),
    "lsqml_conj_object_in_b": ("b = Oj[j][None] * dPj[i]", "b = np.conj(Oj[j])[None] * dPj[i]"),
    "lsqml_swapped_weights": ("object_numerator(P, chi, pos, O.shape, weights=aO,",
                              "object_numerator(P, chi, pos, O.shape, weights=aP,"),
    "lsqml_lambda_too_big": ("lam = 1e-6 * tr / 2.0", "lam = 1e-3 * tr / 2.0"),
    "epie_no_conj_probe": ("alpha * np.sum(np.conj(Pj) * Delta, axis=0) / pmax",
                           "alpha * np.sum(Pj * Delta, axis=0) / pmax"),
    "epie_sum_not_max": ("pmax = float(np.max(np.sum(np.abs(Pj) ** 2, axis=0)))",
                         "pmax = float(np.sum(np.abs(Pj) ** 2))"),
    "epie_probe_from_new_object": ("step = np.conj(Oj)[None] * Delta",
                                   "step = np.conj(O[y:y + M, x:x + M])[None] * Delta"),
    "epie_subpixel_probe_unshifted": ("Pj = P if shift is None else shift_probe(P, shift[0], shift[1])", "Pj = P"),
    "epie_subpixel_no_adjoint": ("step = shift_probe(step, -shift[0], -shift[1])", "step = step"),
    "error_den_sqrt": ("den = float(np.sum(np.where(m, I_fft, 0.0)))",
                       "den = float(np.sum(np.where(m, sqrtI, 0.0)))"),
    "splitmix_constant": ("0xBF58476D1CE4E5B9", "0xBF58476D1CE4E5B8"),
    "rounding_floor": ("return np.rint(np.asarray(positions, dtype=np.float64)).astype(np.int64)",
                       "return np.floor(np.asarray(positions, dtype=np.float64)).astype(np.int64)"),
    "poisson_sqrt_counts": ("Iu = np.where(masked, 0.0, I_fft)\n    den", "Iu = np.sqrt(np.where(masked, 0.0, I_fft))\n    den"),
    "poisson_no_mode_sum": ("A2 = np.sum(np.abs(Psi) ** 2, axis=1)\n    masked = I_fft < 0\n    Iu",
                            "A2 = np.abs(Psi[:, 0]) ** 2\n    masked = I_fft < 0\n    Iu"),
    "poisson_raw_gradient": ("(Iu - A2) / np.where(den > 0, den, 1.0))",
                             "(Iu - A2) / np.where(A2 > 0, A2, 1.0))"),
    "poisson_masked_pulls": ("f = np.where(masked | (den <= 0), 0.0,", "f = np.where(den <= 0, 0.0,"),
    "modes_ascending": ("V = V[:, np.argsort(-lam, kind=\"stable\")]", "V = V[:, np.argsort(lam, kind=\"stable\")]"),
    "modes_gram_no_conj": ("G = np.conj(flat) @ flat.T", "G = flat @ flat.T"),
    "modes_mix_transposed": ("return np.moveaxis(np.tensordot(V, np.moveaxis(X, axis, 0), axes=([0], [0])), 0, axis)",
                             "return np.moveaxis(np.tensordot(V, np.moveaxis(X, axis, 0), axes=([1], [0])), 0, axis)"),
    "modes_dm_psi_not_mixed": ("                psi = mix_modes(psi, V, axis=1)", "                pass"),
    "preprocess_clockwise": ("        sy, sx = sx, -sy", "        sy, sx = -sx, sy"),
    "preprocess_no_wrap": ("    sy = np.mod(sy + h, M) - h", "    sy = sy"),
    "preprocess_saturation_strict": ("masked |= v >= float(2 ** saturation_bits - 1)",
                                     "masked |= v > float(2 ** saturation_bits - 1)"),
    "preprocess_center_floor": ("cy, cx = (int(v) for v in np.rint(np.asarray(center, dtype=np.float64)))",
                                "cy, cx = (int(v) + 1 for v in np.rint(np.asarray(center, dtype=np.float64)))"),
    "shift_sign": ("ph = np.exp(-2j * np.pi", "ph = np.exp(2j * np.pi"),
    "shift_half_frequencies": ("f = np.fft.fftfreq(M)", "f = np.fft.fftfreq(M) / 2"),
    "shift_adjoint_same_sign": ("shift_probe(t[j], -dy, -dx)", "shift_probe(t[j], dy, dx)"),
    "subpixel_corner_floor": ("p = np.floor_divide(q + S // 2, S)", "p = np.floor_divide(q, S)"),
    "subpixel_truncate": ("q = np.rint(S * np.asarray(positions, dtype=np.float64)).astype(np.int64)",
                          "q = np.trunc(S * np.asarray(positions, dtype=np.float64)).astype(np.int64)"),
    "subpixel_den_unshifted": ("w = np.sum(np.abs(position_probes(P, delta)) ** 2, axis=1)",
                               "w = np.sum(np.abs(position_probes(P, None)) ** 2, axis=1)"),
    "subpixel_steps_unshifted_dP": ("b = Oj[j][None] * dPj[i]", "b = Oj[j][None] * dP"),
    "subpixel_steps_unshifted_P": ("a = Pj[i] * dOj[j][None]", "a = P * dOj[j][None]"),
    "subpixel_dm_phi_unshifted": ("phi = exit_waves(O, P, pos, delta)\n    psi = psi",
                                  "phi = exit_waves(O, P, pos)\n    psi = psi"),
    "subpixel_cg_unshifted_operator": ("out += shift_probe(D[j][None] * shift_probe(X, dy, dx), -dy, -dx)",
                                       "out += D[j][None] * X"),
    "subpixel_cg_step_sign": ("        X = X + a * p\n", "        X = X - a * p\n"),
    "subpixel_cg_no_conjugation": ("        p = z + b * p\n", "        p = z\n"),
    "subpixel_dm_diagonal_probe": ("    if update_probe and delta is not None:", "    if False:"),
    "posref_forward_difference": ("return (Op[2:, 1:-1] - Op[:-2, 1:-1]) / 2.0,", "return (Op[2:, 1:-1] - Op[1:-1, 1:-1]),"),
    "posref_sign": ("return np.asarray(positions, dtype=np.float64) + step * np.clip",
                    "return np.asarray(positions, dtype=np.float64) - step * np.clip"),
    "posref_xy_swapped": ("Gy, Gx = gather(gy, pos, M), gather(gx, pos, M)", "Gy, Gx = gather(gx, pos, M), gather(gy, pos, M)"),
    "posref_unshifted_probe": ("Pk = Pj[0 if delta is None else j]", "Pk = P"),
    "poisson_residual_minus_phi": ("return ifft2(poisson_correction(fft2(phi), to_fft_order(I)))",
                                   "return ifft2(poisson_correction(fft2(phi), to_fft_order(I))) - phi"),
}


def _mutant(name: str) -> types.ModuleType:
    old, new = MUTATIONS[name]
    assert SRC.count(old) == 1, f"mutation {name}: pattern not found exactly once"
    spec = importlib.util.spec_from_loader(f"oracle_mutant_{name}", loader=None)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(SRC.replace(old, new), f"<mutant {name}>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_some_pin_catches(name):
    mod = _mutant(name)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(mod)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught the planted mistake {name}"

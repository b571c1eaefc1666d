"""The oracle's pins have teeth: plant one plausible mistake at a time in a
copy of the oracle's source (on the CPU), and check that some pin fails."""
import os
import types

import pytest

import oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "rid_oracle.py")

# (name, original text, planted mistake, pins expected to catch it)
MUTATIONS = [
    ("philox_hi_lo_swap", "x0, x1, x2, x3 = hi1 ^ x1", "x0, x1, x2, x3 = lo1 ^ x1", [pins.pin_philox_kat]),
    ("philox_no_key_bump", "k0 = (k0 + _PHILOX_W0) & _MASK32", "k0 = k0", [pins.pin_philox_kat]),
    ("uniform_wrong_shift", "a = (w[..., 0] >> np.uint64(5))", "a = (w[..., 0] >> np.uint64(6))",
     [pins.pin_uniform53]),
    ("box_muller_variance", "rho = np.sqrt(-np.log(u1))", "rho = np.sqrt(-2.0 * np.log(u1))",
     [pins.pin_gaussian_distribution]),
    ("box_muller_angle", "theta = 2.0 * np.pi * u2", "theta = np.pi * u2", [pins.pin_gaussian_distribution]),
    ("sketch_conjugated", "return Omega @ A", "return Omega.conj() @ A", [pins.pin_randomize_exact]),
    ("reflector_sign", "beta = -nrm if alphr >= 0.0 else nrm", "beta = nrm if alphr >= 0.0 else -nrm",
     [pins.pin_qr_lapack]),
    ("reflector_tau_conj", "tau = complex((beta - alphr) / beta, -alphi / beta)",
     "tau = complex((beta - alphr) / beta, alphi / beta)", [pins.pin_qr_lapack]),
    ("update_tau_not_conj", "C -= np.conj(tau_j) * np.outer(v, w)", "C -= tau_j * np.outer(v, w)",
     [pins.pin_qr_lapack]),
    ("update_v_not_conj", "w = v.conj() @ C", "w = v @ C", [pins.pin_qr_lapack]),
    ("norm_dropped_term", "nu = np.sum(tail.real * tail.real + tail.imag * tail.imag, axis=0)",
     "nu = np.sum(tail.real * tail.real, axis=0)", [pins.pin_qr_lapack]),
    ("pivot_last_max", "p = j + int(np.argmax(nu))",
     "p = j + (len(nu) - 1 - int(np.argmax(nu[::-1])))", [pins.pin_qr_pivot_rule]),
    ("no_pivoting", "p = j + int(np.argmax(nu))", "p = j", [pins.pin_qr_lapack]),
    ("solve_sign", "T[i, :] = (R2[i, :] - R1[i, i + 1:] @ T[i + 1:, :]) / R1[i, i]",
     "T[i, :] = (R2[i, :] + R1[i, i + 1:] @ T[i + 1:, :]) / R1[i, i]", [pins.pin_factor_r]),
    ("solve_transposed", "T[i, :] = (R2[i, :] - R1[i, i + 1:] @ T[i + 1:, :]) / R1[i, i]",
     "T[i, :] = (R2[i, :] - R1[i + 1:, i] @ T[i + 1:, :]) / R1[i, i]", [pins.pin_factor_r]),
    ("P_conjugated", "P[:, perm[k:]] = T", "P[:, perm[k:]] = T.conj()", [pins.pin_factor_r]),
    ("probe_sign", "w[J, :] = -(T @ omega[Jc, :])", "w[J, :] = (T @ omega[Jc, :])", [pins.pin_error_estimate]),
    ("upper_constant", "upper = float(10.0 * math.sqrt(2.0 / math.pi) * np.max(e_norm))",
     "upper = float(0.1 * math.sqrt(2.0 / math.pi) * np.max(e_norm))", [pins.pin_error_estimate]),
    ("left_probe_conjugated", "Z = G @ E", "Z = G.conj() @ E", [pins.pin_error_estimate_left]),
    ("left_probe_wrong_norm", "g_norm = np.sqrt(np.sum(G.real ** 2 + G.imag ** 2, axis=1))",
     "g_norm = np.sqrt(np.sum(G.real ** 2, axis=1))", [pins.pin_error_estimate_left]),
    ("left_probe_P_not_applied", "E = A - A[:, np.asarray(perm)[:k]] @ P", "E = A - A[:, np.asarray(perm)[:k]] @ P.conj()",
     [pins.pin_error_estimate_left]),
    ("round_ties_up", "re = np.ldexp(np.clip(np.rint(np.ldexp(row.real, bits - E)), -top, top), E - bits)",
     "re = np.ldexp(np.clip(np.floor(np.ldexp(row.real, bits - E) + 0.5), -top, top), E - bits)",
     [pins.pin_round_test_matrix]),
    ("round_no_clamp", "top = 2.0 ** bits - 1.0", "top = 2.0 ** bits", [pins.pin_round_test_matrix]),
    ("round_coarse_exponent", "E = int(np.max(np.frexp(nz)[1]))", "E = int(np.max(np.frexp(nz)[1])) + 1",
     [pins.pin_round_test_matrix]),
    ("srft_phase_sign", "DA = np.exp(2j * np.pi * phi)[:, None] * A", "DA = np.exp(-2j * np.pi * phi)[:, None] * A",
     [pins.pin_srft]),
    ("srft_dft_sign", "F_rows = np.exp(-2j * np.pi * (jk / m))", "F_rows = np.exp(2j * np.pi * (jk / m))",
     [pins.pin_srft]),
    ("srft_phase_half_range", "    return phi, s\n", "    return phi * 0.5, s\n", [pins.pin_srft_distribution]),
    ("srft_sample_biased", "s = np.minimum(np.floor(u * m)", "s = np.minimum(np.floor(u * u * m)",
     [pins.pin_srft_distribution]),
    ("srft_sample_drops_last", "s = np.minimum(np.floor(u * m)", "s = np.minimum(np.floor(u * (m - 1))",
     [pins.pin_srft_distribution]),
    ("srft_phase_omega_stream", "    ctr[:, 2] = 0\n    ctr[:, 3] = STREAM_SRFT", "    ctr[:, 2] = 0\n    ctr[:, 3] = STREAM_OMEGA",
     [pins.pin_srft_distribution]),
]


def mutated_oracle(old, new):
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = SRC
    exec(compile(src.replace(old, new, 1), SRC, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name,old,new,catchers", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, old, new, catchers):
    mutant = mutated_oracle(old, new)
    caught = []
    for pin in catchers:
        try:
            pin(mutant)
        except Exception:          # an assertion or a downstream failure both count
            caught.append(pin.__name__)
    assert caught, f"planted mistake {name!r} passed every pin"

"""The oracle's pins bind: each plausible mistake below (a dropped factor, a
wrong sign, an order off by one, a missing conjugate, a stale value), planted
in the oracle on the CPU by replacing one function, makes the named pin of
tests/test_oracle_pins.py fail.  The oracle itself is untouched outside each
test (monkeypatch restores it)."""
import math

import pytest
import torch

import test_oracle_pins as P
from oracle import afqmc_ref as R

CT = torch.complex128


def _split1_one_half_step(orig):
    def bad(B, A, psi, method, k, spins=None):       # B once instead of B B after e^A
        return B.to(CT) @ R.expm_action(A, psi, method, k, spins)
    return bad


def _ratio_mutant(change):
    """Replace propagate_and_ratio by one whose outputs pass through `change`
    (called with the original's arguments and its output tuple)."""
    def make(orig):
        def bad(*args, **kw):
            return change(args, orig(*args, **kw))
        return bad
    return make


def _with(out, **repl):
    names = ("psi", "logovl", "log_ratio", "log_I", "f", "f_raw")
    return tuple(repl.get(n, v) for n, v in zip(names, out))


def _lanczos_two_term(orig):
    """Lanczos column without the beta_{j-1} v_{j-1} term of the recurrence."""
    def bad(A, psi_col, k, normA, f=None):
        beta = torch.sqrt((psi_col * psi_col).sum())
        kk = min(k, A.shape[-1])
        V, alpha, off = [psi_col / beta], [], []
        for j in range(kk):
            w = A @ V[j]
            alpha.append((V[j] * w).sum())
            w = w - alpha[j] * V[j]
            if j + 1 < kk:
                off.append(torch.sqrt((w * w).sum()))
                V.append(w / off[j])
        T = R._tridiagonal(alpha, off)
        y = (torch.linalg.matrix_exp(T) if f is None else f(T))[:, 0] * beta
        return sum(y[i] * V[i] for i in range(len(alpha))), len(alpha)
    return bad


def _tridiagonal_lower_only(orig):
    def bad(alpha, beta):
        T = orig(alpha, beta)
        return torch.tril(T)
    return bad


# arguments of propagate_and_ratio: (ham, psi, logovl, x, tau, method, k, B, L_bar, ec, ...)
_STEP_MUTANTS = [
    ("step: importance factor with the wrong sign",
     lambda a, o: _with(o, log_I=-o[3])),
    ("step: importance factor without the 1/2",
     lambda a, o: _with(o, log_I=o[3] - 0.5 * (o[4] * o[4]).sum(-1))),
    ("step: scalar s from x instead of c = x - f",
     lambda a, o: _with(o, log_ratio=o[2] - 1j * math.sqrt(a[4]) * (o[4] @ a[8].to(CT)))),
    ("step: scalar s with +i sqrt(tau) c.L_bar",
     lambda a, o: _with(o, log_ratio=o[2] + 2j * math.sqrt(a[4])
                        * ((torch.as_tensor(a[3]).to(CT) - o[4]) @ a[8].to(CT)))),
    ("step: scalar s with +tau E_c'",
     lambda a, o: _with(o, log_ratio=o[2] + 2 * a[4] * a[9])),
]

# (mistake, oracle function, replacement built from the original, pin that must fail)
MUTATIONS = [
    ("Taylor order one short", "taylor_action",
     lambda o: lambda A, psi, k: o(A, psi, max(k - 1, 0)), "test_taylor_order_zero_and_one"),
    ("Chebyshev c_n without the factor 2", "chebyshev_coefficients",
     lambda o: lambda k: torch.cat([o(k)[:1], o(k)[1:] / 2]),
     "test_chebyshev_coefficients_are_the_modified_bessel_values"),
    ("Chebyshev order one short", "chebyshev_action",
     lambda o: lambda A, psi, k: o(A, psi, max(k - 1, 0)),
     "test_chebyshev_action_converges_to_matrix_exp_within_its_bound"),
    ("Krylov without ||psi||", "krylov_action",
     lambda o: lambda A, psi, k: o(A, psi, k) / torch.linalg.vector_norm(psi, dim=-2, keepdim=True),
     "test_krylov_full_dimension_is_exact"),
    ("Krylov dimension one short", "krylov_action",
     lambda o: lambda A, psi, k: o(A, psi, max(k - 1, 1)), "test_krylov_full_dimension_is_exact"),
    ("Lanczos with the Hermitian inner product", "_bilinear",
     lambda o: lambda u, v: torch.vdot(u, v), "test_lanczos_full_dimension_is_exact"),
    ("Lanczos without (psi^T psi)^(1/2)", "lanczos_action",
     lambda o: lambda A, psi, k, f=None: o(A, psi, k, f) / torch.sqrt((psi * psi).sum(-2, keepdim=True)),
     "test_lanczos_full_dimension_is_exact"),
    ("Lanczos dimension one short", "lanczos_action",
     lambda o: lambda A, psi, k, f=None: o(A, psi, max(k - 1, 1), f), "test_lanczos_full_dimension_is_exact"),
    ("Lanczos tridiagonal without its upper diagonal", "_tridiagonal", _tridiagonal_lower_only,
     "test_lanczos_is_exact_for_polynomials_below_the_dimension"),
    ("Lanczos recurrence without the beta_{j-1} v_{j-1} term", "_lanczos_column", _lanczos_two_term,
     "test_lanczos_is_the_bilinear_projection_on_the_krylov_space"),
    ("block Krylov one block short", "block_krylov_action",
     lambda o: lambda A, psi, k, spins=None: o(A, psi, max(k - 1, 1), spins),
     "test_block_krylov_full_space_is_exact"),
    ("exact action of -A", "exact_action",
     lambda o: lambda A, psi: o(-A, psi), "test_exact_action_matches_matrix_exp"),
    ("half step e^{-tau h''}", "half_step_propagator",
     lambda o: lambda hpp, tau: o(hpp, 2 * tau), "test_half_step_squares_to_one_body_exponential"),
    ("field matrix sign", "field_matrix",
     lambda o: lambda ham, c, tau: -o(ham, c, tau), "test_first_step_from_trial_closed_form"),
    ("field matrix without the i", "field_matrix",
     lambda o: lambda ham, c, tau: -1j * o(ham, c, tau),
     "test_hubbard_stratonovich_average_of_the_field_propagator"),
    ("field matrix with sqrt(2 tau)", "field_matrix",
     lambda o: lambda ham, c, tau: o(ham, c, 2 * tau),
     "test_hubbard_stratonovich_average_of_the_field_propagator"),
    ("Split-1 with one half step", "split1_propagate", _split1_one_half_step,
     "test_split1_error_is_half_the_commutator"),
    ("Taylor propagator without tau on h''", "taylor_propagate",
     lambda o: lambda hpp, A, psi, tau, k: o(hpp / tau, A, psi, tau, k),
     "test_taylor_propagator_expands_the_whole_exponent"),
    ("Crank-Nicolson factors swapped", "crank_nicolson_propagate",
     lambda o: lambda hpp, A, psi, tau: o(-hpp, -A, psi, tau), "test_crank_nicolson_pade_error"),
    ("h'' without the mean-field shift", "propagation_h1",
     lambda o: lambda ham, L_bar=None: o(ham, 0 * R.mean_field_shift(ham)),
     "test_propagation_h1_reproduces_one_electron_hamiltonian"),
    ("mean-field shift halved", "mean_field_shift",
     lambda o: lambda ham: 0.5 * o(ham), "test_mean_field_shift_closed_form"),
    ("force bias sign", "force_bias",
     lambda o: lambda ham, psi, tau, L_bar=None: (lambda f, fr: (-f, fr))(*o(ham, psi, tau, L_bar)),
     "test_force_bias_capping_removes_components"),
    ("Theta of the conjugate walker", "theta",
     lambda o: lambda t, p: o(t, p.conj()), "test_mixed_expectation_is_derivative_of_log_overlap"),
    ("log-overlap conjugated", "log_overlap",
     lambda o: lambda ham, psi: o(ham, psi).conj(), "test_log_overlap_closed_form_small_dets"),
    ("stale log-overlap after QR", "reorthonormalise",
     lambda o: lambda ham, psi: (o(ham, psi)[0], R.log_overlap(ham, psi)),
     "test_log_overlap_after_qr_shifts_by_log_det_R"),
    ("MGS columns not normalised", "mgs_qr",
     lambda o: lambda X: (lambda q, r: (2 * q, r / 2))(*o(X)), "test_mgs_qr_against_library_qr"),
    ("local energy of the conjugate walker", "local_energy",
     lambda o: lambda ham, psi: o(ham, psi.conj()), "test_local_energy_matches_bruteforce_for_general_walker"),
    ("energy window four times too wide", "energy_window",
     lambda o: lambda e, e0, tau, n: o(e, e0, tau, 4 * n), "test_energy_window_values"),
    ("energy window centred at 0", "energy_window",
     lambda o: lambda e, e0, tau, n: o(e, 0.0, tau, n), "test_energy_window_values"),
    ("weight update with -E_0", "weight_update",
     lambda o: lambda W, lr, li, tau, e0: o(W, lr, li, tau, -e0), "test_weight_real_positive_special_case"),
    ("phase of the overlap ratio conjugated", "weight_update",
     lambda o: lambda W, lr, li, tau, e0: o(W, lr.conj(), li, tau, e0), "test_weight_caps"),
    ("importance factor dropped", "weight_update",
     lambda o: lambda W, lr, li, tau, e0: o(W, lr, 0 * li, tau, e0), "test_weight_real_positive_special_case"),
    ("importance factor doubled", "weight_update",
     lambda o: lambda W, lr, li, tau, e0: o(W, lr, 2 * li, tau, e0), "test_weight_real_positive_special_case"),
    ("mixed estimate without weights", "mixed_energy",
     lambda o: lambda W, e: o((W > 0).to(W.dtype), e), "test_mixed_energy_ignores_dead_walkers"),
    ("comb teeth shifted by half a spacing", "comb",
     lambda o: lambda W, u: o(W, (u + 0.5) % 1.0), "test_comb_example"),
]
MUTATIONS += [(m, "propagate_and_ratio", _ratio_mutant(ch),
               "test_importance_sampled_step_keeps_the_gaussian_average") for m, ch in _STEP_MUTANTS]


@pytest.mark.parametrize("mistake,name,make,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pin(monkeypatch, mistake, name, make, pin):
    getattr(P, pin)()                                  # the pin passes on the oracle as it is
    monkeypatch.setattr(R, name, make(getattr(R, name)))
    with pytest.raises(AssertionError):
        getattr(P, pin)()

"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every oracle function is checked here against something other than itself:
library routines (matrix_exp, eigh, qr, det), closed forms, invariants,
special cases, brute-force FCI (second quantisation, in fci_bruteforce.py) and
finite differences.  No GPU is needed.
"""
import math

import numpy as np
import pytest
import torch

import fci_bruteforce as fci
from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import make_fields, make_system

CT = torch.complex128
RT = torch.float64


def _rand_c(gen, *shape):
    return (torch.randn(*shape, generator=gen, dtype=RT)
            + 1j * torch.randn(*shape, generator=gen, dtype=RT)).to(CT)


def _small_ham(N=6, n=2, G=10, rho=0.6, seed=3, lambda0=1.0):
    s = make_system(N, n, n, G, rho=rho, seed=seed, lambda0=lambda0)
    return s, R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb, s.e_const)


# ---------------------------------------------------------------- exponentials
def test_taylor_within_truncation_bound():
    """Eq. taylor: ||taylor_k - e^A psi|| <= ||A||^{k+1} e^{||A||} / (k+1)! ||psi||."""
    g = torch.Generator().manual_seed(1)
    for N in (4, 6, 8):
        A = 0.3 * _rand_c(g, N, N)
        psi = _rand_c(g, N, 3)
        ref = torch.linalg.matrix_exp(A) @ psi
        nA = float(torch.linalg.matrix_norm(A, ord=2))
        for k in (2, 4, 6, 10):
            err = float(torch.linalg.matrix_norm(R.taylor_action(A, psi, k) - ref, ord=2))
            bound = nA ** (k + 1) * math.exp(nA) / math.factorial(k + 1) * float(
                torch.linalg.matrix_norm(psi, ord=2))
            assert err <= bound * (1 + 1e-9) + 1e-14


def test_taylor_order_zero_and_one():
    g = torch.Generator().manual_seed(2)
    A = _rand_c(g, 5, 5)
    psi = _rand_c(g, 5, 2)
    assert torch.equal(R.taylor_action(A, psi, 0), psi)
    assert torch.allclose(R.taylor_action(A, psi, 1), psi + A @ psi, atol=1e-15)


def test_chebyshev_coefficients_are_the_modified_bessel_values():
    """Sec. IV.B: J_0(i) = I_0(1) and 2 i^n J_n(-i) = 2 I_n(1), real; tabulated
    I_0(1) = 1.266065878, I_1(1) = 0.565159104, I_2(1) = 0.135747670
    (Abramowitz and Stegun, Table 9.8), and the power series
    I_n(1) = sum_m (1/2)^{2m+n} / (m! (m+n)!)."""
    c = R.chebyshev_coefficients(12)
    assert float(c.imag.abs().max()) < 1e-15
    assert abs(float(c[0].real) - 1.266065878) < 1e-9
    assert abs(float(c[1].real) - 2 * 0.565159104) < 2e-9
    assert abs(float(c[2].real) - 2 * 0.135747670) < 2e-9
    for n in range(13):
        i_n = sum(0.5 ** (2 * m + n) / (math.factorial(m) * math.factorial(m + n)) for m in range(30))
        assert abs(float(c[n].real) - (i_n if n == 0 else 2 * i_n)) < 1e-15 * max(1.0, i_n)


def test_chebyshev_series_of_a_scalar_is_the_exponential():
    """sum_n c_n T_n(x) = e^x with T_n(cos t) = cos(n t) (Eq. chebpoly) for x in
    [-1, 1], and at complex x by the action on a 1 x 1 matrix."""
    for x in (-1.0, -0.3, 0.0, 0.5, 1.0):
        t = math.acos(x)
        c = R.chebyshev_coefficients(25).real
        val = sum(float(c[n]) * math.cos(n * t) for n in range(26))
        assert abs(val - math.exp(x)) < 1e-14
        one = R.chebyshev_action(torch.tensor([[x]], dtype=CT), torch.ones(1, 1, dtype=CT), 25)
        assert abs(complex(one[0, 0]) - math.exp(x)) < 1e-14
    z = 0.2 + 0.7j
    one = R.chebyshev_action(torch.tensor([[z]], dtype=CT), torch.ones(1, 1, dtype=CT), 30)
    assert abs(complex(one[0, 0]) - complex(np.exp(z))) < 1e-14


def test_chebyshev_action_converges_to_matrix_exp_within_its_bound():
    """For Hermitian A with spectrum in [-1, 1], |T_n| <= 1 there, so
    ||cheb_k - e^A psi|| <= sum_{n>k} |c_n| ||psi||; at high order it is
    matrix_exp(A) psi for general complex A of small norm; at equal order it
    beats the Taylor series on [-1, 1] (the smaller error prefactor of Sec. IV.B)."""
    g = torch.Generator().manual_seed(7)
    N = 8
    H = _rand_c(g, N, N)
    H = 0.5 * (H + H.conj().T)
    H = H / float(torch.linalg.eigvalsh(H).abs().max())
    psi = _rand_c(g, N, 3)
    ref = torch.linalg.matrix_exp(H) @ psi
    tail = R.chebyshev_coefficients(40).abs()
    for k in (2, 4, 6, 8):
        err = float(torch.linalg.vector_norm(R.chebyshev_action(H, psi, k) - ref))
        bound = float(tail[k + 1:].sum()) * float(torch.linalg.vector_norm(psi))
        assert err <= bound
        assert err < float(torch.linalg.vector_norm(R.taylor_action(H, psi, k) - ref))
    A = 0.3 * _rand_c(g, N, N)
    got = R.chebyshev_action(A, psi, 30)
    want = torch.linalg.matrix_exp(A) @ psi
    assert float((got - want).abs().max()) < 1e-13


def test_exact_action_matches_matrix_exp():
    g = torch.Generator().manual_seed(3)
    A = _rand_c(g, 7, 7)
    psi = _rand_c(g, 7, 3)
    ref = torch.linalg.matrix_exp(A) @ psi
    assert torch.allclose(R.exact_action(A, psi), ref, rtol=1e-10, atol=1e-10)


def test_krylov_full_dimension_is_exact():
    """k = N: the Krylov space is the whole space, so e^A psi is exact to roundoff."""
    g = torch.Generator().manual_seed(4)
    for N in (3, 5, 8):
        A = 0.5 * _rand_c(g, N, N)
        psi = _rand_c(g, N, 2)
        ref = torch.linalg.matrix_exp(A) @ psi
        out = R.krylov_action(A, psi, N)
        assert torch.allclose(out, ref, rtol=1e-11, atol=1e-12)
        # k > N is clamped to N
        assert torch.allclose(R.krylov_action(A, psi, N + 3), ref, rtol=1e-11, atol=1e-12)


def test_krylov_eigenvector_exact_at_k1():
    """psi an eigenvector of A: K_1 is invariant and krylov_1 = e^lambda psi."""
    g = torch.Generator().manual_seed(5)
    N = 6
    A = _rand_c(g, N, N)
    lam, V = torch.linalg.eig(A)
    psi = V[:, :2] * 3.0
    out = R.krylov_action(A, psi, 1)
    assert torch.allclose(out, psi * torch.exp(lam[:2])[None, :], rtol=1e-10, atol=1e-12)
    # and a higher k detects the invariant subspace (happy breakdown) without harm
    out5 = R.krylov_action(A, psi, 5)
    assert torch.allclose(out5, psi * torch.exp(lam[:2])[None, :], rtol=1e-9, atol=1e-11)


def test_krylov_error_decreases_with_k():
    g = torch.Generator().manual_seed(6)
    N = 12
    A = 0.15 * _rand_c(g, N, N)
    psi = _rand_c(g, N, 1)
    ref = torch.linalg.matrix_exp(A) @ psi
    errs = [float((R.krylov_action(A, psi, k) - ref).norm()) for k in range(1, 10)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6 * float(ref.norm())


def test_krylov_hessenberg_projection():
    """Eq. projham: B_k^dagger A B_k = A_k; checked by recomputing the projection
    from the returned basis of a single column via the Arnoldi relation
    A B_k = B_{k+1} H_{k+1,k} (exact arithmetic identity)."""
    g = torch.Generator().manual_seed(7)
    N, k = 9, 4
    A = _rand_c(g, N, N)
    psi = _rand_c(g, N, 1)[:, 0]
    # run the oracle's per-column routine with k and k+1 and compare the
    # Krylov result to a direct projection computed with an orthonormal basis
    # of span{psi, A psi, ..., A^{k-1} psi} from a library QR
    K = torch.stack([torch.linalg.matrix_power(A, j) @ psi for j in range(k)], 1)
    Q, _ = torch.linalg.qr(K)
    Ak = Q.conj().T @ A @ Q
    e1 = Q.conj().T @ psi
    ref = Q @ (torch.linalg.matrix_exp(Ak) @ e1)
    out = R.krylov_action(A, psi[:, None], k)[:, 0]
    assert torch.allclose(out, ref, rtol=1e-9, atol=1e-11)


def _rand_csym(g, N, scale):
    X = _rand_c(g, N, N)
    return scale * 0.5 * (X + X.T)


def test_lanczos_full_dimension_is_exact():
    """Reading R30, k = N: the Lanczos space is the whole space and V_N is
    complex orthogonal, so V_N e^{T_N} V_N^T psi = e^A psi to roundoff."""
    g = torch.Generator().manual_seed(40)
    for N in (3, 5, 8):
        A = _rand_csym(g, N, 0.5)
        psi = _rand_c(g, N, 2)
        ref = torch.linalg.matrix_exp(A) @ psi
        assert torch.allclose(R.lanczos_action(A, psi, N), ref, rtol=1e-10, atol=1e-11)
        assert torch.allclose(R.lanczos_action(A, psi, N + 2), ref, rtol=1e-10, atol=1e-11)


def test_lanczos_is_exact_for_polynomials_below_the_dimension():
    """Any polynomial p of degree <= k - 1: V_k p(T_k) e_1 beta = p(A) psi
    (the Krylov space of Eq. krylovsub holds p(A) psi and the bilinear
    projection reproduces it), at every k."""
    g = torch.Generator().manual_seed(41)
    N = 10
    A = _rand_csym(g, N, 0.4)
    psi = _rand_c(g, N, 3)
    for k in (1, 2, 4, 7):
        coef = _rand_c(g, k, 1)[:, 0]

        def p(M):
            out = torch.zeros_like(M)
            P = torch.eye(M.shape[0], dtype=CT)
            for c in coef:
                out = out + c * P
                P = P @ M
            return out
        ref = p(A) @ psi
        assert torch.allclose(R.lanczos_action(A, psi, k, f=p), ref, rtol=1e-10, atol=1e-11), k


def test_lanczos_is_the_bilinear_projection_on_the_krylov_space():
    """With the power basis K = [psi, A psi, ..., A^{k-1} psi] and its
    bilinear Gram matrix K^T K, lanczos_k = K exp((K^T K)^{-1} K^T A K) e_1
    (the same space and projection written without the recurrence; library
    solve and matrix_exp)."""
    g = torch.Generator().manual_seed(42)
    N, k = 9, 4
    A = _rand_csym(g, N, 0.6)
    psi = _rand_c(g, N, 1)[:, 0]
    K = torch.stack([torch.linalg.matrix_power(A, j) @ psi for j in range(k)], 1)
    M = torch.linalg.solve(K.T @ K, K.T @ A @ K)
    e1 = torch.zeros(k, dtype=CT)
    e1[0] = 1.0
    ref = K @ (torch.linalg.matrix_exp(M) @ e1)
    out = R.lanczos_action(A, psi[:, None], k)[:, 0]
    assert torch.allclose(out, ref, rtol=1e-8, atol=1e-10)
    # and it is not the Hermitian (Arnoldi) projection for a complex A
    arn = R.krylov_action(A, psi[:, None], k)[:, 0]
    assert float((arn - out).abs().max()) > 1e-6 * float(out.abs().max())


def test_lanczos_equals_arnoldi_for_real_symmetric_matrices():
    """A real symmetric and psi real: the bilinear and Hermitian forms agree,
    so Lanczos and Arnoldi build the same basis and projected matrix."""
    g = torch.Generator().manual_seed(43)
    N = 11
    X = torch.randn(N, N, dtype=torch.float64, generator=g)
    A = (0.2 * (X + X.T)).to(CT)
    psi = torch.randn(N, 3, dtype=torch.float64, generator=g).to(CT)
    for k in (2, 5, 8):
        assert torch.allclose(R.lanczos_action(A, psi, k), R.krylov_action(A, psi, k), rtol=1e-11, atol=1e-12)


def test_lanczos_error_decreases_with_k():
    g = torch.Generator().manual_seed(44)
    N = 12
    A = _rand_csym(g, N, 0.3)
    psi = _rand_c(g, N, 1)
    ref = torch.linalg.matrix_exp(A) @ psi
    errs = [float((R.lanczos_action(A, psi, k) - ref).norm()) for k in range(1, 10)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6 * float(ref.norm())


def test_block_krylov_full_space_is_exact():
    """k n = N (Eq. bkrylov): the block Krylov space is the whole space, so the
    action is e^A X to roundoff, for each spin block separately."""
    g = torch.Generator().manual_seed(41)
    for N, na, nb in ((6, 2, 3), (8, 4, 2), (9, 3, 3)):
        A = 0.4 * _rand_c(g, N, N)
        X = _rand_c(g, N, na + nb)
        ref = torch.linalg.matrix_exp(A) @ X
        spins = (slice(0, na), slice(na, na + nb))
        out = torch.empty_like(X)
        for sl in spins:
            n = sl.stop - sl.start
            out[:, sl] = R.block_krylov_action(A, X[:, sl], N // n)
        assert torch.allclose(out, ref, rtol=1e-11, atol=1e-12)
        # the spin-split call gives the same, and more blocks than N // n are clamped
        assert torch.allclose(R.block_krylov_action(A, X, N, spins), ref, rtol=1e-11, atol=1e-12)


def test_block_krylov_one_column_is_krylov():
    """n = 1: the block algorithm is the column Arnoldi of Eq. krylov."""
    g = torch.Generator().manual_seed(42)
    N = 10
    A = 0.3 * _rand_c(g, N, N)
    x = _rand_c(g, N, 1)
    for k in (1, 3, 6):
        assert torch.allclose(R.block_krylov_action(A, x, k), R.krylov_action(A, x, k), rtol=1e-12, atol=1e-13)


def test_block_krylov_is_a_projection_on_the_block_krylov_space():
    """bkrylov_k = Q e^{Q^dagger A Q} Q^dagger X for any orthonormal basis Q of
    span{X, A X, .., A^{k-1} X}; Q here from a library QR of those blocks."""
    g = torch.Generator().manual_seed(43)
    N, n, k = 14, 3, 3
    A = 0.5 * _rand_c(g, N, N)
    X = _rand_c(g, N, n)
    K = torch.cat([torch.linalg.matrix_power(A, j) @ X for j in range(k)], 1)
    Q, _ = torch.linalg.qr(K)
    ref = Q @ (torch.linalg.matrix_exp(Q.conj().T @ A @ Q) @ (Q.conj().T @ X))
    assert torch.allclose(R.block_krylov_action(A, X, k), ref, rtol=1e-9, atol=1e-11)


def test_block_krylov_equivariance_and_convergence():
    """The block Krylov space depends on span(X) only, so bkrylov(X M) =
    bkrylov(X) M for invertible M; the error against e^A X falls with k."""
    g = torch.Generator().manual_seed(44)
    N, n = 16, 4
    A = 0.3 * _rand_c(g, N, N)
    X = _rand_c(g, N, n)
    M = _rand_c(g, n, n) + 2.0 * torch.eye(n, dtype=CT)
    for k in (1, 2, 3):
        assert torch.allclose(R.block_krylov_action(A, X @ M, k), R.block_krylov_action(A, X, k) @ M,
                              rtol=1e-10, atol=1e-11)
    ref = torch.linalg.matrix_exp(A) @ X
    errs = [float((R.block_krylov_action(A, X, k) - ref).norm()) for k in range(1, 5)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-12 * float(ref.norm())   # k = 4 = N / n: exact


# ---------------------------------------------------------------- other propagators (Sec. III)
def _sym(g, N, scale):
    X = torch.randn(N, N, dtype=RT, generator=g)
    return scale * 0.5 * (X + X.T)


def test_split1_error_is_half_the_commutator():
    """Split-1 (Sec. III): e^{-tau H1} e^{-tau M} = e^{-tau (H1 + M)} + tau^2/2 [H1, M]
    + O(tau^3), the paper's leading term E_S1 = [H1, H2]/2 for a deterministic
    interaction."""
    g = torch.Generator().manual_seed(51)
    N = 6
    H1, M = _sym(g, N, 1.0), _sym(g, N, 1.0)
    I = torch.eye(N, dtype=CT)
    comm = 0.5 * (H1 @ M - M @ H1).to(CT)
    for tau in (1e-2, 1e-3):
        B = R.half_step_propagator(H1, tau)
        U1 = R.split1_propagate(B, (-tau * M).to(CT), I, "exact", 0)
        U = torch.linalg.matrix_exp((-tau * (H1 + M)).to(CT))
        err = float(((U1 - U) / tau ** 2 - comm).norm() / comm.norm())
        assert err < 20 * tau, (tau, err)


def test_taylor_propagator_expands_the_whole_exponent():
    """The Taylor propagator expands e^{-tau (h'' + M)} directly: order 1 is
    1 - tau (h'' + M), a high order is the exponential."""
    g = torch.Generator().manual_seed(52)
    N, tau = 6, 0.1
    H1, M = _sym(g, N, 1.0), _sym(g, N, 1.0)
    psi = torch.randn(N, 3, dtype=RT, generator=g).to(CT)
    A = (-tau * M).to(CT)
    one = R.taylor_propagate(H1, A, psi, tau, 1)
    assert torch.allclose(one, psi - tau * ((H1 + M).to(CT) @ psi), rtol=1e-14, atol=1e-14)
    ref = torch.linalg.matrix_exp((-tau * (H1 + M)).to(CT)) @ psi
    assert torch.allclose(R.taylor_propagate(H1, A, psi, tau, 25), ref, rtol=1e-13, atol=1e-14)


def test_crank_nicolson_pade_error():
    """Crank-Nicolson (Sec. III) is the (1,1) Pade approximant of e^{-tau H}:
    U_CN - e^{-tau H} = -(tau H)^3 / 12 + O(tau^4) for a deterministic H = h'' + M."""
    g = torch.Generator().manual_seed(53)
    N = 5
    H1, M = _sym(g, N, 1.0), _sym(g, N, 1.0)
    H = (H1 + M).to(CT)
    I = torch.eye(N, dtype=CT)
    lead = -(H @ H @ H) / 12.0
    for tau in (1e-2, 1e-3):
        Ucn = R.crank_nicolson_propagate(H1, (-tau * M).to(CT), I, tau)
        U = torch.linalg.matrix_exp(-tau * H)
        err = float(((Ucn - U) / tau ** 3 - lead).norm() / lead.norm())
        assert err < 20 * tau, (tau, err)


def test_propagators_agree_without_interaction():
    """At Psi_T with zero fields the force bias and the field vanish (A = 0):
    Split-1 and Split-2 both give e^{-tau h''} Psi_T, the Taylor propagator of
    high order too, and Crank-Nicolson to O(tau^3)."""
    s, ham = _small_ham()
    tau = 0.05
    psi, lo, W = R.init_walkers(ham, 2)
    x = torch.zeros(2, ham.G, dtype=RT)
    out = {p: R.step(ham, psi, lo, W, x, tau, -5.0, method="exact", k=30, propagator=p)
           for p in ("split2", "split1", "taylor", "cn")}
    hpp, _ = R.propagation_h1(ham)
    ref = torch.linalg.matrix_exp((-tau * hpp).to(CT)) @ ham.trial.to(CT)
    for p in ("split2", "split1", "taylor"):
        assert torch.allclose(out[p][0][0], ref, rtol=1e-12, atol=1e-13), p
    d = float((out["cn"][0][0] - ref).norm() / ref.norm())
    assert d < tau ** 3 * float(torch.linalg.matrix_norm(hpp, 2)) ** 3, d
    with pytest.raises(ValueError):
        R.step(ham, psi, lo, W, x, tau, -5.0, propagator="split3")


# ---------------------------------------------------------------- propagator
def _gauss_average(ham, tau, nodes):
    """E_x[e^{A(x)}] over standard-normal fields x_g (one per Cholesky vector)
    by a tensor Gauss-Hermite rule (weight e^{-x^2/2}), A from field_matrix."""
    import itertools
    xs, ws = np.polynomial.hermite_e.hermegauss(nodes)
    ws = ws / ws.sum()
    acc = torch.zeros(ham.N, ham.N, dtype=CT)
    for idx in itertools.product(range(nodes), repeat=ham.G):
        c = torch.tensor([xs[i] for i in idx], dtype=CT)
        acc = acc + float(np.prod([ws[i] for i in idx])) * torch.linalg.matrix_exp(R.field_matrix(ham, c, tau))
    return acc


def test_hubbard_stratonovich_average_of_the_field_propagator():
    """Eq. hstrafo: the Gaussian average of e^{i sqrt(tau) sum_g x_g L_g} is
    e^{-tau/2 sum_g L_g^2}: exactly for one Cholesky vector, and up to O(tau^2)
    for two non-commuting ones (halving tau divides the error by about 4).  The
    tau^2 term is the one printed in Eq. hserror: with e^{-tau H_2} = average +
    tau^2 E_HS + O(tau^3) (Sec. III), (average - e^{-tau H_2}) / tau^2 tends to
    -E_HS, E_HS = 1/48 sum_{g != g'} {L_g L_g', [L_g', L_g]}
    + 1/24 sum_{g != g'} [L_g, [L_g, L_g'^2]], the residual shrinking like tau."""
    s1 = make_system(4, 1, 1, 1, rho=0.5, seed=21)
    ham1 = R.make_hamiltonian(s1.h1, s1.L, s1.trial, 1, 1)
    for tau in (0.05, 0.2):
        L = ham1.L[0].to(CT)
        want = torch.linalg.matrix_exp(-0.5 * tau * L @ L)
        got = _gauss_average(ham1, tau, 60)
        assert float((got - want).abs().max()) < 1e-12
    s2 = make_system(4, 1, 1, 2, rho=0.8, seed=22)
    ham2 = R.make_hamiltonian(s2.h1, s2.L, s2.trial, 1, 1)
    L2 = ham2.L.to(CT)
    comm = float((L2[0] @ L2[1] - L2[1] @ L2[0]).abs().max())
    assert comm > 1e-2                                   # the two vectors do not commute
    errs = []
    for tau in (0.1, 0.05, 0.025):
        want = torch.linalg.matrix_exp(-0.5 * tau * (L2[0] @ L2[0] + L2[1] @ L2[1]))
        errs.append(float((_gauss_average(ham2, tau, 24) - want).abs().max()))
    for a, b in zip(errs, errs[1:]):
        assert 3.2 < a / b < 4.8, errs

    def cm(a, b):
        return a @ b - b @ a
    E_hs = torch.zeros_like(L2[0])
    for g in range(2):
        for h in range(2):
            if g != h:
                E_hs = E_hs + (L2[g] @ L2[h] @ cm(L2[h], L2[g]) + cm(L2[h], L2[g]) @ L2[g] @ L2[h]) / 48 \
                    + cm(L2[g], cm(L2[g], L2[h] @ L2[h])) / 24
    res = []
    for tau in (0.01, 0.005):
        want = torch.linalg.matrix_exp(-0.5 * tau * (L2[0] @ L2[0] + L2[1] @ L2[1]))
        res.append(float(((_gauss_average(ham2, tau, 30) - want) / tau ** 2 + E_hs).abs().max()))
    assert res[0] < 0.01 * float(E_hs.abs().max())
    assert 1.7 < res[0] / res[1] < 2.3, res


def test_field_averaged_propagators_have_the_printed_tau2_errors():
    """Sec. III: averaged over the fields (Gauss-Hermite, two non-commuting
    Cholesky vectors), each propagator differs from U = e^{-tau (H_1 + H_2)},
    H_2 = 1/2 sum_g L_g^2, by tau^2 E + O(tau^3) with the leading terms the paper
    prints: Split-2 E_HS; Split-1 1/2 [H_1, H_2] + E_HS; Taylor propagator
    1/12 sum_g [[L_g, H_1], L_g] + E_HS; Crank-Nicolson 1/4 {H_1, H_2} +
    1/8 sum_g [[L_g, H_1], L_g] + its HS part.  E_HS enters with the sign of
    Eq. hstrafo (reading R26), and the Crank-Nicolson HS part is
    H_2^2 - 3 E_HS (reading R27).  (U_P - U) / tau^2 - E falls like tau."""
    s2 = make_system(4, 1, 1, 2, rho=0.8, seed=22)
    ham = R.make_hamiltonian(s2.h1, s2.L, s2.trial, 1, 1)
    L = ham.L.to(CT)
    g = torch.Generator().manual_seed(5)
    K = torch.randn(4, 4, generator=g, dtype=RT)
    K = 0.5 * (K + K.T)                                 # H_1, a one-body matrix
    Kc = K.to(CT)
    H2 = 0.5 * (L[0] @ L[0] + L[1] @ L[1])
    eye = torch.eye(4, dtype=CT)

    def cm(a, b):
        return a @ b - b @ a
    E_hs = sum((L[a] @ L[b] @ cm(L[b], L[a]) + cm(L[b], L[a]) @ L[a] @ L[b]) / 48
               + cm(L[a], cm(L[a], L[b] @ L[b])) / 24 for a in range(2) for b in range(2) if a != b)
    LHL = sum(cm(cm(L[a], Kc), L[a]) for a in range(2))
    import itertools
    xs, ws = np.polynomial.hermite_e.hermegauss(30)
    ws = ws / ws.sum()

    def average(prop, tau):
        acc = torch.zeros(4, 4, dtype=CT)
        for i, j in itertools.product(range(30), repeat=2):
            A = R.field_matrix(ham, torch.tensor([xs[i], xs[j]], dtype=CT), tau)
            acc = acc + float(ws[i] * ws[j]) * prop(A, tau)
        return acc
    cases = {
        "split2": (lambda A, t: R.split2_propagate(R.half_step_propagator(K, t), A, eye, "exact", 0), -E_hs),
        "split1": (lambda A, t: R.split1_propagate(R.half_step_propagator(K, t), A, eye, "exact", 0),
                   0.5 * cm(Kc, H2) - E_hs),
        "taylor": (lambda A, t: R.taylor_propagate(K, A, eye, t, 40), LHL / 12 - E_hs),
        "cn": (lambda A, t: R.crank_nicolson_propagate(K, A, eye, t),
               0.25 * (Kc @ H2 + H2 @ Kc) + LHL / 8 + H2 @ H2 - 3 * E_hs),
    }
    for name, (prop, E) in cases.items():
        res = []
        for tau in (0.01, 0.005):
            U = torch.linalg.matrix_exp(-tau * (Kc + H2))
            res.append(float(((average(prop, tau) - U) / tau ** 2 - E).abs().max()))
        assert res[0] < 0.1 * float(E.abs().max()), (name, res)
        assert 1.7 < res[0] / res[1] < 2.3, (name, res)


def test_half_step_squares_to_one_body_exponential():
    s, ham = _small_ham()
    hpp, _ = R.propagation_h1(ham)
    B = R.half_step_propagator(hpp, 0.07)
    assert torch.allclose(B, B.T, atol=1e-15)
    assert torch.allclose(B @ B, torch.linalg.matrix_exp(-0.07 * hpp), rtol=1e-12, atol=1e-13)


def test_split2_local_error_slope_three():
    """Deterministic one-body M: ||B e^{-tau M} B psi - e^{-tau(h''+M)} psi|| ~ tau^3."""
    s, ham = _small_ham()
    hpp, _ = R.propagation_h1(ham)
    g = torch.Generator().manual_seed(8)
    M = torch.randn(ham.N, ham.N, generator=g, dtype=RT)
    M = 0.5 * (M + M.T)
    psi = ham.trial.to(CT)
    taus = [0.04, 0.02, 0.01]
    errs = []
    for tau in taus:
        B = R.half_step_propagator(hpp, tau)
        out = R.split2_propagate(B, (-tau * M).to(CT), psi, "exact", 0)
        ref = torch.linalg.matrix_exp((-tau * (hpp + M)).to(CT)) @ psi
        errs.append(float((out - ref).norm()))
    slopes = [math.log(errs[i] / errs[i + 1]) / math.log(2) for i in range(2)]
    assert all(2.85 < sl < 3.15 for sl in slopes), slopes


def test_noninteracting_walk_closed_form():
    """L = 0: every step is B B = e^{-tau h}, so Psi_n = e^{-n tau h} Psi_T."""
    s = make_system(6, 2, 2, 4, rho=0.5, seed=5)
    ham = R.make_hamiltonian(s.h1, 0.0 * s.L, s.trial, 2, 2)
    psi, lo, W = R.init_walkers(ham, 3)
    tau, n = 0.1, 7
    x = torch.zeros(3, ham.G, dtype=RT)
    for _ in range(n):
        psi, lo, W, _ = R.step(ham, psi, lo, W, x, tau, 0.0, method="taylor", k=4)
    lam, V = np.linalg.eigh(s.h1)
    U = (V * np.exp(-n * tau * lam)) @ V.T
    ref = torch.as_tensor(U @ s.trial).to(CT)
    for w in range(3):
        assert torch.allclose(psi[w], ref, rtol=1e-12, atol=1e-13)


def test_propagation_h1_reproduces_one_electron_hamiltonian():
    """On one-electron states the two-body term vanishes, so h'' + 1/2 sum_g
    (L_g - L_bar_g)^2 + E_c' must equal h + E_const (reading R1)."""
    s, ham = _small_ham()
    Lbar = R.mean_field_shift(ham)
    hpp, ec = R.propagation_h1(ham, Lbar)
    eye = torch.eye(ham.N, dtype=RT)
    sq = sum(0.5 * (ham.L[g] - Lbar[g] * eye) @ (ham.L[g] - Lbar[g] * eye) for g in range(ham.G))
    assert torch.allclose(hpp + sq + ec * eye, ham.h1 + ham.e_const * eye, atol=1e-12)


def test_mean_field_shift_closed_form():
    """RHF trial with orthonormal C: L_bar_g = 2 tr(L_g C C^T)."""
    s, ham = _small_ham()
    C = s.trial[:, :s.na]
    ref = 2.0 * np.einsum("gpq,pq->g", s.L, C @ C.T)
    assert np.allclose(R.mean_field_shift(ham).numpy(), ref, atol=1e-13)


# ---------------------------------------------------------------- force bias
def test_force_bias_zero_at_trial():
    s, ham = _small_ham()
    psi, _, _ = R.init_walkers(ham, 2)
    f, f_raw = R.force_bias(ham, psi, 0.05)
    assert float(f_raw.abs().max()) < 1e-13


def test_mixed_expectation_is_derivative_of_log_overlap():
    """<L_g>_mixed = d/de log <Psi_T| e^{e L_g} |Psi> at e = 0 (one-body operator
    acting on every orbital), by central finite differences with matrix_exp."""
    s, ham = _small_ham()
    g = torch.Generator().manual_seed(9)
    psi = ham.trial.to(CT) + 0.3 * _rand_c(g, ham.N, s.na + s.nb)
    got = R.mixed_L_expectation(ham, psi)
    h = 1e-5
    for gi in (0, 3, 7):
        def lo(eps):
            U = torch.linalg.matrix_exp((eps * ham.L[gi]).to(CT))
            total = 0
            for sl in ham.spins():
                total = total + torch.log(torch.linalg.det(ham.trial[:, sl].to(CT).T @ (U @ psi[:, sl])))
            return total
        fd = (lo(h) - lo(-h)) / (2 * h)
        assert abs(complex(fd) - complex(got[gi])) < 1e-8


def test_force_bias_capping_removes_components():
    """Sec. V.C: components with |f_g| >= 1 are removed (set to 0), not clipped."""
    s, ham = _small_ham()
    g = torch.Generator().manual_seed(10)
    psi = ham.trial.to(CT) + 2.0 * _rand_c(g, ham.N, s.na + s.nb)
    tau = 4.0
    f, f_raw = R.force_bias(ham, psi, tau)
    big = f_raw.abs() >= 1.0
    assert bool(big.any()) and bool((~big).any())
    assert torch.all(f[big] == 0)
    assert torch.equal(f[~big], f_raw[~big])


# ---------------------------------------------------------------- overlaps
def test_log_overlap_closed_form_small_dets():
    g = torch.Generator().manual_seed(11)
    for n in (2, 3):
        N = 7
        trial = torch.linalg.qr(torch.randn(N, 2 * n, generator=g, dtype=RT))[0]
        ham = R.Hamiltonian(torch.zeros(N, N, dtype=RT), torch.zeros(1, N, N, dtype=RT),
                            trial, n, n)
        psi = _rand_c(g, N, 2 * n)
        got = R.log_overlap(ham, psi)
        total = 1.0 + 0j
        for sl in ham.spins():
            O = (trial[:, sl].T.to(CT) @ psi[:, sl]).numpy()
            if n == 2:
                d = O[0, 0] * O[1, 1] - O[0, 1] * O[1, 0]
            else:
                d = (O[0, 0] * (O[1, 1] * O[2, 2] - O[1, 2] * O[2, 1])
                     - O[0, 1] * (O[1, 0] * O[2, 2] - O[1, 2] * O[2, 0])
                     + O[0, 2] * (O[1, 0] * O[2, 1] - O[1, 1] * O[2, 0]))
            total *= d
        assert abs(math.log(abs(total)) - float(got.real)) < 1e-12
        dphi = (float(got.imag) - np.angle(total) + math.pi) % (2 * math.pi) - math.pi
        assert abs(dphi) < 1e-12


def test_log_overlap_after_qr_shifts_by_log_det_R():
    s, ham = _small_ham()
    g = torch.Generator().manual_seed(12)
    psi = ham.trial.to(CT) + 0.5 * _rand_c(g, ham.N, s.na + s.nb)
    lo = R.log_overlap(ham, psi)
    q, lo_q = R.reorthonormalise(ham, psi)
    logdetR = 0
    for sl in ham.spins():
        _, Rm = R.mgs_qr(psi[:, sl])
        logdetR = logdetR + torch.log(torch.diagonal(Rm)).sum()
    d = complex(lo - lo_q - logdetR)
    assert abs(d.real) < 1e-12
    assert abs((d.imag + math.pi) % (2 * math.pi) - math.pi) < 1e-12


def test_mgs_qr_against_library_qr():
    g = torch.Generator().manual_seed(13)
    X = _rand_c(g, 9, 4)
    Q, Rm = R.mgs_qr(X)
    assert torch.allclose(Q.conj().T @ Q, torch.eye(4, dtype=CT), atol=1e-13)
    assert torch.allclose(Q @ Rm, X, atol=1e-13)
    assert torch.all(torch.diagonal(Rm).real > 0) and torch.all(torch.diagonal(Rm).imag == 0)
    Ql, Rl = torch.linalg.qr(X)
    ph = torch.diagonal(Rl) / torch.diagonal(Rl).abs()
    assert torch.allclose(Ql * ph[None, :], Q, atol=1e-12)


# ---------------------------------------------------------------- local energy
def test_local_energy_at_trial_is_slater_condon_energy():
    """E_L(Psi_T) = <D|H|D> with the full 4-index V_pqrs = sum_g L_pr L_qs."""
    s, ham = _small_ham()
    C = s.trial[:, :s.na]
    P = C @ C.T
    V = np.einsum("gpr,gqs->pqrs", s.L, s.L)
    Ptot = 2 * P
    e_hf = (2 * np.einsum("pq,qp->", s.h1, P)
            + 0.5 * np.einsum("pqrs,rp,sq->", V, Ptot, Ptot)
            - 0.5 * 2 * np.einsum("pqrs,sp,rq->", V, P, P))
    got = R.local_energy(ham, ham.trial.to(CT))
    assert abs(complex(got) - e_hf) < 1e-12


def test_local_energy_at_trial_matches_bruteforce_determinant():
    s, ham = _small_ham(N=5, n=2, G=8)
    ref = fci.determinant_energy(s.h1, s.L, s.trial[:, :2], s.trial[:, 2:])
    assert abs(complex(R.local_energy(ham, ham.trial.to(CT))) - ref) < 1e-11


def test_local_energy_matches_bruteforce_for_general_walker():
    """E_L(Psi) = <Psi_T|H|Psi>/<Psi_T|Psi> with both determinants expanded in the
    FCI basis, for a real walker and for a complex one (the trial is real, so
    the brute force takes no complex conjugate)."""
    s, ham = _small_ham(N=5, n=2, G=8)
    g = np.random.default_rng(14)
    H, dets = fci.hamiltonian_matrix(s.h1, s.L, 2, 2)

    def expand(Ca, Cb):
        v = np.zeros(len(dets), dtype=np.result_type(Ca, Cb))
        for i, d in enumerate(dets):
            oa = [p for p in range(5) if (d >> p) & 1]
            ob = [p for p in range(5) if (d >> (5 + p)) & 1]
            v[i] = np.linalg.det(Ca[oa, :]) * np.linalg.det(Cb[ob, :])
        return v
    vt = expand(s.trial[:, :2], s.trial[:, 2:])
    real = s.trial + 0.3 * g.standard_normal(s.trial.shape)
    cplx = real + 0.3j * g.standard_normal(s.trial.shape)
    for psi in (real, cplx):
        vp = expand(psi[:, :2], psi[:, 2:])
        ref = (vt @ H @ vp) / (vt @ vp)
        got = R.local_energy(ham, torch.as_tensor(psi).to(CT))
        assert abs(complex(got) - complex(ref)) < 1e-10
    assert abs(complex(ref).imag) > 1e-3      # the complex case tests the imaginary part


def test_local_energy_gauge_invariance():
    s, ham = _small_ham()
    g = torch.Generator().manual_seed(15)
    psi = ham.trial.to(CT) + 0.4 * _rand_c(g, ham.N, s.na + s.nb)
    M = torch.eye(s.na, dtype=CT) + 0.5 * _rand_c(g, s.na, s.na)
    psi2 = psi.clone()
    psi2[:, :s.na] = psi[:, :s.na] @ M
    psi2[:, s.na:] = psi[:, s.na:] @ M.T
    assert abs(complex(R.local_energy(ham, psi) - R.local_energy(ham, psi2))) < 1e-11


def test_local_energy_noninteracting_projection():
    """L = 0: e^{-t h} Psi_T -> lowest orbitals, E_L -> 2 sum_{i<n} eps_i(h)."""
    s = make_system(6, 2, 2, 4, rho=0.5, seed=5)
    ham = R.make_hamiltonian(s.h1, 0.0 * s.L, s.trial, 2, 2)
    lam, V = np.linalg.eigh(s.h1)
    U = torch.as_tensor((V * np.exp(-2.0 * lam)) @ V.T).to(CT)
    psi = torch.as_tensor(s.trial).to(CT)
    for _ in range(100):                      # e^{-200 h} with re-orthonormalisation
        psi, _ = R.reorthonormalise(ham, U @ psi)
    assert abs(complex(R.local_energy(ham, psi)) - 2 * lam[:2].sum()) < 1e-9


def test_energy_window_values():
    """Eq. enwin with DeltaE = 1/2 sqrt(N_e/tau) + sqrt(N_e tau)."""
    tau, ne, e0 = 0.04, 4, -10.0
    dE = 0.5 * math.sqrt(ne / tau) + math.sqrt(ne * tau)          # = 5.4
    assert abs(dE - 5.4) < 1e-15
    E = torch.tensor([-20.0 + 1j, -10.0 + 0j, -4.0 - 2j, -4.7 + 0j], dtype=CT)
    got = R.energy_window(E, e0, tau, ne)
    assert torch.allclose(got, torch.tensor([-15.4, -10.0, -4.6, -4.7], dtype=RT), atol=1e-14)


# ---------------------------------------------------------------- weights
def test_weight_real_positive_special_case():
    """ratio*I real positive: dtheta = 0 and W' = W |ratio I| e^{tau E0}."""
    tau, e0 = 0.05, -2.0
    W = torch.tensor([1.0, 0.5, 2.0], dtype=RT)
    lr = torch.tensor([0.01, -0.02, 0.03], dtype=CT)
    li = torch.tensor([0.005, 0.0, -0.01], dtype=CT)
    Wn, eh, dth, fac = R.weight_update(W, lr, li, tau, e0)
    assert torch.all(dth == 0)
    ref = W * torch.exp((lr + li).real) * math.exp(tau * e0)
    assert torch.allclose(Wn, ref, rtol=1e-14)


def test_weight_caps():
    """Sec. V.B: a reweighting factor >= 10 is set to 0; cos(dtheta) <= 0 kills."""
    tau, e0 = 0.05, 0.0
    W = torch.ones(4, dtype=RT)
    lr = torch.tensor([math.log(11.0), math.log(9.0), 1j * 2.0, 1j * 0.5], dtype=CT)
    Wn, _, dth, fac = R.weight_update(W, lr, torch.zeros(4, dtype=CT), tau, e0)
    assert float(Wn[0]) == 0.0 and float(fac[0]) == 0.0
    assert abs(float(Wn[1]) - 9.0) < 1e-12
    assert float(Wn[2]) == 0.0
    assert abs(float(Wn[3]) - math.cos(0.5)) < 1e-14
    # phase wrapping: Im log ratio = 2 pi + 0.3 -> dtheta = 0.3
    _, _, dth2, _ = R.weight_update(W[:1], torch.tensor([1j * (2 * math.pi + 0.3)], dtype=CT),
                                    torch.zeros(1, dtype=CT), tau, e0)
    assert abs(float(dth2[0]) - 0.3) < 1e-14


def test_mixed_energy_ignores_dead_walkers():
    W = torch.tensor([1.0, 0.0, 3.0], dtype=RT)
    E = torch.tensor([-1.0, float("nan"), -2.0], dtype=RT)
    e, wsum = R.mixed_energy(W, E)
    assert abs(e - (-7.0 / 4.0)) < 1e-15 and wsum == 4.0


# ---------------------------------------------------------------- whole step
def test_first_step_from_trial_closed_form():
    """At Psi_T the force bias vanishes, so Psi_1 = B e^{i sqrt(tau) sum x_g L_g} B Psi_T
    and ratio = det(T^T Psi_1) e^{-tau E_c' - i sqrt(tau) sum x L_bar}."""
    s, ham = _small_ham()
    tau = 0.05
    psi, lo, W = R.init_walkers(ham, 2)
    x = torch.as_tensor(make_fields(3, 0, 2, ham.G))
    hpp, ec = R.propagation_h1(ham)
    Lbar = R.mean_field_shift(ham)
    B = R.half_step_propagator(hpp, tau).to(CT)
    psi1, lo1, W1, info = R.step(ham, psi, lo, W, x, tau, -5.0, method="krylov", k=ham.N)
    # block Krylov with N // n blocks spans each spin's whole space: the same step
    psib, lob, Wb, _ = R.step(ham, psi, lo, W, x, tau, -5.0, method="bkrylov", k=ham.N)
    assert torch.allclose(psib, psi1, rtol=1e-11, atol=1e-12) and torch.allclose(Wb, W1, rtol=1e-12)
    # and so does the Lanczos space of dimension N (reading R30)
    psil, lol, Wl, _ = R.step(ham, psi, lo, W, x, tau, -5.0, method="lanczos", k=ham.N)
    assert torch.allclose(psil, psi1, rtol=1e-10, atol=1e-11) and torch.allclose(Wl, W1, rtol=1e-11)
    for w in range(2):
        A = 1j * math.sqrt(tau) * torch.einsum("g,gpq->pq", x[w].to(CT), ham.L.to(CT))
        ref = B @ torch.linalg.matrix_exp(A) @ B @ ham.trial.to(CT)
        assert torch.allclose(psi1[w], ref, rtol=1e-11, atol=1e-12)
        det = 1.0
        for sl in ham.spins():
            det = det * torch.linalg.det(ham.trial[:, sl].to(CT).T @ ref[:, sl])
        log_ratio = torch.log(det) - tau * ec - 1j * math.sqrt(tau) * float(x[w] @ Lbar)
        d = complex(info.log_ratio[w] - log_ratio)
        assert abs(d.real) < 1e-11 and abs((d.imag + math.pi) % (2 * math.pi) - math.pi) < 1e-11
        assert abs(complex(info.log_I[w])) < 1e-12     # f = 0 => I = 1


def _shift_identity_sides(tau=0.1, nodes=28, e0=-1.3):
    """Both sides of the Gaussian shift identity behind importance sampling
    (Eqs. wupdate, force_shift) for one walker phi of a 2-electron system
    (N = 4, one alpha and one beta orbital, two Cholesky vectors), where the
    many-body state is the Kronecker product of the two orbitals.

    With p the standard-normal density, I(x, f) = exp(x.f - f.f/2) and any
    entire g, the substitution y = x - f gives
        int p(x) I(x, f) g(x - f) dx = int p(y) g(y) dy,
    for complex f as well.  Here g(c) = e^{tau E0} s(c) |det(B e^{A(c)} B phi)>
    / <Psi_T|phi>, s(c) = e^{-tau E_c' - i sqrt(tau) c.L_bar} (reading R1).
    The left side is the free-projection step of the oracle at its force bias
    f != 0 (weight' |phi'> / <Psi_T|phi'>); the right side is written out here
    at c = x, from B, E_c' and L_bar, and matrix_exp.  Both are integrated by
    the tensor Gauss-Hermite rule.  Returns (left, right, f)."""
    import itertools
    s = make_system(4, 1, 1, 2, rho=0.8, seed=23, lambda0=1.0)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, 1, 1)
    g = torch.Generator().manual_seed(5)
    phi = (ham.trial.to(CT) + 0.6 * _rand_c(g, 4, 2)).unsqueeze(0)
    lo = R.log_overlap(ham, phi)
    Lbar = R.mean_field_shift(ham)
    hpp, ec = R.propagation_h1(ham, Lbar)
    B = R.half_step_propagator(hpp, tau)
    xs, ws = np.polynomial.hermite_e.hermegauss(nodes)
    ws = ws / ws.sum()
    pts = list(itertools.product(range(nodes), repeat=ham.G))
    X = torch.tensor([[xs[i] for i in idx] for idx in pts], dtype=RT)
    wq = torch.tensor([float(np.prod([ws[i] for i in idx])) for idx in pts], dtype=RT)
    nq = len(pts)
    psi = phi.repeat(nq, 1, 1)
    f, _ = R.force_bias(ham, phi, tau, Lbar)
    psi1, lo1, wt1 = R.free_projection_step(ham, psi, lo.repeat(nq), torch.ones(nq, dtype=CT), X,
                                            tau, e0, method="taylor", k=30, B=B, L_bar=Lbar, ec=ec)
    amp = wt1 * torch.exp(-lo1)                                      # weight' / <Psi_T|phi'>
    left = sum(wq[q] * amp[q] * torch.kron(psi1[q, :, 0], psi1[q, :, 1]) for q in range(nq))
    Bc = B.to(CT)
    right = torch.zeros(16, dtype=CT)
    for q in range(nq):
        c = X[q].to(CT)
        M = Bc @ torch.linalg.matrix_exp(1j * math.sqrt(tau) * torch.einsum("g,gpq->pq", c, ham.L.to(CT))) @ Bc
        sc = torch.exp(tau * e0 - tau * ec - 1j * math.sqrt(tau) * (c @ Lbar.to(CT)) - lo[0])
        right = right + wq[q] * sc * torch.kron(M @ phi[0, :, 0], M @ phi[0, :, 1])
    return left, right, f[0]


def test_importance_sampled_step_keeps_the_gaussian_average():
    """The free-projection step, which shares the force bias, the shifted field,
    the importance factor I and the scalar s with the phaseless step
    (propagate_and_ratio), leaves the field average of weight' |phi'> /
    <Psi_T|phi'> unchanged by a force bias f != 0 (the Gaussian shift
    identity; see _shift_identity_sides).  This pins the sign and the 1/2 of
    log I and the c = x - f inside log s where f is not zero."""
    left, right, f = _shift_identity_sides()
    assert 0.05 < float(f.abs().max()) < 1.0 and float(f.abs().min()) > 0.01   # f != 0, not capped
    err = float((left - right).abs().max() / right.abs().max())
    assert err < 1e-11, err


def test_dead_walkers_are_kept():
    s, ham = _small_ham()
    psi, lo, W = R.init_walkers(ham, 3)
    W[1] = 0.0
    x = torch.as_tensor(make_fields(4, 0, 3, ham.G))
    psi1, lo1, W1, _ = R.step(ham, psi, lo, W, x, 0.05, -5.0, method="taylor", k=6)
    assert torch.equal(psi1[1], psi[1]) and float(W1[1]) == 0.0
    assert not torch.equal(psi1[0], psi[0])


def test_comb_example():
    W = torch.tensor([0.5, 0.0, 2.5, 1.0], dtype=RT)
    # total 4, teeth at u + j = 0.25, 1.25, 2.25, 3.25 -> cumulative 0.5, 0.5, 3, 4
    assert R.comb(W, 0.25).tolist() == [0, 2, 2, 3]
    assert R.comb(W, 0.75).tolist() == [2, 2, 2, 3]
    # a tooth exactly on a cumulative boundary belongs to the next walker
    assert R.comb(torch.tensor([1.0, 1.0], dtype=RT), 0.0).tolist() == [0, 1]


def test_comb_is_unbiased_on_average():
    """E[number of copies of walker w] = Nw W_w / sum W for u ~ U[0,1)."""
    g = np.random.default_rng(3)
    W = torch.as_tensor(g.uniform(0, 2, 16))
    W[5] = 0.0
    counts = np.zeros(16)
    us = (np.arange(4000) + 0.5) / 4000
    for u in us:
        counts += np.bincount(R.comb(W, float(u)).numpy(), minlength=16)
    expect = 16 * W.numpy() / W.numpy().sum()
    assert np.allclose(counts / len(us), expect, atol=2e-3)
    assert counts[5] == 0


def test_population_control_keeps_total_weight():
    g = torch.Generator().manual_seed(4)
    psi = _rand_c(g, 6, 5, 2)
    lo = _rand_c(g, 6)
    W = torch.tensor([0.3, 1.2, 0.0, 2.0, 0.5, 1.0], dtype=RT)
    p2, l2, W2, idx = R.population_control(psi, lo, W, 0.4)
    assert abs(float(W2.sum()) - float(W.sum())) < 1e-14
    for j, i in enumerate(idx.tolist()):
        assert torch.equal(p2[j], psi[i]) and l2[j] == lo[i]


# ---------------------------------------------------------------- whole walk
def test_free_projection_matches_fci():
    """fp-AFQMC (Eqs. psiupdate, wupdate) with Split-2 at small tau reproduces the
    brute-force FCI ground-state energy of a 2-electron / 4-orbital system within
    3 sigma, while the HF energy is many sigma away."""
    s = make_system(4, 1, 1, 8, rho=0.7, seed=11, lambda0=0.25)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, 1, 1)
    e_fci = fci.ground_state_energy(s.h1, s.L, 1, 1)
    e_hf = fci.determinant_energy(s.h1, s.L, s.trial[:, :1], s.trial[:, 1:])
    Lbar = R.mean_field_shift(ham)
    hpp, ec = R.propagation_h1(ham, Lbar)
    tau, nw, nsteps, neq = 0.05, 1000, 600, 300
    B = R.half_step_propagator(hpp, tau)
    psi, lo, _ = R.init_walkers(ham, nw)
    wt = torch.ones(nw, dtype=CT)
    series = []
    for k in range(nsteps):
        x = make_fields(7, k, nw, ham.G)
        psi, lo, wt = R.free_projection_step(ham, psi, lo, wt, x, tau, e_fci, method="taylor",
                                             k=10, B=B, L_bar=Lbar, ec=ec)
        if k % 20 == 19:
            psi, lo = R.reorthonormalise(ham, psi)
            wt = wt / wt.abs().mean()
        El = R.local_energy(ham, psi)
        series.append(complex((wt * El).sum() / wt.sum()).real)
    E = np.array(series[neq:])
    blocks = E.reshape(6, -1).mean(1)
    sigma = blocks.std(ddof=1) / math.sqrt(len(blocks))
    mean = E.mean()
    assert abs(mean - e_fci) < 3 * sigma + 1e-4, (mean, e_fci, sigma)
    assert abs(e_hf - e_fci) > 5 * sigma, (e_hf, e_fci, sigma)


def test_phaseless_energy_next_to_fci_gap_reported():
    """The phaseless walk (Eqs. psiupdate, wupdate, phaseless; the oracle's
    `step`, which shares propagate_and_ratio with the free-projection pin
    above) on the same 2-electron / 4-orbital system, with the energy window,
    comb population control every 10 steps and E_0 following the estimate.
    The phaseless constraint biases the energy (the paper's phaseless error),
    so its gap to FCI is reported, not pinned: the test prints it and only
    asks that the walk recovers a part of the correlation energy, i.e. that
    the gap is smaller than the HF-to-FCI distance.  Last run: E = -3.66884
    +- 0.00113 Ha against E_FCI = -3.66310 Ha, gap -5.7 mHa; HF is 23.5 mHa
    above FCI."""
    s = make_system(4, 1, 1, 8, rho=0.7, seed=11, lambda0=0.25)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, 1, 1)
    e_fci = fci.ground_state_energy(s.h1, s.L, 1, 1)
    e_hf = fci.determinant_energy(s.h1, s.L, s.trial[:, :1], s.trial[:, 1:])
    Lbar = R.mean_field_shift(ham)
    hpp, ec = R.propagation_h1(ham, Lbar)
    tau, nw, nsteps, neq = 0.05, 1000, 600, 300
    B = R.half_step_propagator(hpp, tau)
    psi, lo, W = R.init_walkers(ham, nw)
    rng = np.random.Generator(np.random.PCG64(99))
    e0, series = e_hf, []
    for k in range(nsteps):
        x = make_fields(8, k, nw, ham.G)
        psi, lo, W, _ = R.step(ham, psi, lo, W, x, tau, e0, method="taylor", k=10,
                               reortho=(k % 5 == 4), B=B, L_bar=Lbar, ec=ec)
        ek, _ = R.mixed_energy(W, R.energy_window(R.local_energy(ham, psi), e0, tau, 2))
        series.append(ek)
        if k % 10 == 9:
            psi, lo, W, _ = R.population_control(psi, lo, W, float(rng.uniform()))
            W = W / W.mean()
            e0 = ek if k < neq else float(np.mean(series[neq:]))
    E = np.array(series[neq:])
    blocks = E.reshape(10, -1).mean(1)
    sigma = blocks.std(ddof=1) / math.sqrt(len(blocks))
    gap = E.mean() - e_fci
    print(f"phaseless E = {E.mean():.6f} +- {sigma:.6f} Ha, E_FCI = {e_fci:.6f} Ha, "
          f"gap = {gap * 1e3:+.2f} mHa ({gap / sigma:+.1f} sigma), E_HF - E_FCI = {(e_hf - e_fci) * 1e3:.2f} mHa")
    assert np.isfinite(E).all() and sigma > 0
    assert abs(gap) < abs(e_hf - e_fci), (gap, e_hf - e_fci)


# ---------------------------------------------------------------- gradients
def test_oracle_energy_gradient_matches_central_differences():
    """Reverse-mode autograd through the oracle's local energy and mixed
    estimator agrees with central finite differences along random symmetric
    directions (the CPU reference for the adjoint)."""
    s, ham = _small_ham(N=8, n=2, G=10)
    g = torch.Generator().manual_seed(21)
    psi = ham.trial.to(CT).unsqueeze(0).repeat(3, 1, 1) + 0.3 * _rand_c(g, 3, 8, 4)
    W = torch.tensor([1.0, 0.7, 1.3], dtype=RT)
    e0, tau = float(R.local_energy(ham, ham.trial.to(CT)).real), 0.05

    def J(h1, L):
        hm = R.Hamiltonian(h1, L, ham.trial, 2, 2)
        Ec = R.energy_window(R.local_energy(hm, psi), e0, tau, 4)
        return (W * Ec).sum() / W.sum()

    h1 = ham.h1.clone().requires_grad_(True)
    L = ham.L.clone().requires_grad_(True)
    J(h1, L).backward()
    rng = np.random.default_rng(5)
    dH = torch.as_tensor(rng.standard_normal((8, 8))); dH = 0.5 * (dH + dH.T)
    dL = torch.as_tensor(rng.standard_normal((10, 8, 8))); dL = 0.5 * (dL + dL.transpose(1, 2))
    eps = 1e-5
    with torch.no_grad():
        fd_h = (J(ham.h1 + eps * dH, ham.L) - J(ham.h1 - eps * dH, ham.L)) / (2 * eps)
        fd_L = (J(ham.h1, ham.L + eps * dL) - J(ham.h1, ham.L - eps * dL)) / (2 * eps)
    assert abs(float(fd_h) - float((h1.grad * dH).sum())) < 1e-8
    assert abs(float(fd_L) - float((L.grad * dL).sum())) < 1e-8


# ---------------------------------------------------------------- walk adjoint
class _Sys:
    """A synthetic closed-shell system with the trial cut to na alpha and nb
    beta orbitals (na != nb exercises unequal spin blocks)."""

    def __init__(self, N, na, nb, G, seed):
        base = make_system(N, na, na, G, rho=0.8, seed=seed)
        self.h1, self.L, self.e_const = base.h1, base.L, base.e_const
        self.trial = np.concatenate([base.trial[:, :na], base.trial[:, na:na + nb]], axis=1)
        self.na, self.nb = na, nb


def _walk_setup(N=7, na=2, nb=1, G=9, nw=3, steps=5, seed=11, tau=0.05):
    s = _Sys(N, na, nb, G, seed)
    ham0 = R.make_hamiltonian(s.h1, s.L, s.trial, na, nb, s.e_const)
    e0 = float(R.local_energy(ham0, ham0.trial.to(CT)).real)
    fields = [make_fields(seed, k, nw, G) for k in range(steps)]
    return s, e0, fields, tau


def _walk_J(s, h1, L, psi0, fields, tau, e0, r=2, method="taylor", k=6):
    ham = R.Hamiltonian(torch.as_tensor(h1, dtype=RT), torch.as_tensor(L, dtype=RT),
                        torch.as_tensor(s.trial, dtype=RT), s.na, s.nb, s.e_const)
    return R.walk_objective(ham, psi0, torch.ones(psi0.shape[0], dtype=RT), fields, tau, e0,
                            k=k, reortho_every=r, method=method)[0]


def test_walk_objective_gradient_matches_central_differences():
    """Reading R10: torch autograd through the oracle walk (Taylor-6, QR every 2
    steps) against central differences of J along random symmetric dH, dL."""
    s, e0, fields, tau = _walk_setup()
    nw = fields[0].shape[0]
    psi0 = torch.as_tensor(s.trial, dtype=RT).to(CT).unsqueeze(0).repeat(nw, 1, 1)
    h1 = torch.tensor(s.h1, dtype=RT, requires_grad=True)
    L = torch.tensor(s.L, dtype=RT, requires_grad=True)
    J = _walk_J(s, h1, L, psi0, fields, tau, e0)
    gh, gL = torch.autograd.grad(J, [h1, L])
    rng = np.random.default_rng(4)
    dH = rng.standard_normal(s.h1.shape); dH = 0.5 * (dH + dH.T)
    dL = rng.standard_normal(s.L.shape); dL = 0.5 * (dL + dL.transpose(0, 2, 1))
    eps = 1e-5
    with torch.no_grad():
        fd_h = (float(_walk_J(s, s.h1 + eps * dH, s.L, psi0, fields, tau, e0))
                - float(_walk_J(s, s.h1 - eps * dH, s.L, psi0, fields, tau, e0))) / (2 * eps)
        fd_L = (float(_walk_J(s, s.h1, s.L + eps * dL, psi0, fields, tau, e0))
                - float(_walk_J(s, s.h1, s.L - eps * dL, psi0, fields, tau, e0))) / (2 * eps)
    assert abs(fd_h - float((gh * torch.as_tensor(dH)).sum())) <= 1e-6 * max(1.0, abs(fd_h))
    assert abs(fd_L - float((gL * torch.as_tensor(dL)).sum())) <= 1e-6 * max(1.0, abs(fd_L))


def test_walk_objective_gauge_invariance_and_psi_gradient():
    """J is unchanged by Psi_0 -> Psi_0 M (the Taylor action, Theta, the overlap
    ratio and E_L are invariant), so its gradient G with respect to Psi_0
    satisfies Psi_0,s^T G_s = 0 per spin; G = conj(torch's .grad) reproduces
    a central difference along a random complex direction."""
    s, e0, fields, tau = _walk_setup(steps=4, seed=12)
    nw = fields[0].shape[0]
    g = torch.Generator().manual_seed(3)
    psi0 = (torch.as_tensor(s.trial, dtype=RT).to(CT).unsqueeze(0).repeat(nw, 1, 1)
            + 0.1 * _rand_c(g, nw, s.trial.shape[0], s.trial.shape[1]))
    psi0.requires_grad_(True)
    J = _walk_J(s, s.h1, s.L, psi0, fields, tau, e0)
    (tg,) = torch.autograd.grad(J, [psi0])
    G = tg.conj()
    with torch.no_grad():
        M = torch.eye(3, dtype=CT) + 0.3 * _rand_c(g, 3, 3)
        M[:2, 2] = 0
        M[2, :2] = 0                      # block diagonal: alpha (2) and beta (1) columns
        J2 = float(_walk_J(s, s.h1, s.L, psi0.detach() @ M, fields, tau, e0))
        assert abs(J2 - float(J)) <= 1e-11 * abs(float(J))
        for sl in (slice(0, 2), slice(2, 3)):
            P = psi0.detach()[:, :, sl]
            Z = P.transpose(1, 2) @ G[:, :, sl]
            assert float(Z.abs().max()) <= 1e-10 * float(G.abs().max()) * 10
        dP = _rand_c(g, *psi0.shape)
        eps = 1e-6
        fd = (float(_walk_J(s, s.h1, s.L, psi0.detach() + eps * dP, fields, tau, e0))
              - float(_walk_J(s, s.h1, s.L, psi0.detach() - eps * dP, fields, tau, e0))) / (2 * eps)
        assert abs(fd - float((G * dP).sum().real)) <= 1e-6 * max(1.0, abs(fd))


def test_krylov_walk_gradient_matches_central_differences_and_exact_at_full_dimension():
    """The Krylov path of the walk objective (Eq. krylov, dimension 4 < N = 7):
    autograd through the Arnoldi steps and the small exponential against
    central differences along random symmetric dH, dL; at dimension N the
    Krylov action is the exact e^A psi, so J and its gradients equal those of
    the exact action (matrix_exp)."""
    s, e0, fields, tau = _walk_setup(steps=4, seed=13)
    nw = fields[0].shape[0]
    psi0 = torch.as_tensor(s.trial, dtype=RT).to(CT).unsqueeze(0).repeat(nw, 1, 1)
    rng = np.random.default_rng(6)
    dH = rng.standard_normal(s.h1.shape); dH = 0.5 * (dH + dH.T)
    dL = rng.standard_normal(s.L.shape); dL = 0.5 * (dL + dL.transpose(0, 2, 1))
    h1 = torch.tensor(s.h1, dtype=RT, requires_grad=True)
    L = torch.tensor(s.L, dtype=RT, requires_grad=True)
    J = _walk_J(s, h1, L, psi0, fields, tau, e0, method="krylov", k=4)
    gh, gL = torch.autograd.grad(J, [h1, L])
    eps = 1e-5
    with torch.no_grad():
        def Jk(hh, LL):
            return float(_walk_J(s, hh, LL, psi0, fields, tau, e0, method="krylov", k=4))
        fd_h = (Jk(s.h1 + eps * dH, s.L) - Jk(s.h1 - eps * dH, s.L)) / (2 * eps)
        fd_L = (Jk(s.h1, s.L + eps * dL) - Jk(s.h1, s.L - eps * dL)) / (2 * eps)
    assert abs(fd_h - float((gh * torch.as_tensor(dH)).sum())) <= 1e-6 * max(1.0, abs(fd_h))
    assert abs(fd_L - float((gL * torch.as_tensor(dL)).sum())) <= 1e-6 * max(1.0, abs(fd_L))
    N = s.h1.shape[0]
    grads = {}
    for method, k in (("krylov", N), ("exact", 0)):
        h1 = torch.tensor(s.h1, dtype=RT, requires_grad=True)
        L = torch.tensor(s.L, dtype=RT, requires_grad=True)
        Jm = _walk_J(s, h1, L, psi0, fields, tau, e0, method=method, k=k)
        grads[method] = (float(Jm.detach()),) + tuple(torch.autograd.grad(Jm, [h1, L]))
    (Jk_, ghk, gLk), (Je, ghe, gLe) = grads["krylov"], grads["exact"]
    assert abs(Jk_ - Je) <= 1e-11 * abs(Je)
    assert float((ghk - ghe).abs().max()) <= 1e-8 * float(ghe.abs().max())
    assert float((gLk - gLe).abs().max()) <= 1e-8 * float(gLe.abs().max())
    # and the dimension-4 gradient differs from the exact one (the test sees the truncation)
    assert float((gh - ghe).abs().max()) > 1e-10


def test_lanczos_walk_gradient_matches_central_differences_and_exact_at_full_dimension():
    """The walk objective with the complex-symmetric Lanczos action (reading
    R30, dimension 4 < N = 7), no re-orthonormalisation: autograd through the
    three-term recurrence (bilinear forms, principal square roots) and the
    small exponential against central differences along random symmetric
    dH, dL and along a random complex direction of Psi_0 (G = conj(torch's
    .grad)); at dimension N the Lanczos action is the exact e^A psi, so J and
    its gradients equal those of the exact action (matrix_exp), QR included."""
    s, e0, fields, tau = _walk_setup(steps=4, seed=14)
    nw = fields[0].shape[0]
    g = torch.Generator().manual_seed(5)
    psi0 = (torch.as_tensor(s.trial, dtype=RT).to(CT).unsqueeze(0).repeat(nw, 1, 1)
            + 0.1 * _rand_c(g, nw, s.trial.shape[0], s.trial.shape[1]))
    rng = np.random.default_rng(7)
    dH = rng.standard_normal(s.h1.shape); dH = 0.5 * (dH + dH.T)
    dL = rng.standard_normal(s.L.shape); dL = 0.5 * (dL + dL.transpose(0, 2, 1))
    h1 = torch.tensor(s.h1, dtype=RT, requires_grad=True)
    L = torch.tensor(s.L, dtype=RT, requires_grad=True)
    p0 = psi0.clone().requires_grad_(True)
    J = _walk_J(s, h1, L, p0, fields, tau, e0, r=0, method="lanczos", k=4)
    gh, gL, tg = torch.autograd.grad(J, [h1, L, p0])
    G = tg.conj()
    eps = 1e-5
    with torch.no_grad():
        def Jl(hh, LL, pp):
            return float(_walk_J(s, hh, LL, pp, fields, tau, e0, r=0, method="lanczos", k=4))
        fd_h = (Jl(s.h1 + eps * dH, s.L, psi0) - Jl(s.h1 - eps * dH, s.L, psi0)) / (2 * eps)
        fd_L = (Jl(s.h1, s.L + eps * dL, psi0) - Jl(s.h1, s.L - eps * dL, psi0)) / (2 * eps)
        dP = _rand_c(g, *psi0.shape)
        fd_p = (Jl(s.h1, s.L, psi0 + eps * dP) - Jl(s.h1, s.L, psi0 - eps * dP)) / (2 * eps)
    assert abs(fd_h - float((gh * torch.as_tensor(dH)).sum())) <= 1e-6 * max(1.0, abs(fd_h))
    assert abs(fd_L - float((gL * torch.as_tensor(dL)).sum())) <= 1e-6 * max(1.0, abs(fd_L))
    assert abs(fd_p - float((G * dP).sum().real)) <= 1e-8 * max(1.0, abs(fd_p))
    N = s.h1.shape[0]
    grads = {}
    for method, k in (("lanczos", N), ("exact", 0)):
        h1 = torch.tensor(s.h1, dtype=RT, requires_grad=True)
        L = torch.tensor(s.L, dtype=RT, requires_grad=True)
        Jm = _walk_J(s, h1, L, psi0, fields, tau, e0, method=method, k=k)
        grads[method] = (float(Jm.detach()),) + tuple(torch.autograd.grad(Jm, [h1, L]))
    (Jn, ghn, gLn), (Je, ghe, gLe) = grads["lanczos"], grads["exact"]
    assert abs(Jn - Je) <= 1e-10 * abs(Je)
    assert float((ghn - ghe).abs().max()) <= 1e-7 * float(ghe.abs().max())
    assert float((gLn - gLe).abs().max()) <= 1e-7 * float(gLe.abs().max())
    # the dimension-4 gradient differs from the exact one (the test sees the truncation)
    assert float((gh - ghe).abs().max()) > 1e-10


@pytest.mark.parametrize("method", ["krylov", "lanczos"])
def test_qr_as_fixed_factor_is_exact_only_for_actions_linear_in_psi(method):
    """Reading R10 holds the re-orthonormalisation Psi <- Psi R^{-1} as a
    fixed right factor.  That is exact where everything downstream is
    invariant under Psi -> Psi M, which holds for the Taylor action (linear in
    Psi) but not for a column-wise Krylov action of dimension k < N (each
    column has its own Krylov space): there the gradient drops the part of
    dJ that flows through R, a term of the order of the Krylov truncation.
    Measured here against central differences with QR every 2 steps: the
    Taylor gradient is exact, the Krylov ones differ by less than 1e-4 of the
    derivative but by more than the differences' own error."""
    s, e0, fields, tau = _walk_setup(steps=4, seed=14)
    nw = fields[0].shape[0]
    g = torch.Generator().manual_seed(5)
    psi0 = (torch.as_tensor(s.trial, dtype=RT).to(CT).unsqueeze(0).repeat(nw, 1, 1)
            + 0.1 * _rand_c(g, nw, s.trial.shape[0], s.trial.shape[1]))
    dP = _rand_c(torch.Generator().manual_seed(99), *psi0.shape)
    eps = 1e-5

    def gap(m, k):
        p0 = psi0.clone().requires_grad_(True)
        J = _walk_J(s, s.h1, s.L, p0, fields, tau, e0, r=2, method=m, k=k)
        (tg,) = torch.autograd.grad(J, [p0])
        with torch.no_grad():
            fd = (float(_walk_J(s, s.h1, s.L, psi0 + eps * dP, fields, tau, e0, r=2, method=m, k=k))
                  - float(_walk_J(s, s.h1, s.L, psi0 - eps * dP, fields, tau, e0, r=2, method=m, k=k))) / (2 * eps)
        return abs(fd - float((tg.conj() * dP).sum().real)) / abs(fd)

    assert gap("taylor", 6) <= 1e-8
    assert 1e-8 < gap(method, 4) <= 1e-4

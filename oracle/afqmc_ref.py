"""CPU oracle for the phaseless-AFQMC walker step (test infrastructure only).

This module is the slow, plain FP64 statement of what the walker step of
large-time-step ph-AFQMC computes (Sukurma et al., "Towards Large-Scale AFQMC
Calculations: Large Time Step Auxiliary-Field Quantum Monte Carlo").  It is
used only by the tests, by the smoke check and by the CPU-baseline leg of the
benchmark; the product path never imports it.  It shares no code with the CUDA
library: every quantity is written from its definition with PyTorch CPU
primitives (matmul, solve, slogdet, eigh, eig, matrix_exp), in float64 /
complex128, walker by walker where the method is per walker.

Conventions.
  * A walker is psi [N, na+nb] complex; columns [0, na) hold the alpha
    orbitals, [na, na+nb) the beta orbitals.  Batches carry a leading walker
    axis: psi [Nw, N, na+nb].
  * trial [N, na+nb] real, same column split.
  * L [G, N, N] real symmetric Cholesky vectors, <pq|rs> = sum_g L_g,pr L_g,qs
    (Sec. II.A).
  * logovl = sum_sigma log det(trial_sigma^T psi_sigma) (complex; the
    imaginary part is defined modulo 2 pi).

Readings of the paper used here (the paper is silent or ambiguous on them):
  R1  The mean-field shift L_bar_g enters as an operator constant:
      H = h'' + 1/2 sum_g (L_g - L_bar_g)^2 + E_c' with
      h'' = h - 1/2 sum_g L_g L_g + sum_g L_bar_g L_g and
      E_c' = E_const - 1/2 sum_g L_bar_g^2.  e^{-tau h''/2} is the Split-2
      half step; the shift contributes one scalar factor
      s = exp(-tau E_c' - i sqrt(tau) sum_g c_g L_bar_g) per walker to the
      overlap ratio.
  R5  Krylov = Arnoldi with one modified Gram-Schmidt pass per vector; an
      invariant subspace is declared when the new subdiagonal entry is
      <= 1e-12 ||A||_F (the basis vectors are unit vectors).
  R6  The small exponential e^{A_k} is torch.linalg.matrix_exp.
  R30 Lanczos variant of the Krylov action: the paper uses Arnoldi (Sec.
      IV.C) for a general non-Hermitian A; the field matrix is complex
      symmetric, so the three-term recurrence with the bilinear form u^T v
      spans the same Krylov space with a tridiagonal projected matrix
      (lanczos_action).  No re-orthogonalisation; the breakdown test of R5
      on |beta_j|.
  R20 Block Krylov (Sec. IV.D, Eqs. bkrylovsub-bkrylov) works on each spin
      block separately (the two determinants span separate spaces); the QR
      of Psi and of every new block is modified Gram-Schmidt (mgs_qr), the
      new block is orthogonalised against the previous ones by one block
      modified Gram-Schmidt pass, the number of blocks is at most N // n, and
      the space is declared invariant at the first new block whose QR has a
      diagonal entry <= 1e-12 ||A||_F.
  R23 The Chebyshev expansion (Sec. IV.B) is applied to A as printed, with
      no rescaling of its spectrum into [-1, 1]: A is O(sqrt(tau)) small at
      the paper's time steps, and the coefficients c_n = 2 I_n(1) fall off
      like 1 / (2^n n!).
  R7  E_0 is a caller-supplied scalar.
  R8  Population control: comb with caller-supplied uniform u.
  R9  Threshold tests use the strict inequalities printed in Sec. V.
  R11 The mixed estimator and the energy window use Re E_L.
  R25 The walkers are re-orthonormalised every r steps (a caller's choice) by
      modified Gram-Schmidt per spin; the paper does not discuss it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

RT = torch.float64
CT = torch.complex128

__all__ = [
    "Hamiltonian", "make_hamiltonian", "overlap", "greens_function",
    "log_overlap", "theta", "mean_field_shift", "mixed_L_expectation",
    "force_bias", "propagation_h1", "half_step_propagator", "field_matrix",
    "taylor_action", "chebyshev_coefficients", "chebyshev_action", "krylov_action", "lanczos_action", "block_krylov_action", "exact_action", "expm_action",
    "split2_propagate", "split1_propagate", "taylor_propagate", "crank_nicolson_propagate", "propagate",
    "local_energy", "energy_window", "mixed_energy",
    "mgs_qr", "reorthonormalise", "weight_update", "propagate_and_ratio", "step", "init_walkers",
    "free_projection_step", "comb", "population_control", "StepInfo",
    "walk_objective",
]


# --------------------------------------------------------------------------
# Hamiltonian data (Sec. II.A, Eq. mbham and the Cholesky decomposition)
# --------------------------------------------------------------------------
@dataclass
class Hamiltonian:
    h1: torch.Tensor        # [N, N] real symmetric one-body matrix h_pq
    L: torch.Tensor         # [G, N, N] Cholesky vectors L_g,pq
    trial: torch.Tensor     # [N, na+nb] real trial orbitals
    na: int
    nb: int
    e_const: float = 0.0

    @property
    def N(self):
        return self.h1.shape[0]

    @property
    def G(self):
        return self.L.shape[0]

    def spins(self):
        """Column slices of the two spin blocks."""
        return (slice(0, self.na), slice(self.na, self.na + self.nb))


def make_hamiltonian(h1, L, trial, na, nb, e_const=0.0) -> Hamiltonian:
    return Hamiltonian(torch.as_tensor(h1, dtype=RT), torch.as_tensor(L, dtype=RT),
                       torch.as_tensor(trial, dtype=RT), int(na), int(nb), float(e_const))


# --------------------------------------------------------------------------
# Overlaps and the mixed one-particle density (Sec. II.A, Eqs. force_shift,
# hyben, eloc)
# --------------------------------------------------------------------------
def overlap(trial_s, psi_s):
    """O = <Psi_T|Psi> matrix for one spin: O = trial^T psi  ([..., n, n])."""
    return trial_s.to(psi_s.dtype).transpose(-1, -2) @ psi_s


def log_overlap(ham: Hamiltonian, psi):
    """log <Psi_T|Psi> = sum_sigma log det(trial_sigma^T psi_sigma)."""
    total = 0
    for sl in ham.spins():
        if sl.stop == sl.start:
            continue
        sign, logabs = torch.linalg.slogdet(overlap(ham.trial[:, sl], psi[..., sl]))
        total = total + logabs + 1j * torch.angle(sign)
    return total


def theta(trial_s, psi_s):
    """Theta = psi (trial^T psi)^{-1}, the N x n factor of the mixed density."""
    O = overlap(trial_s, psi_s)
    # Theta O = psi  <=>  O^T Theta^T = psi^T
    return torch.linalg.solve(O.transpose(-1, -2), psi_s.transpose(-1, -2)).transpose(-1, -2)


def greens_function(trial_s, psi_s):
    """Mixed one-particle density G_pq = <Psi_T|a+_p a_q|Psi>/<Psi_T|Psi>.

    For Slater determinants G_pq = [psi (trial^T psi)^{-1} trial^T]_{qp}.
    """
    M = theta(trial_s, psi_s) @ trial_s.to(psi_s.dtype).transpose(-1, -2)
    return M.transpose(-1, -2)


def mixed_L_expectation(ham: Hamiltonian, psi):
    """<Psi_T|L_g|Psi>/<Psi_T|Psi> = sum_sigma sum_pq L_g,pq G^sigma_pq  ([..., G])."""
    out = 0
    for sl in ham.spins():
        if sl.stop == sl.start:
            continue
        Gs = greens_function(ham.trial[:, sl], psi[..., sl])
        out = out + torch.einsum("gpq,...pq->...g", ham.L.to(Gs.dtype), Gs)
    return out


def mean_field_shift(ham: Hamiltonian):
    """L_bar_g = <Psi_T|L_g|Psi_T>/<Psi_T|Psi_T> (Eq. force_shift, first line)."""
    return mixed_L_expectation(ham, ham.trial.to(CT)).real


# --------------------------------------------------------------------------
# Force bias and the effective interaction (Eqs. heffTOT, force_shift;
# force-bias capping of Sec. V.C)
# --------------------------------------------------------------------------
def force_bias(ham: Hamiltonian, psi, tau, L_bar=None):
    """f_g = -i sqrt(tau) (<L_g>_mixed - L_bar_g), components with |f_g| >= 1 set to 0.

    Returns (f_capped, f_uncapped).
    """
    if L_bar is None:
        L_bar = mean_field_shift(ham)
    f = -1j * math.sqrt(tau) * (mixed_L_expectation(ham, psi) - L_bar)
    capped = torch.where(f.abs() < 1.0, f, torch.zeros_like(f))
    return capped, f


def propagation_h1(ham: Hamiltonian, L_bar=None):
    """h'' and E_c' of reading R1.

    1/2 sum_pqrs V a+a+aa = 1/2 sum_g L_g^2 - 1/2 sum_g (L_g L_g)_pq a+_p a_q,
    and 1/2 sum_g L_g^2 = 1/2 sum_g (L_g - L_bar_g)^2 + sum_g L_bar_g L_g
    - 1/2 sum_g L_bar_g^2.
    """
    if L_bar is None:
        L_bar = mean_field_shift(ham)
    LL = torch.einsum("gpr,grq->pq", ham.L, ham.L)
    hpp = ham.h1 - 0.5 * LL + torch.einsum("g,gpq->pq", L_bar, ham.L)
    ec = ham.e_const - 0.5 * (L_bar * L_bar).sum()      # a 0-dim tensor (stays on the autograd graph)
    return hpp, ec


def half_step_propagator(hpp, tau):
    """B = exp(-tau h''/2), exact by diagonalisation (Sec. III.B)."""
    lam, V = torch.linalg.eigh(hpp)
    return (V * torch.exp(-0.5 * tau * lam)[None, :]) @ V.T


def field_matrix(ham: Hamiltonian, c, tau):
    """A = -tau H_int (Sec. IV) without the L_bar delta term (reading R1).

    H_int,pq = -(i/sqrt(tau)) sum_g c_g L_g,pq with c_g = x_g - f_g, so
    A = i sqrt(tau) sum_g c_g L_g.  c: [..., G] complex -> A [..., N, N].
    """
    return 1j * math.sqrt(tau) * torch.einsum("...g,gpq->...pq", c, ham.L.to(CT))


# --------------------------------------------------------------------------
# Action of the exponential (Sec. IV)
# --------------------------------------------------------------------------
def taylor_action(A, psi, k):
    """taylor_k{A, Psi} = sum_{n=0}^{k} A^n / n! Psi  (Eq. taylor)."""
    term = psi
    acc = psi
    for n in range(1, k + 1):
        term = (A @ term) / n
        acc = acc + term
    return acc


def chebyshev_coefficients(k):
    """c_0 = J_0(i) and c_n = 2 i^n J_n(-i) for n = 1..k (Sec. IV.B), the
    Bessel functions of the first kind at complex argument from scipy.special
    (a library routine).  Returns a complex tensor [k+1]."""
    from scipy.special import jv
    c = [complex(jv(0, 1j))] + [2.0 * (1j ** n) * complex(jv(n, -1j)) for n in range(1, k + 1)]
    return torch.tensor(c, dtype=CT)


def chebyshev_action(A, psi, k):
    """cheb_k{A, Psi} = sum_{n=0}^{k} c_n T_n(A) Psi (Sec. IV.B) with the
    polynomials of Eq. chebpoly: T_0 = 1, T_1 = A, T_n = 2 A T_{n-1} - T_{n-2},
    applied to Psi without rescaling A (reading R23)."""
    c = chebyshev_coefficients(k)
    acc = c[0] * psi
    if k == 0:
        return acc
    t_prev, t_cur = psi, A @ psi
    acc = acc + c[1] * t_cur
    for n in range(2, k + 1):
        t_prev, t_cur = t_cur, 2.0 * (A @ t_cur) - t_prev
        acc = acc + c[n] * t_cur
    return acc


def _arnoldi_column(A, psi_col, k, normA):
    """Krylov approximation of e^A psi for one orbital vector (Eqs. krylovsub-krylov)."""
    N = A.shape[-1]
    beta = torch.linalg.vector_norm(psi_col)
    if float(beta.detach()) == 0.0:
        return torch.zeros_like(psi_col), 0
    kk = min(k, N)
    basis = [psi_col / beta]                                 # b_1 = psi/||psi||
    entries = {}                                             # (i, j) -> H_ij of A_k
    k_eff = kk
    for j in range(kk):
        w = A @ basis[j]
        for i in range(j + 1):                               # modified Gram-Schmidt
            entries[i, j] = torch.vdot(basis[i], w)          # b_i^dagger w
            w = w - entries[i, j] * basis[i]
        if j + 1 < kk:
            h = torch.linalg.vector_norm(w)
            if float(h.detach()) <= 1e-12 * float(normA.detach()):   # invariant subspace (R5)
                k_eff = j + 1
                break
            entries[j + 1, j] = h.to(psi_col.dtype)
            basis.append(w / h)
    # A_k assembled once all its entries exist (so that autograd can follow them)
    H = torch.zeros(k_eff, k_eff, dtype=psi_col.dtype)
    for (i, j), v in entries.items():
        if i < k_eff and j < k_eff:
            H[i, j] = v
    y = torch.linalg.matrix_exp(H)[:, 0] * beta              # e^{A_k} e_1 ||psi||
    out = torch.zeros_like(psi_col)
    for i in range(k_eff):
        out = out + y[i] * basis[i]                          # B_k y
    return out, k_eff


def krylov_action(A, psi, k):
    """krylov_k{A, psi} = B_k e^{A_k} e_1 ||psi|| for every orbital column."""
    if psi.dim() == 3:
        return torch.stack([krylov_action(A[w], psi[w], k) for w in range(psi.shape[0])])
    normA = torch.linalg.matrix_norm(A)
    cols = [_arnoldi_column(A, psi[:, j], k, normA)[0] for j in range(psi.shape[1])]
    return torch.stack(cols, dim=1)


def _bilinear(u, v):
    """u^T v, the symmetric bilinear form of complex-symmetric Lanczos (no conjugation)."""
    return (u * v).sum()


def _tridiagonal(alpha, beta):
    """Symmetric tridiagonal T with diagonal alpha and off-diagonals beta."""
    k = len(alpha)
    T = torch.zeros(k, k, dtype=CT)
    for j in range(k):
        T[j, j] = alpha[j]
    for j in range(k - 1):
        T[j + 1, j] = beta[j]
        T[j, j + 1] = beta[j]
    return T


def _lanczos_column(A, psi_col, k, normA, f=None):
    """Complex-symmetric Lanczos approximation of e^A psi for one orbital
    vector (reading R30).  The field matrix is complex symmetric (A^T = A,
    Eq. heffTOT with real symmetric L_g), so the three-term recurrence with
    the bilinear form u^T v builds a basis V_k of the Krylov space of Eq.
    krylovsub with V_k^T V_k = 1 and the symmetric tridiagonal
    T_k = V_k^T A V_k; the action is V_k f(T_k) e_1 beta with
    beta = (psi^T psi)^{1/2} (principal root; the result does not depend on
    the sign) and f = exp (Eq. krylov with the Hermitian projection replaced
    by the bilinear one).  The recurrence stops like the Arnoldi one (R5)
    when |beta_j| <= 1e-12 ||A||_F."""
    N = A.shape[-1]
    beta = torch.sqrt(_bilinear(psi_col, psi_col))
    if float(beta.detach().abs()) == 0.0:
        return torch.zeros_like(psi_col), 0
    kk = min(k, N)
    V = [psi_col / beta]
    alpha, off = [], []
    for j in range(kk):
        w = A @ V[j]
        if j > 0:
            w = w - off[j - 1] * V[j - 1]
        alpha.append(_bilinear(V[j], w))
        w = w - alpha[j] * V[j]
        if j + 1 < kk:
            b = torch.sqrt(_bilinear(w, w))
            if float(b.detach().abs()) <= 1e-12 * float(normA.detach()):
                break
            off.append(b)
            V.append(w / b)
    k_eff = len(alpha)
    T = _tridiagonal(alpha, off[:k_eff - 1])
    fT = torch.linalg.matrix_exp(T) if f is None else f(T)
    y = fT[:, 0] * beta
    out = torch.zeros_like(psi_col)
    for i in range(k_eff):
        out = out + y[i] * V[i]
    return out, k_eff


def lanczos_action(A, psi, k, f=None):
    """lanczos_k{A, psi} = V_k e^{T_k} e_1 (psi^T psi)^{1/2} for every orbital
    column (reading R30); f replaces exp for the pins."""
    if psi.dim() == 3:
        return torch.stack([lanczos_action(A[w], psi[w], k, f) for w in range(psi.shape[0])])
    normA = torch.linalg.matrix_norm(A)
    cols = [_lanczos_column(A, psi[:, j], k, normA, f)[0] for j in range(psi.shape[1])]
    return torch.stack(cols, dim=1)


def _block_arnoldi(A, X, k, normA):
    """Block-Krylov approximation of e^A X for one spin block X [N, n]
    (Eqs. bkrylovsub-bkrylov): X = B_1 R, the orthonormal basis
    B_k = [B_1 .. B_k] of span{X, A X, .., A^{k-1} X}, the block upper
    Hessenberg A_k = B_k^dagger A B_k, and bkrylov_k = B_k e^{A_k} E_n R."""
    N, n = X.shape
    if n == 0:
        return X.clone(), 0
    B1, Rx = mgs_qr(X)                                       # X = B_1 R
    kk = max(1, min(k, N // n))
    blocks = [B1]
    H = torch.zeros(kk * n, kk * n, dtype=CT)
    k_eff = kk
    for j in range(kk):
        W = A @ blocks[j]
        for i in range(j + 1):                               # block modified Gram-Schmidt
            Hij = blocks[i].conj().T @ W                     # B_i^dagger W
            H[i * n:(i + 1) * n, j * n:(j + 1) * n] = Hij
            W = W - blocks[i] @ Hij
        if j + 1 < kk:
            Bn, Rn = mgs_qr(W)                               # W = B_{j+1} H_{j+1,j}
            if float(Rn.diagonal().abs().min()) <= 1e-12 * float(normA):   # invariant (R20)
                k_eff = j + 1
                break
            H[(j + 1) * n:(j + 2) * n, j * n:(j + 1) * n] = Rn
            blocks.append(Bn)
    m = k_eff * n
    F = torch.linalg.matrix_exp(H[:m, :m])[:, :n] @ Rx      # e^{A_k} E_n R
    return torch.cat(blocks[:k_eff], dim=1) @ F, k_eff


def block_krylov_action(A, psi, k, spins=None):
    """bkrylov_k{A, Psi} for every spin block of psi [N, nc] (or [Nw, N, nc])."""
    if psi.dim() == 3:
        return torch.stack([block_krylov_action(A[w], psi[w], k, spins) for w in range(psi.shape[0])])
    normA = torch.linalg.matrix_norm(A)
    out = psi.clone()
    for sl in (spins if spins is not None else (slice(0, psi.shape[1]),)):
        if sl.stop > sl.start:
            out[:, sl] = _block_arnoldi(A, psi[:, sl], k, normA)[0]
    return out


def exact_action(A, psi):
    """e^A Psi by (non-Hermitian) diagonalisation, A = V diag(l) V^{-1} (Sec. IV)."""
    lam, V = torch.linalg.eig(A.to(CT))
    return V @ (torch.exp(lam)[..., :, None] * torch.linalg.solve(V, psi.to(CT)))


def expm_action(A, psi, method, k, spins=None):
    if method == "taylor":
        return taylor_action(A, psi, k)
    if method == "krylov":
        return krylov_action(A, psi, k)
    if method == "lanczos":
        return lanczos_action(A, psi, k)
    if method == "bkrylov":
        return block_krylov_action(A, psi, k, spins)
    if method == "chebyshev":
        return chebyshev_action(A, psi, k)
    if method == "exact":
        return exact_action(A, psi)
    raise ValueError(method)


def split2_propagate(B, A, psi, method, k, spins=None):
    """U_S2 Psi = e^{-tau H1/2} e^{A} e^{-tau H1/2} Psi (Sec. III.B)."""
    Bc = B.to(CT)
    return Bc @ expm_action(A, Bc @ psi, method, k, spins)


def split1_propagate(B, A, psi, method, k, spins=None):
    """U_S1 Psi = e^{-tau H1} e^{A} Psi (Sec. III.A, Split-1): the interaction
    exponential first, then the whole one-body step B B = e^{-tau h''}."""
    Bc = B.to(CT)
    return Bc @ (Bc @ expm_action(A, psi, method, k, spins))


def taylor_propagate(hpp, A, psi, tau, k):
    """U_T Psi = taylor_k{-tau Heff, Psi} with -tau Heff = A - tau h'' (Sec. III.C,
    Taylor propagator: the refactorised exponent expanded directly)."""
    return taylor_action(A - tau * hpp.to(CT), psi, k)


def crank_nicolson_propagate(hpp, A, psi, tau):
    """U_CN Psi = (1 + tau Heff/2)^{-1} (1 - tau Heff/2) Psi (Sec. III,
    Crank-Nicolson) with -tau Heff = A - tau h''."""
    X = A - tau * hpp.to(CT)
    eye = torch.eye(X.shape[-1], dtype=CT)
    return torch.linalg.solve(eye - 0.5 * X, psi + 0.5 * (X @ psi))


def propagate(propagator, B, hpp, A, psi, tau, method, k, spins=None):
    """The walker update of Eq. psiupdate for one of the propagators of Sec. III:
    "split2" (default), "split1", "taylor" (the Taylor propagator; k is its
    order and `method` is ignored) or "cn" (Crank-Nicolson)."""
    if propagator == "split2":
        return split2_propagate(B, A, psi, method, k, spins)
    if propagator == "split1":
        return split1_propagate(B, A, psi, method, k, spins)
    if propagator == "taylor":
        return taylor_propagate(hpp, A, psi, tau, k)
    if propagator == "cn":
        return crank_nicolson_propagate(hpp, A, psi, tau)
    raise ValueError(propagator)


# --------------------------------------------------------------------------
# Local energy and the mixed estimator (Eq. eloc; Sec. V.A capping)
# --------------------------------------------------------------------------
def local_energy(ham: Hamiltonian, psi):
    """E_L = <Psi_T|H|Psi>/<Psi_T|Psi> by Wick's theorem with the mixed density.

    E_L = E_const + sum_s sum_pq h_pq G^s_pq
          + 1/2 sum_pqrs V_pqrs [sum_{s,s'} G^s_pr G^s'_qs - sum_s G^s_ps G^s_qr],
    V_pqrs = sum_g L_g,pr L_g,qs, so the direct term is 1/2 sum_g (sum_s
    tr(L_g G^s^T))^2 and the exchange term 1/2 sum_g sum_s tr(L_g G^sT L_g G^sT).
    """
    if psi.dim() == 3 and psi.shape[0] * ham.G * ham.N * ham.N > (1 << 22):
        # bound the [walkers, G, N, N] temporaries: evaluate walker by walker
        return torch.stack([local_energy(ham, psi[w]) for w in range(psi.shape[0])])
    e = torch.full(psi.shape[:-2], ham.e_const, dtype=CT)
    direct = 0
    exch = 0
    L = ham.L.to(CT)
    for sl in ham.spins():
        if sl.stop == sl.start:
            continue
        Gs = greens_function(ham.trial[:, sl], psi[..., sl])
        e = e + torch.einsum("pq,...pq->...", ham.h1.to(CT), Gs)
        direct = direct + torch.einsum("gpr,...pr->...g", L, Gs)
        GT = Gs.transpose(-1, -2)
        M = torch.einsum("gpr,...rq->...gpq", L, GT)          # L_g G^T
        exch = exch + torch.einsum("...gpq,...gqp->...", M, M)
    return e + 0.5 * ((direct * direct).sum(-1) - exch)


def energy_window(e_loc, e0, tau, n_elec):
    """Capped local energy of Eq. enwin, DeltaE = 1/2 sqrt(N_e/tau) + sqrt(N_e tau)."""
    dE = 0.5 * math.sqrt(n_elec / tau) + math.sqrt(n_elec * tau)
    return torch.clamp(e_loc.real, e0 - dE, e0 + dE)


def mixed_energy(W, e_loc_capped):
    """E_k = sum_w W^w E_L^w / sum_w W^w over live walkers (Sec. II.A)."""
    live = W > 0
    Wl = torch.where(live, W, torch.zeros_like(W))
    El = torch.where(live, e_loc_capped, torch.zeros_like(e_loc_capped))
    return float((Wl * El).sum() / Wl.sum()), float(Wl.sum())


# --------------------------------------------------------------------------
# Re-orthonormalisation (reading R25: the paper is silent on the periodic
# orthonormalisation of the walkers; its only QR of Psi is the block-Krylov
# start Psi = B_1 R of Sec. IV.D, which is the same factorisation)
# --------------------------------------------------------------------------
def mgs_qr(X):
    """Modified Gram-Schmidt QR of the columns of X ([N, n]) -> (Q, R)."""
    N, n = X.shape
    Q = X.clone()
    R = torch.zeros(n, n, dtype=X.dtype)
    for j in range(n):
        for i in range(j):
            R[i, j] = torch.vdot(Q[:, i], Q[:, j])
            Q[:, j] = Q[:, j] - R[i, j] * Q[:, i]
        R[j, j] = torch.linalg.vector_norm(Q[:, j])
        Q[:, j] = Q[:, j] / R[j, j]
    return Q, R


def reorthonormalise(ham: Hamiltonian, psi):
    """Per walker and spin Psi_sigma <- Q of its MGS QR; returns (psi, logovl)."""
    out = psi.clone()
    batch = psi.shape[0] if psi.dim() == 3 else None
    for w in (range(batch) if batch is not None else [None]):
        for sl in ham.spins():
            if sl.stop == sl.start:
                continue
            X = psi[w][:, sl] if w is not None else psi[:, sl]
            Q, _ = mgs_qr(X)
            if w is not None:
                out[w][:, sl] = Q
            else:
                out[:, sl] = Q
    return out, log_overlap(ham, out)


# --------------------------------------------------------------------------
# Weights (Eqs. wupdate, hyben, phaseless, theta; Sec. V.B)
# --------------------------------------------------------------------------
@dataclass
class StepInfo:
    f: torch.Tensor          # capped force bias [Nw, G]
    n_fcap: torch.Tensor     # number of removed force-bias components [Nw]
    log_ratio: torch.Tensor  # log of the overlap ratio incl. the scalar s [Nw]
    log_I: torch.Tensor      # log of the importance factor [Nw]
    e_hybrid: torch.Tensor   # E_H [Nw] complex
    dtheta: torch.Tensor     # phase change in (-pi, pi] [Nw]
    factor: torch.Tensor     # capped reweighting factor [Nw]


def weight_update(W, log_ratio, log_I, tau, e0):
    """Phaseless update W' = W exp(-tau(Re E_H - E0)) max(0, cos dtheta).

    E_H = -(1/tau) log(ratio I) (Eq. hyben); dtheta = Im log ratio (Eq.
    theta), wrapped to (-pi, pi]; the reweighting factor is set to 0 unless
    it is < 10 (Sec. V.B).
    """
    e_h = -(log_ratio + log_I) / tau
    dth = torch.remainder(log_ratio.imag + math.pi, 2 * math.pi) - math.pi
    dth = torch.where(dth == -math.pi, torch.full_like(dth, math.pi), dth)
    fac = torch.exp(-tau * (e_h.real - e0))
    fac = torch.where(fac < 10.0, fac, torch.zeros_like(fac))
    Wn = W * fac * torch.clamp(torch.cos(dth), min=0.0)
    Wn = torch.where(torch.isfinite(Wn) & torch.isfinite(e_h.real), Wn, torch.zeros_like(Wn))
    return Wn, e_h, dth, fac


# --------------------------------------------------------------------------
# The walker step
# --------------------------------------------------------------------------
def init_walkers(ham: Hamiltonian, n_walkers):
    """Psi_0 = Psi_T, W_0 = 1, logovl_0 = log <Psi_T|Psi_T> (Sec. II.A)."""
    psi = ham.trial.to(CT).unsqueeze(0).repeat(n_walkers, 1, 1)
    W = torch.ones(n_walkers, dtype=RT)
    return psi, log_overlap(ham, psi), W


def propagate_and_ratio(ham: Hamiltonian, psi, logovl, x, tau, method, k, B, L_bar, ec,
                        hpp=None, propagator="split2"):
    """The part of one step that the phaseless and the free-projection walks
    share: force bias, field matrix, walker update, and the two factors of the
    weight.

    f_g = -i sqrt(tau)(<L_g> - L_bar_g), capped (Eq. force_shift, Sec. V.C);
    c_g = x_g - f_g and A = i sqrt(tau) sum_g c_g L_g (Eq. heffTOT);
    Psi' = U Psi (Eq. psiupdate, Sec. III);
    log ratio = log<Psi_T|Psi'> - log<Psi_T|Psi> + log s with the scalar
    s = exp(-tau E_c' - i sqrt(tau) sum_g c_g L_bar_g) of reading R1;
    log I = sum_g (x_g f_g - f_g^2 / 2), the importance factor that goes with
    the shifted fields (Eq. wupdate).
    Returns (psi', logovl', log_ratio, log_I, f, f_uncapped).
    """
    x = torch.as_tensor(x, dtype=RT)
    f, f_raw = force_bias(ham, psi, tau, L_bar)                     # Eq. force_shift
    c = x.to(CT) - f
    A = field_matrix(ham, c, tau)                                   # Eq. heffTOT
    psi_new = propagate(propagator, B, hpp, A, psi, tau, method, k, ham.spins())   # Eq. psiupdate
    logovl_new = log_overlap(ham, psi_new)
    log_s = -tau * ec - 1j * math.sqrt(tau) * (c @ L_bar.to(CT))
    log_ratio = logovl_new - logovl + log_s
    log_I = (x.to(CT) * f - 0.5 * f * f).sum(-1)                    # importance factor
    return psi_new, logovl_new, log_ratio, log_I, f, f_raw


def step(ham: Hamiltonian, psi, logovl, W, x, tau, e0, method="krylov", k=10,
         reortho=False, B=None, L_bar=None, ec=None, propagator="split2"):
    """One phaseless walker step (by default with the Split-2 propagator;
    `propagator` selects another walker update of Sec. III, see `propagate`).

    psi [Nw, N, na+nb] complex, logovl [Nw] complex, W [Nw] real, x [Nw, G]
    real standard-normal fields.  Walkers with W = 0 are kept as they are.
    Returns (psi', logovl', W', StepInfo).
    """
    if L_bar is None:
        L_bar = mean_field_shift(ham)
    hpp = None
    if B is None or ec is None or propagator in ("taylor", "cn"):
        hpp, ec = propagation_h1(ham, L_bar)
        B = half_step_propagator(hpp, tau) if B is None else B
    psi_new, logovl_new, log_ratio, log_I, f, f_raw = propagate_and_ratio(
        ham, psi, logovl, x, tau, method, k, B, L_bar, ec, hpp, propagator)
    W_new, e_h, dth, fac = weight_update(W, log_ratio, log_I, tau, e0)
    if reortho:
        psi_new, logovl_new = reorthonormalise(ham, psi_new)
    alive = W > 0
    psi_out = torch.where(alive[:, None, None], psi_new, psi)
    logovl_out = torch.where(alive, logovl_new, logovl)
    W_out = torch.where(alive, W_new, W)
    info = StepInfo(f=f, n_fcap=(f_raw.abs() >= 1.0).sum(-1), log_ratio=log_ratio,
                    log_I=log_I, e_hybrid=e_h, dtheta=dth, factor=fac)
    return psi_out, logovl_out, W_out, info


def free_projection_step(ham: Hamiltonian, psi, logovl, weight, x, tau, e0,
                         method="taylor", k=6, B=None, L_bar=None, ec=None):
    """Free-projection step (Eqs. psiupdate, wupdate): complex weight, no phaseless cut.

    weight' = weight * ratio * I * e^{tau E0} = weight e^{-tau(E_H - E0)}, with
    the ratio and I of `propagate_and_ratio`, the same code as the phaseless step.
    """
    if L_bar is None:
        L_bar = mean_field_shift(ham)
    if B is None or ec is None:
        hpp, ec = propagation_h1(ham, L_bar)
        B = half_step_propagator(hpp, tau)
    psi_new, logovl_new, log_ratio, log_I, _, _ = propagate_and_ratio(
        ham, psi, logovl, x, tau, method, k, B, L_bar, ec)
    return psi_new, logovl_new, weight * torch.exp(log_ratio + log_I + tau * e0)


# --------------------------------------------------------------------------
# Population control (the paper is silent; reading R8)
# --------------------------------------------------------------------------
def comb(W, u):
    """Comb resampling (reading R8): with cumulative weights C_w = W_0 + ... + W_w
    summed in walker order, tooth j sits at (u + j) C_{Nw-1} / Nw and picks the
    first walker whose C_w exceeds it (zero-weight walkers are never picked).
    Returns the indices [Nw]."""
    W = [float(x) for x in torch.as_tensor(W, dtype=RT)]
    n = len(W)
    cum = []
    acc = 0.0
    for x in W:
        acc = acc + x
        cum.append(acc)
    total = cum[-1]
    idx = []
    w = 0
    for j in range(n):
        tooth = (u + j) * total / n
        while w < n - 1 and not (tooth < cum[w]):
            w += 1
        idx.append(w)
    return torch.tensor(idx, dtype=torch.int64)


def population_control(psi, logovl, W, u):
    """Replace the population by Nw comb-selected copies, each of weight
    C_{Nw-1} / Nw (the total weight is kept)."""
    idx = comb(W, u)
    total = 0.0
    for x in torch.as_tensor(W, dtype=RT).tolist():
        total = total + x
    n = W.shape[0]
    return psi[idx].clone(), logovl[idx].clone(), torch.full((n,), total / n, dtype=RT), idx


# --------------------------------------------------------------------------
# Objective of the adjoint (the paper has no gradients; reading R10)
# --------------------------------------------------------------------------
def _reortho_fixed_R(ham: Hamiltonian, psi, alive):
    """Psi_sigma <- Psi_sigma R^{-1} with R of the MGS QR held constant
    (reading R10), for live walkers; dead walkers are returned unchanged."""
    out = []
    for w in range(psi.shape[0]):
        if not bool(alive[w]):
            out.append(psi[w])
            continue
        blocks = []
        for sl in ham.spins():
            if sl.stop == sl.start:
                continue
            X = psi[w][:, sl]
            with torch.no_grad():
                _, Rm = mgs_qr(X.detach().clone())
            blocks.append(X @ torch.linalg.inv(Rm))
        out.append(torch.cat(blocks, dim=1))
    return torch.stack(out)


def walk_objective(ham: Hamiltonian, psi0, W0, fields, tau, e0, k=6, reortho_every=0, method="taylor"):
    """J = E_n, the mixed estimator of the capped local energy after n
    fixed-field Split-2 steps with the Taylor exponential of order k (Sec.
    II.A, Sec. III.B, Eq. taylor) or another action of Sec. IV (`method`, e.g.
    "krylov" of dimension k, differentiated through the Arnoldi steps and the
    small exponential), as a function that torch autograd differentiates with
    respect to ham.h1, ham.L and psi0.

    Reading R10: the fields are fixed inputs; every threshold decision is
    whatever the forward walk takes (torch.where / clamp give zero derivative
    in a removed or capped branch); L_bar, h'', E_c' and B are recomputed from
    ham.h1 and ham.L; the initial log-overlap follows psi0; after step k with
    (k+1) % reortho_every == 0 the orbitals of live walkers are multiplied by
    R^{-1} of their MGS QR, R held constant.  Returns (J, W_n, E_L(Psi_n)).
    """
    L_bar = mean_field_shift(ham)
    hpp, ec = propagation_h1(ham, L_bar)
    B = half_step_propagator(hpp, tau)
    psi = psi0
    logovl = log_overlap(ham, psi)
    W = torch.as_tensor(W0, dtype=RT)
    for kk, x in enumerate(fields):
        alive = W > 0
        psi, logovl, W, _ = step(ham, psi, logovl, W, x, tau, e0, method=method, k=k,
                                 reortho=False, B=B, L_bar=L_bar, ec=ec)
        if reortho_every and (kk + 1) % reortho_every == 0:
            psi = _reortho_fixed_R(ham, psi, alive)
            logovl = torch.where(alive, log_overlap(ham, psi), logovl)
    El = local_energy(ham, psi)
    live = W > 0
    Ebar = torch.where(live, energy_window(El, e0, tau, ham.na + ham.nb), torch.zeros_like(W))
    Wl = torch.where(live, W, torch.zeros_like(W))
    return (Wl * Ebar).sum() / Wl.sum(), W, El

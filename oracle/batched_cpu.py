"""Batched FP64 CPU variant of the walker step (measurement infrastructure).

The arithmetic of oracle.afqmc_ref.step (Split-2 with the Krylov action,
phaseless weights, optional re-orthonormalisation) followed by the local
energy and the mixed estimate, written for throughput on the host cores:
every per-walker operation is one batched tensor operation over the walkers,
and the Krylov action runs Arnoldi on all orbital columns of all walkers at
once.  The contractions with the Cholesky vectors use the half-rotated
vectors Lh_g = trial^T L_g, which the trial's Green's function allows
(tr(L_g G^T) = tr(Lh_g Theta), tr(L_g G^T L_g G^T) = tr(T_g T_g) with
T_g = Lh_g Theta, Eq. eloc), and products of real and complex tensors are
taken as two real products.  It is the "batched" CPU baseline beside the
walker-by-walker oracle: the tests compare it with the oracle, and only the
benchmark's CPU-baseline leg runs it.  It shares no code with the CUDA
library.  Plain PyTorch CPU, float64 / complex128.
"""
from __future__ import annotations

import math

import torch

from . import afqmc_ref as R

RT, CT = torch.float64, torch.complex128


def _rc(real, z):
    """real @ z for a real matrix and a complex operand, as two real products."""
    return torch.complex(real @ z.real, real @ z.imag)


class BatchedStep:
    """One context: the Hamiltonian's derived quantities (reading R1) for a
    time step tau, then `step` and `local_energy` over walker batches
    psi [Nw, N, na+nb]."""

    def __init__(self, ham: R.Hamiltonian, tau: float):
        self.ham, self.tau = ham, float(tau)
        N, G = ham.N, ham.G
        self.Lbar = R.mean_field_shift(ham)                  # Eq. force_shift
        self.hpp, self.ec = R.propagation_h1(ham, self.Lbar)
        self.B = R.half_step_propagator(self.hpp, tau)       # e^{-tau h''/2}, real
        self.Lflat = ham.L.reshape(G, N * N)
        self.spins = [sl for sl in ham.spins() if sl.stop > sl.start]
        self.trial = [ham.trial[:, sl] for sl in self.spins]                    # [N, n] real
        self.Lh = [torch.einsum("pi,gpq->giq", t, ham.L) for t in self.trial]  # [G, n, N] real
        self.hh = [t.T @ ham.h1 for t in self.trial]                            # [n, N] real

    # Theta_s = psi_s (trial_s^T psi_s)^{-1} and log det per spin
    def _theta_logdet(self, psi):
        thetas, logov = [], torch.zeros(psi.shape[0], dtype=CT)
        for sl, t in zip(self.spins, self.trial):
            ps = psi[..., sl]
            O = torch.complex(t.T @ ps.real, t.T @ ps.imag)
            sign, logabs = torch.linalg.slogdet(O)
            logov = logov + logabs + 1j * torch.angle(sign)
            thetas.append(torch.linalg.solve(O.transpose(-1, -2), ps.transpose(-1, -2)).transpose(-1, -2))
        return thetas, logov

    def log_overlap(self, psi):
        return self._theta_logdet(psi)[1]

    def _traces(self, thetas):
        """t_g = sum_s tr(Lh_gs Theta_s)  [Nw, G] (the mixed <L_g>)."""
        t = 0
        for Lh, th in zip(self.Lh, thetas):
            t = t + torch.complex(torch.einsum("giq,wqi->wg", Lh, th.real), torch.einsum("giq,wqi->wg", Lh, th.imag))
        return t

    def krylov(self, A, X, k):
        """Column Arnoldi (Eqs. krylovsub-krylov, reading R5) on every column
        of X [Nw, N, nc] at once; a column whose subdiagonal entry falls to
        1e-12 ||A||_F continues with zero vectors, which leaves the leading
        block of its Hessenberg matrix and so e^{A_k} e_1 unchanged."""
        Nw, N, nc = X.shape
        kk = min(k, N)
        V = X.transpose(1, 2)                                    # [Nw, nc, N]
        beta = torch.linalg.vector_norm(V, dim=-1)               # [Nw, nc]
        inv = torch.where(beta > 0, 1.0 / torch.where(beta > 0, beta, torch.ones_like(beta)),
                          torch.zeros_like(beta))
        basis = [V * inv[..., None]]
        H = torch.zeros(Nw, nc, kk, kk, dtype=CT)
        thr = 1e-12 * torch.linalg.matrix_norm(A)                # [Nw]
        for j in range(kk):
            w = torch.matmul(basis[j], A.transpose(1, 2))        # rows: A b_j
            for i in range(j + 1):
                h = (basis[i].conj() * w).sum(-1)                # b_i^dagger w
                H[:, :, i, j] = h
                w = w - h[..., None] * basis[i]
            if j + 1 < kk:
                nu = torch.linalg.vector_norm(w, dim=-1)
                keep = nu > thr[:, None]
                safe = torch.where(keep, nu, torch.ones_like(nu))
                H[:, :, j + 1, j] = torch.where(keep, nu, torch.zeros_like(nu)).to(CT)
                basis.append(torch.where(keep[..., None], w / safe[..., None], torch.zeros_like(w)))
        y = torch.linalg.matrix_exp(H)[..., :, 0] * beta[..., None]   # [Nw, nc, kk]
        out = 0
        for i in range(kk):
            out = out + y[..., i:i + 1] * basis[i]
        return out.transpose(1, 2)                               # [Nw, N, nc]

    def step(self, psi, logovl, W, x, e0, k=10, reortho=False):
        """One phaseless Split-2 + Krylov step (oracle.afqmc_ref.step)."""
        tau, ham = self.tau, self.ham
        x = torch.as_tensor(x, dtype=RT)
        thetas, _ = self._theta_logdet(psi)
        f = -1j * math.sqrt(tau) * (self._traces(thetas) - self.Lbar)
        f = torch.where(f.abs() < 1.0, f, torch.zeros_like(f))     # Sec. V.C
        c = x.to(CT) - f
        st = math.sqrt(tau)
        # A = i sqrt(tau) sum_g c_g L_g (Eq. heffTOT) by two real products
        A = torch.complex(-st * (c.imag @ self.Lflat), st * (c.real @ self.Lflat)).reshape(-1, ham.N, ham.N)
        psi_new = _rc(self.B, self.krylov(A, _rc(self.B, psi), k))
        logovl_new = self.log_overlap(psi_new)
        log_s = -tau * self.ec - 1j * st * (c @ self.Lbar.to(CT))
        log_ratio = logovl_new - logovl + log_s
        log_I = (x.to(CT) * f - 0.5 * f * f).sum(-1)
        W_new, _, _, _ = R.weight_update(W, log_ratio, log_I, tau, e0)
        if reortho:
            psi_new, logovl_new = self.reorthonormalise(psi_new)
        alive = W > 0
        return (torch.where(alive[:, None, None], psi_new, psi), torch.where(alive, logovl_new, logovl),
                torch.where(alive, W_new, W))

    def reorthonormalise(self, psi):
        """Psi_s <- Q of its QR with a positive real diagonal of R (the Q of
        modified Gram-Schmidt, reading R25), per walker and spin."""
        out = psi.clone()
        for sl in self.spins:
            Q, Rm = torch.linalg.qr(psi[..., sl])
            d = torch.diagonal(Rm, dim1=-2, dim2=-1)
            ph = torch.where(d.abs() > 0, d / torch.where(d.abs() > 0, d.abs(), torch.ones_like(d.abs())),
                             torch.ones_like(d))
            out[..., sl] = Q * ph[..., None, :]
        return out, self.log_overlap(out)

    def local_energy(self, psi):
        """E_L (Eq. eloc) with the half-rotated vectors: E_const +
        sum_s tr(h_half,s Theta_s) + 1/2 sum_g [(sum_s tr T_gs)^2 - sum_s tr(T_gs T_gs)]."""
        thetas, _ = self._theta_logdet(psi)
        e = torch.full((psi.shape[0],), self.ham.e_const, dtype=CT)
        direct = 0
        exch = torch.zeros(psi.shape[0], dtype=CT)
        G, N = self.ham.G, self.ham.N
        for hh, Lh, th in zip(self.hh, self.Lh, thetas):
            n = th.shape[-1]
            e = e + torch.complex(torch.einsum("iq,wqi->w", hh, th.real), torch.einsum("iq,wqi->w", hh, th.imag))
            Lf = Lh.reshape(G * n, N)
            for w in range(psi.shape[0]):                      # T_g for all g by one product per walker
                T = _rc(Lf, th[w]).reshape(G, n, n)
                exch[w] = exch[w] + (T * T.transpose(-1, -2)).sum()
            direct = direct + torch.complex(torch.einsum("giq,wqi->wg", Lh, th.real),
                                            torch.einsum("giq,wqi->wg", Lh, th.imag))
        return e + 0.5 * ((direct * direct).sum(-1) - exch)

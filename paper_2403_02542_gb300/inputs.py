"""Seeded synthetic inputs for the ph-AFQMC walker step.

This module only *generates* inputs: a one-body matrix h1, Cholesky vectors
L_g, a closed-shell RHF trial determinant and Gaussian auxiliary fields.  It
contains none of the walker-step arithmetic; both the CUDA path and the CPU
oracle receive the arrays it returns.

The molecules of the paper (HEAT set, water clusters, N2) cannot be built
without integral code, so these Hamiltonians stand in for them with the
paper's shape relations (Sec. II.A: N_g of the order of 5-10 N; Sec. VI.B:
N = 855, 40 electrons, 5685 vectors for the largest run):

* h1: strict upper triangle i.i.d. N(0, 0.1^2), mirrored; diagonal i.i.d.
  U(-2, 0).
* L_g = sqrt(lambda_g) U_g, where U_g are random real symmetric N x N
  matrices orthonormalised in the Frobenius inner product, so that the
  two-electron integrals <pq|rs> = sum_g L_g,pr L_g,qs (Sec. II.A) are PSD
  with rank N_g and eigenvalues lambda_g = lambda0 * rho^g.
* trial: RHF orbitals, i.e. the lowest n eigenvectors of the closed-shell
  Fock matrix F = h + sum_g [2 tr(L_g P) L_g - L_g P L_g], P = C C^T,
  iterated with Fock-matrix damping to a fixed point.

The batched workload (16 uneven systems up to N = 400 with N_g = 5N) uses a
recipe whose cost does not grow as N^4 per SCF iteration or as a QR of
N^2 x N_g: L_g = sqrt(lambda_g) S_g / ||S_g||_F with S_g random symmetric
(not orthogonalised; the two-electron integrals stay PSD with rank <= N_g),
and the trial is the lowest n eigenvectors of the Fock matrix of the
core-guess density (one Fock step instead of a converged SCF).

The random generator is numpy's PCG64 throughout.
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "System",
    "make_system",
    "make_fields",
    "config_system",
    "batched_systems",
    "CONFIGS",
]


@dataclasses.dataclass
class System:
    """A synthetic Hamiltonian plus its trial determinant.

    Attributes:
      h1:      [N, N] float64, symmetric one-body matrix.
      L:       [G, N, N] float64, symmetric Cholesky vectors.
      trial:   [N, na + nb] float64; columns [0, na) are the alpha orbitals,
               columns [na, na + nb) the beta orbitals (orthonormal per spin).
      na, nb:  electrons per spin.
      e_const: constant energy shift (0 for the synthetic systems).
      meta:    the recipe parameters, for logging.
    """

    h1: np.ndarray
    L: np.ndarray
    trial: np.ndarray
    na: int
    nb: int
    e_const: float = 0.0
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.h1.shape[0]

    @property
    def G(self) -> int:
        return self.L.shape[0]


def _random_h1(rng: np.random.Generator, N: int) -> np.ndarray:
    h = np.zeros((N, N))
    iu = np.triu_indices(N, 1)
    h[iu] = rng.normal(0.0, 0.1, size=len(iu[0]))
    h = h + h.T
    h[np.diag_indices(N)] = rng.uniform(-2.0, 0.0, size=N)
    return h


def _random_cholesky(rng: np.random.Generator, N: int, G: int, rho: float,
                     lambda0: float) -> np.ndarray:
    if G > N * (N + 1) // 2:
        raise ValueError("more Cholesky vectors than symmetric N x N matrices")
    X = rng.normal(size=(G, N, N))
    X = 0.5 * (X + X.transpose(0, 2, 1))
    # Orthonormalise the G symmetric matrices in the Frobenius inner product
    # (a QR of their vectorisations; Q's columns stay symmetric matrices).
    Q, R = np.linalg.qr(X.reshape(G, N * N).T)
    Q = Q * np.sign(np.diag(R))[None, :]
    U = Q.T.reshape(G, N, N)
    U = 0.5 * (U + U.transpose(0, 2, 1))
    lam = lambda0 * rho ** np.arange(G)
    return np.sqrt(lam)[:, None, None] * U


def _rhf_orbitals(h1: np.ndarray, L: np.ndarray, n: int, tol: float = 1e-10,
                  max_iter: int = 1000, damping: float = 0.5) -> tuple[np.ndarray, dict]:
    """Closed-shell RHF by Roothaan iterations with Fock-matrix damping."""
    _, C = np.linalg.eigh(h1)
    C = C[:, :n]
    P = C @ C.T
    F_prev = None
    converged = False
    it = 0
    G, N = L.shape[0], L.shape[1]
    Lf = L.reshape(G, N * N)
    for it in range(1, max_iter + 1):
        coul = Lf @ P.reshape(N * N)                # tr(L_g P)
        LC = L @ C                                  # [G, N, n]
        M = LC.transpose(1, 0, 2).reshape(N, G * n)
        K = M @ M.T                                 # sum_g L_g P L_g
        F = h1 + 2.0 * (coul @ Lf).reshape(N, N) - K
        if F_prev is not None:
            F = (1.0 - damping) * F + damping * F_prev
        F_prev = F
        _, V = np.linalg.eigh(F)
        C = V[:, :n]
        Pn = C @ C.T
        dP = np.abs(Pn - P).max()
        P = Pn
        if dP < tol:
            converged = True
            break
    return C.copy(), {"scf_iterations": it, "scf_converged": converged}


def make_system(N: int, na: int, nb: int, G: int, *, rho: float, seed: int,
                lambda0: float = 1.0) -> System:
    """Build one synthetic system (recipe in the module docstring)."""
    if na != nb:
        raise ValueError("the synthetic recipe builds closed-shell RHF trials")
    rng = np.random.Generator(np.random.PCG64(seed))
    h1 = _random_h1(rng, N)
    L = _random_cholesky(rng, N, G, rho, lambda0)
    C, info = _rhf_orbitals(h1, L, na)
    trial = np.concatenate([C, C], axis=1)
    meta = dict(N=N, na=na, nb=nb, G=G, rho=rho, lambda0=lambda0, seed=seed, **info)
    return System(h1=h1, L=L, trial=np.ascontiguousarray(trial), na=na, nb=nb,
                  e_const=0.0, meta=meta)


def make_fields(seed: int, step: int, n_walkers: int, G: int) -> np.ndarray:
    """Standard-normal auxiliary fields x_g^w for one step, [n_walkers, G]."""
    rng = np.random.Generator(np.random.PCG64([seed, step]))
    return rng.standard_normal((n_walkers, G))


# The workloads: sizes, decay and seeds.  rho for a cutoff c over G vectors is
# c**(1/G), so that lambda_{G-1} is close to the cutoff.
CONFIGS = {
    # small FP64 case: N=8, 2+2 electrons, 32 vectors decaying as 0.5^g,
    # 64 walkers, tau=0.01, Split-2 Taylor-6, 200 steps, QR every 5 steps
    "small": dict(N=8, na=2, G=32, rho=0.5, walkers=64, tau=0.01, steps=200,
                  expm="taylor", order=6, reortho=5),
    # large-step plain method: N=128, 20+20 electrons, 640 vectors,
    # 1024 walkers, Split-2 with Krylov dimension 10, QR every 5 steps
    "large": dict(N=128, na=20, G=640, rho=1e-5 ** (1.0 / 640), walkers=1024,
                  tau=0.05, steps=500, expm="krylov", order=10, reortho=5),
    # precision form: N=300, 50+50 electrons, 1500 vectors, 2048 walkers
    "precision": dict(N=300, na=50, G=1500, rho=1e-5 ** (1.0 / 1500),
                      walkers=2048, tau=0.05, steps=50, expm="krylov", order=10,
                      reortho=5),
    # differentiation form: N=96, 15+15 electrons, 480 vectors, 512 walkers
    "grad": dict(N=96, na=15, G=480, rho=1e-5 ** (1.0 / 480), walkers=512,
                 tau=0.05, steps=100, expm="taylor", order=6, reortho=10),
}
_CONFIG_INDEX = {"small": 1, "large": 2, "precision": 3, "grad": 5}


_SYSTEM_CACHE: dict = {}


def config_system(name: str, system: int = 0, **overrides) -> System:
    """The synthetic system of a named workload; seed 20240304 + 100*config + system.

    Generated once per process and key (the N = 300 workload takes tens of
    seconds); every call returns its own copy of the arrays."""
    c = dict(CONFIGS[name])
    c.update(overrides)
    seed = 20240304 + 100 * _CONFIG_INDEX.get(name, 9) + system
    key = (c["N"], c["na"], c["G"], c["rho"], seed)
    if key not in _SYSTEM_CACHE:
        _SYSTEM_CACHE[key] = make_system(c["N"], c["na"], c["na"], c["G"], rho=c["rho"], seed=seed)
    s = _SYSTEM_CACHE[key]
    return dataclasses.replace(s, h1=s.h1.copy(), L=s.L.copy(), trial=s.trial.copy(), meta=dict(s.meta))


def _plain_cholesky(rng: np.random.Generator, N: int, G: int, rho: float, chunk: int = 64) -> np.ndarray:
    """L_g = sqrt(rho^g) S_g / ||S_g||_F, S_g random symmetric, in chunks of g."""
    L = np.empty((G, N, N))
    for g0 in range(0, G, chunk):
        g1 = min(G, g0 + chunk)
        X = rng.standard_normal((g1 - g0, N, N), dtype=np.float32)
        X = X + X.transpose(0, 2, 1)
        scale = np.sqrt(rho ** np.arange(g0, g1)) / np.sqrt(np.einsum("gpq,gpq->g", X, X, dtype=np.float64))
        np.multiply(X, scale[:, None, None], out=L[g0:g1])
    return L


def _one_step_fock_orbitals(h1: np.ndarray, L: np.ndarray, n: int, chunk: int = 64) -> np.ndarray:
    """Lowest n eigenvectors of F = h + sum_g [2 tr(L_g P) L_g - L_g P L_g] for
    the core-guess density P = C C^T (C: lowest n eigenvectors of h)."""
    _, C = np.linalg.eigh(h1)
    C = C[:, :n]
    N = h1.shape[0]
    F = h1.copy()
    for g0 in range(0, L.shape[0], chunk):
        Lc = L[g0:g0 + chunk]
        m = Lc.shape[0]
        LC = (Lc.reshape(m * N, N) @ C).reshape(m, N, n)          # L_g C
        coul = (LC * C[None]).sum(axis=(1, 2))                    # tr(L_g P)
        F += 2.0 * np.tensordot(coul, Lc, axes=1)
        M = LC.transpose(1, 0, 2).reshape(N, m * n)
        F -= M @ M.T                                              # sum_g L_g P L_g
    F = 0.5 * (F + F.T)
    _, V = np.linalg.eigh(F)
    return V[:, :n]


def batched_systems(seed: int = 20240304 + 400, n_systems: int = 16, n_min: int = 64, n_max: int = 400,
                    walkers: tuple = (256, 2048)) -> list:
    """The batched workload: n_systems systems with N uniform in [n_min, n_max],
    n = N // 6 electrons per spin, N_g = 5N vectors decaying to 1e-5, and a
    walker count uniform in `walkers` for each.  Returns [(System, n_walkers)]."""
    from concurrent.futures import ThreadPoolExecutor
    import os

    rng = np.random.Generator(np.random.PCG64(seed))
    Ns = rng.integers(n_min, n_max + 1, size=n_systems).tolist()
    nws = rng.integers(walkers[0], walkers[1] + 1, size=n_systems).tolist()

    def build(i):  # every system has its own generator: the result does not depend on the threads
        r = np.random.Generator(np.random.PCG64([seed, i]))
        N = Ns[i]
        n, G = N // 6, 5 * N
        rho = 1e-5 ** (1.0 / G)
        h1 = _random_h1(r, N)
        L = _plain_cholesky(r, N, G, rho)
        C = _one_step_fock_orbitals(h1, L, n)
        meta = dict(N=N, na=n, nb=n, G=G, rho=rho, seed=[seed, i], recipe="batched")
        return (System(h1=h1, L=L, trial=np.ascontiguousarray(np.concatenate([C, C], axis=1)), na=n, nb=n,
                       e_const=0.0, meta=meta), int(nws[i]))

    with ThreadPoolExecutor(max_workers=min(n_systems, os.cpu_count() or 1)) as ex:
        return list(ex.map(build, range(n_systems)))

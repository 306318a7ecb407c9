"""Brute-force full configuration interaction in second quantisation.

Independent of the oracle: determinants are bit strings over 2N spin
orbitals, operators act by explicit creation/annihilation with fermionic
signs, and the Hamiltonian of Eq. mbham, H = sum h_pq a+_p a_q
+ 1/2 sum V_pqrs a+_p a+_q a_s a_r with V_pqrs = sum_g L_g,pr L_g,qs,
is assembled element by element in the (na, nb) sector and diagonalised.
"""
import itertools

import numpy as np


def _annihilate(det, j):
    if not (det >> j) & 1:
        return None, 0
    sign = -1 if bin(det & ((1 << j) - 1)).count("1") % 2 else 1
    return det & ~(1 << j), sign


def _create(det, i):
    if (det >> i) & 1:
        return None, 0
    sign = -1 if bin(det & ((1 << i) - 1)).count("1") % 2 else 1
    return det | (1 << i), sign


def _apply(ops, det):
    """Apply a product of operators, rightmost first. ops: list of (kind, orbital)."""
    sign = 1
    for kind, orb in reversed(ops):
        det, s = (_create if kind == "+" else _annihilate)(det, orb)
        if det is None:
            return None, 0
        sign *= s
    return det, sign


def sector_basis(N, na, nb):
    dets = []
    for occ_a in itertools.combinations(range(N), na):
        for occ_b in itertools.combinations(range(N), nb):
            d = 0
            for p in occ_a:
                d |= 1 << p
            for p in occ_b:
                d |= 1 << (N + p)
            dets.append(d)
    return dets


def hamiltonian_matrix(h1, L, na, nb, e_const=0.0):
    N = h1.shape[0]
    V = np.einsum("gpr,gqs->pqrs", L, L)
    dets = sector_basis(N, na, nb)
    index = {d: i for i, d in enumerate(dets)}
    H = np.zeros((len(dets), len(dets)))
    so = [(p, s) for s in range(2) for p in range(N)]
    for col, d in enumerate(dets):
        H[col, col] += e_const
        for (p, sp), (q, sq) in itertools.product(so, so):
            if sp != sq or h1[p, q] == 0.0:
                continue
            nd, sg = _apply([("+", p + sp * N), ("-", q + sq * N)], d)
            if nd is not None:
                H[index[nd], col] += h1[p, q] * sg
        for (p, s1), (q, s2) in itertools.product(so, so):
            for r, s in itertools.product(range(N), range(N)):
                v = V[p, q, r, s]
                if v == 0.0:
                    continue
                # a+_{p s1} a+_{q s2} a_{s s2} a_{r s1}
                nd, sg = _apply([("+", p + s1 * N), ("+", q + s2 * N),
                                 ("-", s + s2 * N), ("-", r + s1 * N)], d)
                if nd is not None:
                    H[index[nd], col] += 0.5 * v * sg
    return H, dets


def ground_state_energy(h1, L, na, nb, e_const=0.0):
    H, _ = hamiltonian_matrix(h1, L, na, nb, e_const)
    return float(np.linalg.eigvalsh(0.5 * (H + H.T))[0])


def determinant_energy(h1, L, C_a, C_b, e_const=0.0):
    """<D|H|D> of a single determinant with real orthonormal orbitals, by
    expanding D in the sector basis and taking the FCI matrix element."""
    N = h1.shape[0]
    na, nb = C_a.shape[1], C_b.shape[1]
    H, dets = hamiltonian_matrix(h1, L, na, nb, e_const)
    vec = np.zeros(len(dets))
    for i, d in enumerate(dets):
        occ_a = [p for p in range(N) if (d >> p) & 1]
        occ_b = [p for p in range(N) if (d >> (N + p)) & 1]
        ca = np.linalg.det(C_a[occ_a, :]) if na else 1.0
        cb = np.linalg.det(C_b[occ_b, :]) if nb else 1.0
        vec[i] = ca * cb
    return float(vec @ H @ vec / (vec @ vec))

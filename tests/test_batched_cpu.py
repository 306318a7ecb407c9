"""The batched FP64 CPU variant of the step (oracle/batched_cpu.py, the
benchmark's batched CPU baseline) against the walker-by-walker oracle on the
same seeded systems and fields: walkers, log-overlaps, weights and local
energies element by element within 1e-10 relative, including
re-orthonormalisation, a dead walker, unequal spins and a Krylov dimension
above N (the whole space)."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from oracle.batched_cpu import BatchedStep
from paper_2403_02542_gb300.inputs import make_fields, make_system

RTOL = 1e-10


def _rel(a, b):
    return float((a - b).abs().max() / max(float(b.abs().max()), 1e-300))


@pytest.mark.parametrize("N,na,nb,G,nw,steps,k,reo,dead", [
    (10, 2, 2, 14, 5, 4, 6, 2, (1,)),
    (12, 3, 1, 20, 4, 3, 14, 0, ()),      # k > N: the whole space
    (16, 3, 0, 24, 3, 3, 8, 1, ()),       # no beta electrons
])
def test_batched_step_matches_oracle(N, na, nb, G, nw, steps, k, reo, dead):
    base = make_system(N, na, na, G, rho=0.8, seed=N + G)
    trial = np.concatenate([base.trial[:, :na], base.trial[:, na:na + nb]], axis=1)
    s = dataclasses.replace(base, trial=trial, na=na, nb=nb)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, na, nb, s.e_const)
    tau = 0.05
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    Lbar = R.mean_field_shift(ham)
    hpp, ec = R.propagation_h1(ham, Lbar)
    B = R.half_step_propagator(hpp, tau)
    bs = BatchedStep(ham, tau)
    psi, lo, W = R.init_walkers(ham, nw)
    for d in dead:
        W[d] = 0.0
    bpsi, blo, bW = psi.clone(), bs.log_overlap(psi), W.clone()
    assert _rel(blo, lo) <= RTOL
    for kk in range(steps):
        x = make_fields(7, kk, nw, G)
        reortho = reo > 0 and (kk + 1) % reo == 0
        psi, lo, W, _ = R.step(ham, psi, lo, W, x, tau, e0, method="krylov", k=k, reortho=reortho,
                               B=B, L_bar=Lbar, ec=ec)
        bpsi, blo, bW = bs.step(bpsi, blo, bW, x, e0, k=k, reortho=reortho)
        assert _rel(bpsi, psi) <= RTOL, kk
        assert _rel(torch.exp(1j * (blo.imag - lo.imag)), torch.ones_like(lo)) <= RTOL
        assert _rel(blo.real, lo.real) <= RTOL
        assert torch.allclose(bW, W, rtol=RTOL, atol=0.0)
        El = R.local_energy(ham, psi)
        assert _rel(bs.local_energy(bpsi), El) <= RTOL
    assert int((W > 0).sum()) == nw - len(dead)

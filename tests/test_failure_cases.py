"""Failures made on the host, never by faulting the GPU: non-finite fields, a
walker whose overlap with the trial is exactly zero, a population with no
weight left, and a tensor-core pipeline wait that runs out.  Each must give
the affected walker W = 0 and its status bit (or a reported timeout) while
every call returns normally, the other walkers follow the oracle, and the
context stays usable."""
import ctypes
import math

import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import make_fields, make_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


TOL = {"fp64": 1e-10, "mixed": 1e-4}


def _oracle_one_step(s, trial, psi, lo, W, x, tau, e0, order):
    ham = R.make_hamiltonian(s.h1, s.L, trial, s.na, s.nb, s.e_const)
    Lbar = R.mean_field_shift(ham)
    hpp, ec = R.propagation_h1(ham, Lbar)
    B = R.half_step_propagator(hpp, tau)
    psi1, lo1, W1, _ = R.step(ham, psi, lo, W, torch.as_tensor(x), tau, e0, method="krylov", k=order,
                              B=B, L_bar=Lbar, ec=ec)
    El = R.local_energy(ham, psi1)
    return psi1, W1, El, R.mixed_energy(W1, R.energy_window(El, e0, tau, s.na + s.nb))[0]


def _check_survivors(ctx, w, e_loc, e_mix, keep, ref, prec):
    psi1, W1, El, emix = ref
    tol = TOL[prec]
    W = w.weight.cpu()
    got_E = torch.complex(e_loc[:, 0], e_loc[:, 1]).cpu()
    for j, i in enumerate(keep):
        assert abs(float(W[i]) - float(W1[j])) <= tol * abs(float(W1[j])), (i, float(W[i]), float(W1[j]))
        dE = abs(complex(got_E[i] - El[j]))
        assert dE <= (tol * abs(complex(El[j])) if prec == "fp64" else 1e-4), (i, dE)
    assert abs(float(e_mix[2]) - emix) <= (tol * abs(emix) if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_non_finite_fields_kill_only_their_walkers(prec):
    from paper_2403_02542_gb300 import _lib as L
    from paper_2403_02542_gb300.api import Context
    s = make_system(16, 3, 3, 30, rho=0.85, seed=161)
    nw, tau, order = 6, 0.05, 8
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb, s.e_const)
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    x = make_fields(5, 0, nw, s.G)
    x[1, :] = np.nan
    x[3, 7] = np.inf
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision=prec)
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    e_loc = torch.empty(nw, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    ctx.step(w, torch.as_tensor(x, device=ctx.device), tau, e0, expm="krylov", order=order, measure=True,
             e_loc=e_loc, e_mix=e_mix, reuse_bias=True)
    ctx.sync()
    st = w.status.cpu()
    for i in (1, 3):
        assert float(w.weight[i]) == 0.0 and int(st[i]) & L.W_NONFINITE, (i, int(st[i]))
    keep = [0, 2, 4, 5]
    psi0, lo0, W0 = R.init_walkers(ham, len(keep))
    ref = _oracle_one_step(s, s.trial, psi0, lo0, W0, x[keep], tau, e0, order)
    _check_survivors(ctx, w, e_loc, e_mix, keep, ref, prec)
    assert float(e_mix[3]) == len(keep)
    # the dead walkers are left alone by the next step, which succeeds
    x2 = torch.as_tensor(make_fields(5, 1, nw, s.G), device=ctx.device)
    ctx.step(w, x2, tau, e0, expm="krylov", order=order, measure=True, e_loc=e_loc, e_mix=e_mix, reuse_bias=True)
    ctx.sync()
    assert float(w.weight[1]) == 0.0 and float(w.weight[3]) == 0.0
    assert math.isfinite(float(e_mix[2])) and float(e_mix[3]) == len(keep)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_walker_with_zero_overlap_is_marked_singular(prec):
    """The trial is the first unit vectors of each spin, and walker 0's alpha
    orbitals are the next unit vectors: trial_alpha^T psi_alpha = 0 exactly."""
    from paper_2403_02542_gb300 import _lib as L
    from paper_2403_02542_gb300.api import Context
    s = make_system(12, 2, 2, 24, rho=0.85, seed=121)
    N, na, nb = 12, 2, 2
    trial = np.zeros((N, na + nb))
    trial[0, 0] = trial[1, 1] = 1.0
    trial[0, 2] = trial[1, 3] = 1.0
    nw, tau, order = 5, 0.05, 8
    ham = R.make_hamiltonian(s.h1, s.L, trial, na, nb, s.e_const)
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    psi = torch.as_tensor(trial).to(torch.complex128).unsqueeze(0).repeat(nw, 1, 1)
    psi[0, :, 0:2] = 0.0
    psi[0, 2, 0] = psi[0, 3, 1] = 1.0
    x = make_fields(6, 0, nw, s.G)
    ctx = Context(s.h1, s.L, trial, na, nb, precision=prec)
    w = ctx.new_walkers(nw)
    w.psi.copy_(psi.transpose(1, 2).to(ctx.ctype))
    w.weight.fill_(1.0)
    w.logovl.zero_()
    w.status.zero_()
    e_loc = torch.empty(nw, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    ctx.step(w, torch.as_tensor(x, device=ctx.device), tau, e0, expm="krylov", order=order, measure=True,
             e_loc=e_loc, e_mix=e_mix)
    ctx.sync()
    st = int(w.status[0])
    assert float(w.weight[0]) == 0.0 and st & L.W_SINGULAR, st
    keep = [1, 2, 3, 4]
    lo = torch.zeros(len(keep), dtype=torch.complex128)
    ref = _oracle_one_step(s, trial, psi[keep], lo, torch.ones(len(keep), dtype=torch.float64), x[keep], tau,
                           e0, order)
    _check_survivors(ctx, w, e_loc, e_mix, keep, ref, prec)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_population_without_weight(prec):
    """Every W = 0: a step leaves every walker as it was, E_k is NaN with zero
    total weight and no live walker, and the comb leaves the population
    unchanged with every index -1; no call fails."""
    from paper_2403_02542_gb300.api import Context
    s = make_system(16, 3, 3, 30, rho=0.85, seed=162)
    nw, tau = 8, 0.05
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision=prec)
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    w.weight.zero_()
    before = w.psi.clone()
    e_loc = torch.empty(nw, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    ctx.step(w, torch.as_tensor(make_fields(7, 0, nw, s.G), device=ctx.device), tau, -20.0, expm="krylov",
             order=8, reortho=True, measure=True, e_loc=e_loc, e_mix=e_mix)
    idx = torch.zeros(nw, dtype=torch.int32, device=ctx.device)
    ctx.population_control(w, 0.3, idx)
    ctx.sync()
    assert torch.equal(w.psi, before) and float(w.weight.abs().sum()) == 0.0
    m = e_mix.cpu()
    assert float(m[1]) == 0.0 and float(m[3]) == 0.0 and math.isnan(float(m[2]))
    assert (idx.cpu() == -1).all()
    ctx.close()


def test_pipeline_wait_that_runs_out_is_reported_and_cleared():
    """A tensor-core pipeline wait bounded to about 1 ms on an mbarrier phase
    that nothing completes (afqmc_wait_probe): afqmc_sync reports the timeout
    once, the next sync is clean, and the context then runs a step whose
    local energies match the oracle."""
    from paper_2403_02542_gb300 import _lib as L
    from paper_2403_02542_gb300.api import Context
    s = make_system(32, 4, 4, 64, rho=0.9, seed=163)
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="mixed")
    lib = L.lib()
    assert lib.afqmc_wait_probe(ctx._h, 0) == L.AFQMC_EINVAL
    assert lib.afqmc_wait_probe(ctx._h, 2_000_000) == L.AFQMC_OK
    st = lib.afqmc_sync(ctx._h)
    assert st == L.AFQMC_ECUDA
    assert b"timed out (code 128)" in lib.afqmc_last_cuda_error()
    assert lib.afqmc_sync(ctx._h) == L.AFQMC_OK
    nw, tau = 4, 0.05
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb, s.e_const)
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    x = make_fields(8, 0, nw, s.G)
    e_loc = torch.empty(nw, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    ctx.step(w, torch.as_tensor(x, device=ctx.device), tau, e0, expm="krylov", order=8, measure=True,
             e_loc=e_loc, e_mix=e_mix)
    assert lib.afqmc_sync(ctx._h) == L.AFQMC_OK
    psi0, lo0, W0 = R.init_walkers(ham, nw)
    ref = _oracle_one_step(s, s.trial, psi0, lo0, W0, x, tau, e0, 8)
    _check_survivors(ctx, w, e_loc, e_mix, list(range(nw)), ref, "mixed")
    ctx.close()
    # a context without the tensor-core exchange has no such pipeline
    c64 = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="fp64")
    assert lib.afqmc_wait_probe(c64._h, 1000) == L.AFQMC_ENOTSUP
    c64.close()

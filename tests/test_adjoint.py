"""Adjoint of the mixed energy estimator (afqmc_energy_backward) against
torch reverse-mode autograd through the CPU oracle and against central finite
differences of the GPU forward.  Walker states are produced by the oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import make_fields, make_system

pytestmark = pytest.mark.gpu
CT, RT = torch.complex128, torch.float64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _oracle_state(s, nw, steps, tau, e0, seed):
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb)
    psi, lo, W = R.init_walkers(ham, nw)
    for k in range(steps):
        psi, lo, W, _ = R.step(ham, psi, lo, W, make_fields(seed, k, nw, ham.G), tau, e0,
                               method="taylor", k=6, reortho=(k % 2 == 1))
    return psi, lo, W


def _oracle_J(h1, L, s, psi, W, e0, tau):
    ham = R.Hamiltonian(h1, L, torch.as_tensor(s.trial, dtype=RT), s.na, s.nb, s.e_const)
    El = R.local_energy(ham, psi)
    Ecap = R.energy_window(El, e0, tau, s.na + s.nb)
    live = W > 0
    Wl = torch.where(live, W, torch.zeros_like(W))
    return (Wl * Ecap).sum() / Wl.sum()


def _gpu_walkers(ctx, psi, lo, W):
    w = ctx.new_walkers(psi.shape[0])
    w.psi.copy_(psi.transpose(1, 2).to(ctx.ctype))
    w.weight.copy_(W)
    w.logovl.copy_(torch.stack([lo.real, lo.imag], 1))
    w.status.zero_()
    return w


@pytest.mark.parametrize("N,n,G,nw", [(10, 2, 12, 6), (24, 3, 40, 9)])
def test_energy_adjoint_matches_oracle_autograd(N, n, G, nw):
    from paper_2403_02542_gb300.api import Context
    s = make_system(N, n, n, G, rho=0.8, seed=N)
    tau = 0.05
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, n, n)
    e0 = float(R.local_energy(ham, ham.trial.to(CT)).real)
    psi, lo, W = _oracle_state(s, nw, 3, tau, e0, seed=9)
    W[1] = 0.0  # a dead walker does not contribute
    h1 = torch.as_tensor(s.h1, dtype=RT).clone().requires_grad_(True)
    L = torch.as_tensor(s.L, dtype=RT).clone().requires_grad_(True)
    J = _oracle_J(h1, L, s, psi, W, e0, tau)
    J.backward()
    ctx = Context(s.h1, s.L, s.trial, n, n, precision="fp64")
    w = _gpu_walkers(ctx, psi, lo, W)
    gh, gL = ctx.energy_backward(w, e0, tau)
    gh, gL = gh.cpu(), gL.cpu()
    assert torch.allclose(gh, h1.grad, rtol=1e-9, atol=1e-12 * float(h1.grad.abs().max()))
    assert torch.allclose(gL, L.grad, rtol=1e-9, atol=1e-12 * float(L.grad.abs().max()))
    # the forward value agrees as well
    _, e_mix = ctx.local_energy(w, e0, tau)
    assert abs(float(e_mix[2]) - float(J.detach())) <= 1e-10 * abs(float(J.detach()))


def test_energy_adjoint_matches_central_differences():
    """Directional derivatives along random symmetric dH1, dL (step 1e-5)."""
    from paper_2403_02542_gb300.api import Context
    N, n, G, nw, tau = 16, 3, 20, 8, 0.05
    s = make_system(N, n, n, G, rho=0.8, seed=7)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, n, n)
    e0 = float(R.local_energy(ham, ham.trial.to(CT)).real)
    psi, lo, W = _oracle_state(s, nw, 2, tau, e0, seed=4)
    rng = np.random.default_rng(1)
    dH = rng.standard_normal((N, N)); dH = 0.5 * (dH + dH.T)
    dL = rng.standard_normal((G, N, N)); dL = 0.5 * (dL + dL.transpose(0, 2, 1))

    def energy(h1, chol):
        c = Context(h1, chol, s.trial, n, n, precision="fp64")
        w = _gpu_walkers(c, psi, lo, W)
        _, em = c.local_energy(w, e0, tau)
        v = float(em[2])
        c.close()
        return v

    ctx = Context(s.h1, s.L, s.trial, n, n, precision="fp64")
    gh, gL = ctx.energy_backward(_gpu_walkers(ctx, psi, lo, W), e0, tau)
    gh, gL = gh.cpu().numpy(), gL.cpu().numpy()
    eps = 1e-5
    fd_h = (energy(s.h1 + eps * dH, s.L) - energy(s.h1 - eps * dH, s.L)) / (2 * eps)
    fd_L = (energy(s.h1, s.L + eps * dL) - energy(s.h1, s.L - eps * dL)) / (2 * eps)
    assert abs(fd_h - float((gh * dH).sum())) <= 1e-7 * max(1.0, abs(fd_h))
    assert abs(fd_L - float((gL * dL).sum())) <= 1e-7 * max(1.0, abs(fd_L))


def test_autograd_function_wrapper():
    from paper_2403_02542_gb300.api import MixedEnergy
    N, n, G, nw, tau = 12, 2, 16, 5, 0.05
    s = make_system(N, n, n, G, rho=0.8, seed=3)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, n, n)
    e0 = float(R.local_energy(ham, ham.trial.to(CT)).real)
    psi, lo, W = _oracle_state(s, nw, 2, tau, e0, seed=2)
    dev = torch.device("cuda")
    walkers = dict(psi=psi.transpose(1, 2).contiguous().to(dev), weight=W.to(dev),
                   logovl=torch.stack([lo.real, lo.imag], 1).contiguous().to(dev))
    h1 = torch.as_tensor(s.h1, dtype=RT).clone().requires_grad_(True)
    L = torch.as_tensor(s.L, dtype=RT).clone().requires_grad_(True)
    J = MixedEnergy.apply(h1, L, walkers, s.trial, n, n, e0, tau)
    J.backward()
    h1r = torch.as_tensor(s.h1, dtype=RT).clone().requires_grad_(True)
    Lr = torch.as_tensor(s.L, dtype=RT).clone().requires_grad_(True)
    Jr = _oracle_J(h1r, Lr, s, psi, W, e0, tau)
    Jr.backward()
    assert abs(float(J) - float(Jr)) <= 1e-10 * abs(float(Jr))
    assert torch.allclose(h1.grad, h1r.grad, rtol=1e-9, atol=1e-13)
    assert torch.allclose(L.grad, Lr.grad, rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("N,n,G,nw", [(10, 2, 12, 6), (24, 3, 40, 9)])
def test_energy_adjoint_mixed_matches_oracle_autograd(N, n, G, nw):
    """Mixed context: the walkers are held as complex64 and the per-walker
    terms formed in FP32 (sums over walkers in FP64), so the gradients agree
    with the oracle's to FP32 rounding of O(N) terms: 1e-5 of the largest
    entry, far below the O(1) change of any misplaced term."""
    from paper_2403_02542_gb300.api import Context
    s = make_system(N, n, n, G, rho=0.8, seed=N)
    tau = 0.05
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, n, n)
    e0 = float(R.local_energy(ham, ham.trial.to(CT)).real)
    psi, lo, W = _oracle_state(s, nw, 3, tau, e0, seed=9)
    W[1] = 0.0
    h1 = torch.as_tensor(s.h1, dtype=RT).clone().requires_grad_(True)
    L = torch.as_tensor(s.L, dtype=RT).clone().requires_grad_(True)
    J = _oracle_J(h1, L, s, psi, W, e0, tau)
    J.backward()
    ctx = Context(s.h1, s.L, s.trial, n, n, precision="mixed")
    w = _gpu_walkers(ctx, psi, lo, W)
    gh, gL = ctx.energy_backward(w, e0, tau)
    gh, gL = gh.cpu(), gL.cpu()
    for got, ref in ((gh, h1.grad), (gL, L.grad)):
        scale = float(ref.abs().max())
        assert float((got - ref).abs().max()) <= 1e-5 * scale
    ctx.close()

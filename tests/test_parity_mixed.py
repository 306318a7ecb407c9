"""Mixed-precision CUDA path (complex64 walkers; FP32 contractions; FP64
overlaps, log-determinants, Krylov coefficients, small exponential, weights)
against the FP64 CPU oracle.

Bound (per step, from a common FP64 state produced by the oracle):
|E_L(mixed) - E_L(oracle)| <= 1e-4 Ha per walker.  Weights, log-overlaps and
walkers are reported with looser relative bounds that follow from complex64
storage (unit roundoff 6e-8) amplified by the step."""
import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import config_system, make_fields, make_system
from walk_helpers import oracle_walk

pytestmark = pytest.mark.gpu
E_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mixed_step_from_oracle_state(s, nw, n_pre, tau, k, seed, expm="krylov"):
    from paper_2403_02542_gb300.api import Context
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb)
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    ref, ties = oracle_walk(s, nw, n_pre + 1, tau, e0, expm, k, 0, seed=seed)
    assert ties == 0
    state, nxt = ref[n_pre - 1], ref[n_pre]
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="mixed")
    w = ctx.new_walkers(nw)
    w.psi.copy_(state["psi"].transpose(1, 2).to(torch.complex64))
    w.weight.copy_(state["W"])
    w.logovl.copy_(torch.stack([state["lo"].real, state["lo"].imag], 1))
    w.status.zero_()
    x = torch.as_tensor(make_fields(seed, n_pre, nw, s.G), device=ctx.device)
    e_loc = torch.empty(nw, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    ctx.step(w, x, tau, e0, expm=expm, order=k, measure=True, e_loc=e_loc, e_mix=e_mix)
    torch.cuda.synchronize()
    El = torch.complex(e_loc[:, 0], e_loc[:, 1]).cpu()
    live = nxt["W"] > 0
    dE = (El - nxt["El"]).abs()[live]
    dW = ((w.weight.cpu() - nxt["W"]).abs() / nxt["W"])[live]
    g = w.psi.cpu().to(torch.complex128).transpose(1, 2)
    dpsi = ((g - nxt["psi"]).flatten(1).norm(dim=1) / nxt["psi"].flatten(1).norm(dim=1))[live]
    ctx.close()
    return float(dE.max()), float(dW.max()), float(dpsi.max())


def test_mixed_step_large_workload():
    """N=128, 20+20 electrons, 640 vectors, Krylov 10, tau=0.05."""
    s = config_system("large")
    dE, dW, dpsi = _mixed_step_from_oracle_state(s, 6, 3, 0.05, 10, seed=77)
    print(f"mixed vs oracle, large workload: max|dE_L| = {dE:.2e} Ha, "
          f"max rel dW = {dW:.2e}, max rel dPsi = {dpsi:.2e}")
    assert dE <= E_TOL
    assert dW <= 1e-4 and dpsi <= 1e-4


def test_mixed_step_taylor_ragged():
    s = make_system(72, 5, 5, 150, rho=1e-5 ** (1 / 150), seed=4242)
    dE, dW, dpsi = _mixed_step_from_oracle_state(s, 9, 2, 0.05, 6, seed=8, expm="taylor")
    print(f"mixed vs oracle, N=72 Taylor-6: max|dE_L| = {dE:.2e} Ha, "
          f"max rel dW = {dW:.2e}, max rel dPsi = {dpsi:.2e}")
    assert dE <= E_TOL
    assert dW <= 1e-4 and dpsi <= 1e-4


@pytest.mark.parametrize("n", [1, 2, 3])
def test_mixed_local_energy_small_blocks(n):
    """Tensor-core exchange with many g blocks per 128-row tile (128 / n of
    them): E_L of fresh walkers and after a local energy of other walkers
    (nothing may be left from an earlier evaluation), against the oracle."""
    from paper_2403_02542_gb300.api import Context
    s = make_system(32, n, n, 200, rho=0.98, seed=40 + n)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, n, n)
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    g = torch.Generator().manual_seed(n)
    nw = 6
    psi = (torch.as_tensor(s.trial).to(torch.complex128).unsqueeze(0).repeat(nw, 1, 1)
           + 0.2 * torch.complex(torch.randn(nw, 32, 2 * n, generator=g, dtype=torch.float64),
                                 torch.randn(nw, 32, 2 * n, generator=g, dtype=torch.float64)))
    ref = R.local_energy(ham, psi)
    ctx = Context(s.h1, s.L, s.trial, n, n, precision="mixed")
    other = ctx.new_walkers(nw)
    ctx.init_walkers(other)
    w = ctx.new_walkers(nw)
    w.psi.copy_(psi.transpose(1, 2).to(torch.complex64))
    w.weight.fill_(1.0)
    w.logovl.zero_()
    w.status.zero_()
    for first in (other, w):
        ctx.local_energy(first, e0, 0.05)  # a different population first, then ours
    e_loc, _ = ctx.local_energy(w, e0, 0.05)
    got = torch.complex(e_loc[:, 0], e_loc[:, 1]).cpu()
    assert float((got - ref).abs().max()) <= E_TOL, float((got - ref).abs().max())
    ctx.close()


def _sampled_mixed_walk(cfg_name, nw, steps, reortho_every, sample, seed):
    """The mixed path at full size in the benchmark's launch configuration
    (force bias reused from the previous E_L); the oracle follows a sample of
    the walkers one by one with the same fields."""
    from paper_2403_02542_gb300.api import Context
    from walk_helpers import gpu_walk
    s = config_system(cfg_name)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb)
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="mixed")
    got, _ = gpu_walk(ctx, nw, steps, 0.05, e0, "krylov", 10, reortho_every, seed=seed, reuse_bias=True,
                      record=set(range(steps)))
    ref, ties = oracle_walk(s, len(sample), steps, 0.05, e0, "krylov", 10, reortho_every, seed=None,
                            field_fn=lambda step: make_fields(seed, step, nw, s.G)[sample])
    assert ties == 0
    worst = 0.0
    for step in range(steps):
        dE = (got[step]["El"][sample] - ref[step]["El"]).abs()
        dW = ((got[step]["W"][sample] - ref[step]["W"]).abs() / ref[step]["W"]).max()
        worst = max(worst, float(dE.max()))
        assert float(dE.max()) <= E_TOL, (cfg_name, step, float(dE.max()))
        assert float(dW) <= 1e-4, (cfg_name, step, float(dW))
    print(f"{cfg_name}: max |dE_L| over sampled walkers = {worst:.2e} Ha")
    ctx.close()


def test_mixed_large_workload_full_launch_sampled():
    """N=128, 20+20 electrons, 640 vectors, 1024 walkers, Krylov 10, QR every 2."""
    _sampled_mixed_walk("large", 1024, 3, 2, [0, 511, 1023], seed=4096)


def test_mixed_precision_workload_full_launch_sampled():
    """N=300, 50+50 electrons, 1500 vectors, 2048 walkers, Krylov 10, two steps."""
    _sampled_mixed_walk("precision", 2048, 2, 0, [0, 2047], seed=5120)


@pytest.mark.parametrize("N,n,G", [(192, 48, 200), (300, 50, 120)])
def test_mixed_local_energy_streamed_operand(N, n, G):
    """Tensor-core exchange for N > 128, where the Theta tile streams through
    the pipeline with every K slab (two and one epilogue warpgroups)."""
    from paper_2403_02542_gb300.api import Context
    s = make_system(N, n, n, G, rho=0.97, seed=N + n)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, n, n)
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    g = torch.Generator().manual_seed(N)
    nw = 5
    psi = (torch.as_tensor(s.trial).to(torch.complex128).unsqueeze(0).repeat(nw, 1, 1)
           + 0.1 * torch.complex(torch.randn(nw, N, 2 * n, generator=g, dtype=torch.float64),
                                 torch.randn(nw, N, 2 * n, generator=g, dtype=torch.float64)))
    ref = R.local_energy(ham, psi)
    ctx = Context(s.h1, s.L, s.trial, n, n, precision="mixed")
    w = ctx.new_walkers(nw)
    w.psi.copy_(psi.transpose(1, 2).to(torch.complex64))
    w.weight.fill_(1.0)
    w.logovl.zero_()
    w.status.zero_()
    e_loc, _ = ctx.local_energy(w, e0, 0.05)
    got = torch.complex(e_loc[:, 0], e_loc[:, 1]).cpu()
    assert float((got - ref).abs().max()) <= E_TOL, float((got - ref).abs().max())
    ctx.close()

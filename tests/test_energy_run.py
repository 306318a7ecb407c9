"""An energy run of the library (steps with E_L every step, comb population
control, E_0 updates) against the same protocol driven through the CPU oracle
with the same fields and comb numbers: the per-step total weights and mixed
estimates agree to 1e-10 in FP64, and the run's statistics follow."""
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300 import energy as S
from paper_2403_02542_gb300.inputs import make_fields, make_system
from walk_helpers import oracle_energy_run as _oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_energy_run_matches_the_oracle_protocol():
    from paper_2403_02542_gb300.api import Context
    s = make_system(10, 2, 2, 16, rho=0.8, seed=12)
    nw, tau, n_steps, n_eq, order, reo, pop, seed, fseed = 12, 0.05, 12, 4, 6, 3, 4, 5, 77
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb, s.e_const)
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    Wr, Er = _oracle_run(s, nw, tau, e0, n_steps, n_eq, order, reo, pop, seed, fseed)
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    out = S.energy_run(ctx, w, tau, e0, n_steps, fields=lambda k: torch.as_tensor(
        make_fields(fseed, k, nw, s.G), device=ctx.device), n_eq=n_eq, order=order, reortho_every=reo,
        pop_every=pop, seed=seed, update_e0=True)
    ctx.close()
    for k in range(n_steps):
        assert out["W"][k] == pytest.approx(Wr[k], rel=1e-10), k
        assert out["E"][k] == pytest.approx(Er[k], rel=1e-10), k
    # E_0 follows the protocol: the latest estimate during equilibration, the running average after
    assert out["e0"][4] == pytest.approx(Er[3], rel=1e-12)
    assert out["e0"][8] == pytest.approx(S.time_average(Wr[:8], Er[:8], n_eq)[0], rel=1e-10)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_run_far_from_zero_seeds_e0_from_the_uncapped_energy(precision):
    """A system whose energy lies several DeltaE (Eq. enwin) below 0, run with
    e0=None as the time-step scan of the benchmark runs it: E_0 starts at the
    uncapped E_L of the trial, no walker is lost to the reweighting cap, and
    the run follows the oracle protocol started at E_L(Psi_T) (FP64: 1e-10
    relative per step; mixed: 1e-4 Ha in E_k, 1e-4 relative in the weights)."""
    from paper_2403_02542_gb300.api import Context
    s = make_system(24, 4, 4, 60, rho=0.9, seed=2424)
    nw, tau, n_steps, n_eq, order, reo, pop, seed, fseed = 10, 0.05, 8, 4, 8, 4, 4, 9, 79
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb, s.e_const)
    e_trial = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    dE = 0.5 * (8 / tau) ** 0.5 + (8 * tau) ** 0.5
    assert e_trial < -1.5 * dE, (e_trial, dE)
    Wr, Er = _oracle_run(s, nw, tau, e_trial, n_steps, n_eq, order, reo, pop, seed, fseed)
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision=precision)
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    out = S.energy_run(ctx, w, tau, None, n_steps, fields=lambda k: torch.as_tensor(
        make_fields(fseed, k, nw, s.G), device=ctx.device), n_eq=n_eq, order=order, reortho_every=reo,
        pop_every=pop, seed=seed, update_e0=True)
    ctx.close()
    assert out["e0"][0] == pytest.approx(e_trial, rel=1e-10 if precision == "fp64" else 1e-6)
    for k in range(n_steps):
        if precision == "fp64":
            assert out["W"][k] == pytest.approx(Wr[k], rel=1e-10), k
            assert out["E"][k] == pytest.approx(Er[k], rel=1e-10), k
        else:
            assert out["W"][k] == pytest.approx(Wr[k], rel=1e-4), k
            assert abs(out["E"][k] - Er[k]) <= 1e-4, k
    assert min(out["W"]) > 0.5 * nw

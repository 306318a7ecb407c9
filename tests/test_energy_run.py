"""An energy run of the library (steps with E_L every step, comb population
control, E_0 updates) against the same protocol driven through the CPU oracle
with the same fields and comb numbers: the per-step total weights and mixed
estimates agree to 1e-10 in FP64, and the run's statistics follow."""
import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300 import energy as S
from paper_2403_02542_gb300.inputs import make_fields, make_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _oracle_run(s, nw, tau, e0, n_steps, n_eq, order, reortho_every, pop_every, seed, fseed):
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb, s.e_const)
    Lbar = R.mean_field_shift(ham)
    hpp, ec = R.propagation_h1(ham, Lbar)
    B = R.half_step_propagator(hpp, tau)
    psi, lo, W = R.init_walkers(ham, nw)
    rng = np.random.Generator(np.random.PCG64(seed))
    Ws, Es = [], []
    for k in range(n_steps):
        reo = reortho_every > 0 and (k + 1) % reortho_every == 0
        x = make_fields(fseed, k, nw, ham.G)
        psi, lo, W, _ = R.step(ham, psi, lo, W, x, tau, e0, method="krylov", k=order, reortho=reo,
                               B=B, L_bar=Lbar, ec=ec)
        El = R.local_energy(ham, psi)
        emix, wsum = R.mixed_energy(W, R.energy_window(El, e0, tau, ham.na + ham.nb))
        Ws.append(float(wsum))
        Es.append(float(emix))
        if (k + 1) % pop_every == 0:
            psi, lo, W, _ = R.population_control(psi, lo, W, float(rng.random()))
            e0 = Es[-1] if k < n_eq else S.time_average(Ws, Es, n_eq)[0]
    return Ws, Es


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

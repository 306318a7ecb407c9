"""Statistics of the energy run (no GPU): the weighted time average and
variance of Sec. II.A, the correlation length of Eq. variance from a blocking
analysis, checked on series whose correlation is known in closed form, and the
time-step extrapolation fits, checked on exact and on noisy synthetic data."""
import math

import numpy as np
import pytest

from paper_2403_02542_gb300 import energy as S


def test_time_average_small_example_and_weight_scale():
    W, E = [5.0, 1.0, 2.0, 1.0], [9.0, 1.0, 2.0, 4.0]
    ebar, var = S.time_average(W, E, n_eq=1)          # the first sample is equilibration
    assert ebar == pytest.approx(9.0 / 4.0) and var == pytest.approx(25.0 / 4.0 - (9.0 / 4.0) ** 2)
    e2, v2 = S.time_average([3 * x for x in W], E, n_eq=1)   # a common weight factor cancels
    assert e2 == pytest.approx(ebar) and v2 == pytest.approx(var)
    with pytest.raises(ValueError):
        S.time_average([0.0, 0.0], [1.0, 2.0])


def test_blocking_uncorrelated_series():
    rng = np.random.default_rng(1)
    n = 1 << 14
    E = rng.standard_normal(n)
    r = S.blocking(np.ones(n), E)
    assert 0.75 < r["kappa"] < 1.35
    assert r["sigma"] == pytest.approx(1.0 / math.sqrt(n), rel=0.25)


@pytest.mark.parametrize("rho", [0.5, 0.8, 0.9])
def test_blocking_ar1_correlation_length(rho):
    """AR(1) E_k = rho E_{k-1} + noise: kappa = (1 + rho) / (1 - rho)."""
    rng = np.random.default_rng(7)
    n = 1 << 17
    x = np.empty(n)
    x[0] = 0.0
    eps = rng.standard_normal(n)
    for k in range(1, n):
        x[k] = rho * x[k - 1] + eps[k]
    r = S.blocking(np.ones(n), 10.0 + x, n_eq=0)
    kappa = (1 + rho) / (1 - rho)
    assert r["kappa"] == pytest.approx(kappa, rel=0.3), (r["kappa"], kappa)
    assert r["E_bar"] == pytest.approx(10.0, abs=6 * r["sigma"])


@pytest.mark.parametrize("power", [1, 2])
def test_extrapolation_exact_data(power):
    taus = [0.01, 0.02, 0.05, 0.1]
    e0, c = -75.25, 3.5
    y = [e0 + c * t ** power for t in taus]
    f0, fc, s0, sc, chi2 = S.extrapolate(taus, y, None, power)
    assert f0 == pytest.approx(e0, abs=1e-12) and fc == pytest.approx(c, rel=1e-10)
    assert chi2 == pytest.approx(0.0, abs=1e-20)


def test_extrapolation_errors_match_the_scatter():
    """Noisy replicas: the spread of the fitted E_0 matches its reported error
    and chi^2 per degree of freedom averages to one."""
    rng = np.random.default_rng(3)
    taus = np.array([0.01, 0.02, 0.05, 0.1, 0.2])
    sig = np.array([2e-3, 1.5e-3, 1e-3, 1e-3, 1e-3])
    e0, c = -1.0, 0.8
    fits, chis = [], []
    for _ in range(4000):
        y = e0 + c * taus ** 2 + sig * rng.standard_normal(taus.size)
        f0, fc, s0, sc, chi2 = S.extrapolate(taus, y, sig, 2)
        fits.append(f0)
        chis.append(chi2)
    assert np.std(fits) == pytest.approx(s0, rel=0.06)
    assert np.mean(fits) == pytest.approx(e0, abs=4 * s0 / math.sqrt(len(fits)))
    assert np.mean(chis) == pytest.approx(1.0, rel=0.06)


def test_general_time_step_fit_recovers_linear_and_quadratic_terms():
    """Eq. square_fit, E(tau) = E_0 + alpha tau + beta tau^2: exact data give back
    all three coefficients; noisy replicas scatter as the reported errors; the
    pure forms are the special cases with one power."""
    taus = np.array([0.005, 0.01, 0.02, 0.05, 0.1, 0.2])
    e0, a, b = -40.125, -0.35, 2.5
    f = S.fit_time_step(taus, e0 + a * taus + b * taus ** 2, None, (1, 2))
    assert f["E0"] == pytest.approx(e0, abs=1e-11)
    assert f["c"] == pytest.approx([a, b], rel=1e-9) and f["chi2_dof"] == pytest.approx(0.0, abs=1e-18)
    one = S.fit_time_step(taus, e0 + b * taus ** 2, None, (2,))
    assert (one["E0"], one["c"][0]) == pytest.approx((e0, b), rel=1e-12)
    assert one["E0"] == pytest.approx(S.extrapolate(taus, e0 + b * taus ** 2, None, 2)[0], abs=0)
    rng = np.random.default_rng(8)
    sig = np.full(taus.size, 1e-3)
    fits = [S.fit_time_step(taus, e0 + a * taus + b * taus ** 2 + sig * rng.standard_normal(taus.size), sig)
            for _ in range(3000)]
    e0s = np.array([q["E0"] for q in fits])
    assert np.std(e0s) == pytest.approx(fits[0]["sigma_E0"], rel=0.06)
    assert np.mean([q["chi2_dof"] for q in fits]) == pytest.approx(1.0, rel=0.06)
    with pytest.raises(ValueError):
        S.fit_time_step(taus[:2], [1.0, 2.0], None, (1, 2))


def test_extrapolation_error_of_eq_staterr():
    """sigma_x = sqrt(sum sigma_i^2) / N_tau: equal errors give sigma / sqrt(N_tau);
    a worked case sqrt(9 + 16) / 2 = 2.5."""
    assert S.extrapolation_error([0.2] * 4) == pytest.approx(0.2 / 2.0, rel=1e-15)
    assert S.extrapolation_error([3.0, 4.0]) == pytest.approx(2.5, rel=1e-15)
    with pytest.raises(ValueError):
        S.extrapolation_error([])


def test_energy_run_driver_follows_its_protocol_on_the_oracle():
    """energy_run's host logic (steps with E_L every step, QR every 3 steps, the
    comb every 4 steps with numbers from PCG64(seed), E_0 updates at each comb)
    driven through the oracle-backed stand-in context gives exactly the
    per-step weights and estimates of the same protocol written out on the
    oracle, and E_0 takes the values the protocol names."""
    import torch
    from oracle import afqmc_ref as R
    from oracle_context import OracleContext
    from paper_2403_02542_gb300.inputs import make_fields, make_system
    from walk_helpers import oracle_energy_run
    s = make_system(10, 2, 2, 16, rho=0.8, seed=12)
    nw, tau, n_steps, n_eq, order, reo, pop, seed, fseed = 12, 0.05, 12, 4, 6, 3, 4, 5, 77
    octx = OracleContext(s)
    e0 = float(R.local_energy(octx.ham, octx.ham.trial.to(torch.complex128)).real)
    Wr, Er = oracle_energy_run(s, nw, tau, e0, n_steps, n_eq, order, reo, pop, seed, fseed)
    w = octx.new_walkers(nw)
    octx.init_walkers(w)
    out = S.energy_run(octx, w, tau, e0, n_steps, fields=lambda k: torch.as_tensor(make_fields(fseed, k, nw, s.G)),
                       n_eq=n_eq, order=order, reortho_every=reo, pop_every=pop, seed=seed, update_e0=True)
    assert out["W"] == pytest.approx(Wr, rel=1e-14)
    assert out["E"] == pytest.approx(Er, rel=1e-14)
    assert out["e0"][:4] == [e0] * 4
    assert out["e0"][4] == pytest.approx(Er[3], rel=1e-14)
    assert out["e0"][8] == pytest.approx(S.time_average(Wr[:8], Er[:8], n_eq)[0], rel=1e-14)


def test_energy_run_seeds_e0_from_the_uncapped_local_energy():
    """With e0=None the run starts from the weighted mean of the uncapped E_L
    of its starting walkers (initial_e0).  On a system whose energy lies far
    outside the window DeltaE around 0, an E_0 taken from a mixed estimate
    clamped around 0 would be wrong by many DeltaE; the seeded run instead
    equals the protocol started at E_L(Psi_T) step for step."""
    import torch
    from oracle import afqmc_ref as R
    from oracle_context import OracleContext
    from paper_2403_02542_gb300.inputs import make_fields, make_system
    from walk_helpers import oracle_energy_run
    s = make_system(8, 2, 2, 32, rho=0.5, seed=20240304)
    nw, tau, n_steps, n_eq, order, reo, pop, seed, fseed = 10, 0.04, 8, 4, 6, 3, 4, 6, 78
    octx = OracleContext(s)
    e_trial = float(R.local_energy(octx.ham, octx.ham.trial.to(torch.complex128)).real)
    dE = 0.5 * math.sqrt(4 / tau) + math.sqrt(4 * tau)
    assert abs(e_trial) > dE                 # E_L lies outside the window around 0
    w = octx.new_walkers(nw)
    octx.init_walkers(w)
    assert S.initial_e0(octx, w, tau) == pytest.approx(e_trial, rel=1e-13)
    Wr, Er = oracle_energy_run(s, nw, tau, e_trial, n_steps, n_eq, order, reo, pop, seed, fseed)
    out = S.energy_run(octx, w, tau, None, n_steps, fields=lambda k: torch.as_tensor(make_fields(fseed, k, nw, s.G)),
                       n_eq=n_eq, order=order, reortho_every=reo, pop_every=pop, seed=seed, update_e0=True)
    assert out["e0"][0] == pytest.approx(e_trial, rel=1e-13)
    assert out["W"] == pytest.approx(Wr, rel=1e-12)
    assert out["E"] == pytest.approx(Er, rel=1e-12)
    assert all(x > 0 for x in out["W"])


def test_energy_run_reports_a_dead_population():
    """A population whose total weight is 0 at a comb cannot update E_0: the
    run stops with an error naming the step instead of passing a NaN E_0 on
    to the next step; a run asked to seed E_0 from such a population refuses."""
    import torch
    from oracle_context import OracleContext
    from paper_2403_02542_gb300.inputs import make_fields, make_system
    s = make_system(8, 2, 2, 32, rho=0.5, seed=20240304)
    octx = OracleContext(s)
    w = octx.new_walkers(4)
    octx.init_walkers(w)
    w.W = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError, match="positive weight"):
        S.initial_e0(octx, w, 0.05)
    with pytest.raises(RuntimeError, match="died at step 1"):
        S.energy_run(octx, w, 0.05, -7.0, 4, fields=lambda k: torch.as_tensor(make_fields(1, k, 4, s.G)),
                     order=6, pop_every=2, seed=1, update_e0=True)

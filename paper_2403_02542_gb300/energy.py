"""Energy runs and their statistics: the time average of the mixed estimator
with its variance and correlation length (Sec. II.A), and the time-step
extrapolation E(tau) = E_0 + alpha tau + beta tau^2 (Eq. square_fit) or its
pure quadratic (Split-2, Taylor propagator) and linear (Split-1,
Crank-Nicolson) forms (Sec. V.G).

Readings where the paper leaves the procedure open:
  * the correlation length kappa of the variance sigma_Ebar^2 = sigma_E^2 kappa / N
    is taken from a blocking analysis: the post-equilibration series E_k is
    averaged (weights W_k) in blocks of 2^b steps, the variance of the mean is
    estimated from the block means at every level, and the first level whose
    estimate is within its own statistical uncertainty of the next level's (a
    plateau) is kept; kappa = N sigma_Ebar^2 / sigma_E^2;
  * E_0 (the best estimate of the ground-state energy, Eq. imag_prop) may be
    updated during a run: at every population-control event it becomes the
    latest mixed estimate E_k during equilibration and the running time
    average after it;
  * population control is the comb of afqmc_population_control with uniform
    numbers drawn from one seeded generator per run.
The statistics are host arithmetic on the per-step estimates; the steps run in
the library.
"""
from __future__ import annotations

import math

import numpy as np


def time_average(W, E, n_eq: int = 0):
    """(E_bar, sigma_E^2) of the samples k > n_eq: E_bar = sum W_k E_k / sum W_k,
    sigma_E^2 = <E^2> - E_bar^2 with the same weights (Sec. II.A)."""
    W = np.asarray(W, dtype=np.float64)[n_eq:]
    E = np.asarray(E, dtype=np.float64)[n_eq:]
    if W.size == 0 or not W.sum() > 0:
        raise ValueError("no samples after equilibration")
    wsum = W.sum()
    ebar = float((W * E).sum() / wsum)
    e2 = float((W * E * E).sum() / wsum)
    return ebar, max(e2 - ebar * ebar, 0.0)


def blocking(W, E, n_eq: int = 0, min_blocks: int = 8):
    """Blocking analysis of the post-equilibration series.  Returns a dict with
    E_bar, sigma_E2, the chosen block size, sigma (the standard error of E_bar),
    kappa = N sigma^2 / sigma_E^2 and the per-level estimates [(size, sigma, dsigma)]."""
    W = np.asarray(W, dtype=np.float64)[n_eq:]
    E = np.asarray(E, dtype=np.float64)[n_eq:]
    n = E.size
    ebar, var = time_average(W, E)
    levels = []
    size = 1
    while n // size >= min_blocks:
        nb = n // size
        Wb = W[: nb * size].reshape(nb, size)
        Eb = E[: nb * size].reshape(nb, size)
        means = (Wb * Eb).sum(1) / Wb.sum(1)
        s2 = float(((means - means.mean()) ** 2).sum() / (nb - 1) / nb)  # variance of the mean
        s = math.sqrt(max(s2, 0.0))
        levels.append((size, s, s / math.sqrt(2.0 * (nb - 1))))
        size *= 2
    if not levels:
        raise ValueError("too few samples for a blocking analysis")
    chosen = levels[-1]
    for a, b in zip(levels, levels[1:]):
        if b[1] - a[1] <= a[2]:  # the next level agrees within this level's uncertainty
            chosen = a
            break
    sigma = chosen[1]
    kappa = n * sigma * sigma / var if var > 0 else 1.0
    return dict(E_bar=ebar, sigma_E2=var, block=chosen[0], sigma=sigma, kappa=kappa, levels=levels, n=n)


def fit_time_step(taus, energies, sigmas=None, powers=(1, 2)):
    """Weighted least-squares fit E(tau) = E_0 + sum_p c_p tau^p over the given
    powers (Sec. V.G): (1, 2) is the general form E_0 + alpha tau + beta tau^2 of
    Eq. square_fit, (2,) the pure quadratic of Split-2 and the Taylor propagator,
    (1,) the linear form of Split-1 and Crank-Nicolson.  Returns a dict with E_0,
    the coefficients c [per power], their standard errors, and chi^2 per
    degree of freedom (None without a spare point)."""
    t = np.asarray(taus, dtype=np.float64)
    y = np.asarray(energies, dtype=np.float64)
    powers = tuple(powers)
    if t.size < 1 + len(powers):
        raise ValueError("need at least one time step per fitted coefficient")
    s = np.ones_like(y) if sigmas is None else np.asarray(sigmas, dtype=np.float64)
    X = np.stack([np.ones_like(t)] + [t ** p for p in powers], axis=1)
    wgt = 1.0 / (s * s)
    cov = np.linalg.inv(X.T @ (X * wgt[:, None]))
    coef = cov @ (X.T @ (wgt * y))
    resid = y - X @ coef
    dof = t.size - X.shape[1]
    chi2 = float((wgt * resid * resid).sum() / dof) if dof > 0 else None
    err = np.sqrt(np.diag(cov))
    return {"E0": float(coef[0]), "sigma_E0": float(err[0]), "powers": powers,
            "c": [float(v) for v in coef[1:]], "sigma_c": [float(v) for v in err[1:]], "chi2_dof": chi2}


def extrapolation_error(sigmas) -> float:
    """The paper's estimate of the statistical error of an extrapolated energy
    (Eq. staterr): sigma_x = sqrt(sum_i sigma_i^2) / N_tau over the N_tau time
    steps of the fit, sigma_i their 1-sigma errors.  (fit_time_step also reports
    the least-squares standard error of E_0, which weighs the points.)"""
    s = np.asarray(sigmas, dtype=np.float64)
    if s.size == 0:
        raise ValueError("no time steps")
    return float(math.sqrt((s * s).sum()) / s.size)


def extrapolate(taus, energies, sigmas=None, power: int = 2):
    """Weighted least-squares fit E(tau) = E_0 + c tau^power (power 2: Split-2 and
    the Taylor propagator; power 1: Split-1 and Crank-Nicolson).  Returns
    (E_0, c, sigma_E0, sigma_c, chi2 per degree of freedom or None)."""
    f = fit_time_step(taus, energies, sigmas, (power,))
    return f["E0"], f["c"][0], f["sigma_E0"], f["sigma_c"][0], f["chi2_dof"]


def initial_e0(ctx, walkers, tau: float) -> float:
    """A starting E_0 for a run: the weighted mean of Re E_L over the live
    walkers, uncapped.  (A local energy evaluated with some other E_0 is
    clamped to that E_0 +- DeltaE by Eq. enwin, so its mixed estimate is not a
    usable seed when |E| is large against DeltaE.)"""
    import torch
    e_loc = torch.empty(walkers.n, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    ctx.local_energy(walkers, 0.0, tau, e_loc, e_mix)
    W = walkers.weight.double()
    live = W > 0
    if not bool(live.any()):
        raise ValueError("initial_e0: no walker has a positive weight")
    return float((W[live] * e_loc[live, 0]).sum() / W[live].sum())


def energy_run(ctx, walkers, tau: float, e0, n_steps: int, *, fields, n_eq: int = 0,
               expm: str = "krylov", order: int = 10, reortho_every: int = 5, pop_every: int = 0,
               seed: int = 0, update_e0: bool = False, reuse_bias: bool = False, propagator: str = "split2",
               group=None):
    """Propagate `walkers` for n_steps steps of the library with the local energy
    measured every step.  fields(k) returns the device fields [Nw, G] of step k.
    propagator selects the walker update of Sec. III (see Context.step); fit
    the energies of Split-1 and Crank-Nicolson runs with power 1 in
    `extrapolate`.
    With pop_every > 0 the population is combed after every pop_every steps
    (uniform numbers from numpy's PCG64 seeded with `seed`).  Returns a dict
    with the per-step total weight W, mixed estimate E and E_0 used, and the
    blocking analysis of the steps after n_eq.

    e0: the starting E_0, or None to take it from the uncapped local energies
    of the starting walkers (initial_e0; with a group, the weighted mean over
    all ranks).

    group: a torch.distributed process group whose ranks each propagate their
    own walkers (the population sharded by walkers).  Every step then
    all-reduces [sum W E_k, sum W] once, so W and E are the whole population's
    (W_local and E_local keep this rank's); each rank combs its own walkers
    with numbers from PCG64([seed, rank]) (the comb keeps each rank's total
    weight, so the global estimate needs no further exchange); E_0 is updated
    from the global estimates and stays the same on every rank.  With an NCCL
    group the two numbers are reduced on ctx's device."""
    import torch
    nw = walkers.n
    dev = ctx.device
    e_loc = torch.empty(nw, 2, dtype=torch.float64, device=dev)
    e_mix = torch.empty(4, dtype=torch.float64, device=dev)
    if group is None:
        rng = np.random.Generator(np.random.PCG64(seed))
    else:
        import torch.distributed as dist
        rng = np.random.Generator(np.random.PCG64([seed, dist.get_rank(group)]))
        red_dev = dev if dist.get_backend(group) == "nccl" else torch.device("cpu")
    if e0 is None:
        if group is None:
            e0 = initial_e0(ctx, walkers, tau)
        else:
            e_loc0 = torch.empty(nw, 2, dtype=torch.float64, device=dev)
            e_mix0 = torch.empty(4, dtype=torch.float64, device=dev)
            ctx.local_energy(walkers, 0.0, tau, e_loc0, e_mix0)
            W0 = walkers.weight.double()
            live = W0 > 0
            t = torch.stack([(W0[live] * e_loc0[live, 0]).sum(), W0[live].sum()]).to(red_dev)
            dist.all_reduce(t, group=group)
            t = t.cpu()
            if not float(t[1]) > 0:
                raise ValueError("energy_run: no walker has a positive weight")
            e0 = float(t[0] / t[1])
    Ws, Es, E0s, Wl, El = [], [], [], [], []
    for k in range(n_steps):
        reo = reortho_every > 0 and (k + 1) % reortho_every == 0
        ctx.step(walkers, fields(k), tau, e0, expm=expm, order=order, reortho=reo, measure=True,
                 e_loc=e_loc, e_mix=e_mix, reuse_bias=reuse_bias, propagator=propagator)
        m = e_mix.cpu()
        E0s.append(e0)
        w_k, e_k = float(m[1]), float(m[2])
        if group is None:
            Ws.append(w_k)
            Es.append(e_k)
        else:
            Wl.append(w_k)
            El.append(e_k)
            t = torch.tensor([w_k * e_k if w_k > 0 else 0.0, w_k], dtype=torch.float64, device=red_dev)
            dist.all_reduce(t, group=group)
            t = t.cpu()
            Ws.append(float(t[1]))
            Es.append(float(t[0] / t[1]) if float(t[1]) > 0 else float("nan"))
        if pop_every > 0 and (k + 1) % pop_every == 0:
            ctx.population_control(walkers, float(rng.random()))
            if update_e0:
                if not (Ws[-1] > 0 and math.isfinite(Es[-1])):
                    raise RuntimeError(f"energy_run: the population has died at step {k} "
                                       f"(total weight {Ws[-1]}, E_k {Es[-1]}); E_0 cannot be updated")
                e0 = Es[-1] if k < n_eq else time_average(Ws, Es, n_eq)[0]
    out = dict(W=Ws, E=Es, e0=E0s)
    if group is not None:
        out["W_local"], out["E_local"] = Wl, El
    if n_steps - n_eq >= 16:
        out["stats"] = blocking(Ws, Es, n_eq)
    return out

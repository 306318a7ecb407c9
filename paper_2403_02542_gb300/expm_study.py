"""Accuracy of the actions of the one-body exponential inside a short ph-AFQMC
run (Sec. IV.E, Fig. 1): the smallest order k_min of an action, that is the
number of A|Psi> products it makes per step, whose run energy stays within
eps of the same run with an exact exponential.

Readings where the paper leaves the protocol open:
  * the energy of a run is the mixed estimate E_k (Sec. II.A) averaged over
    its steps; every run starts from the trial with unit weights, draws the
    same fields and does not re-orthonormalise, so two runs differ only by the
    action and its order;
  * the exact exponential is the Taylor series of order 64 (the paper
    diagonalises instead; for ||A|| <= 8 the order-64 remainder
    ||A||^65 e^||A|| / 65! is below 1e-28, so the two agree to rounding);
  * k_min is the first order k = 1, 2, ... whose error is below eps, or None
    when no order up to the action's largest one is.
The runs go through the library (`Context.step`); this module only drives them
and compares their energies.
"""
from __future__ import annotations

# largest order each action accepts (afqmc_step)
K_MAX = {"taylor": 64, "chebyshev": 64, "krylov": 32, "bkrylov": 16, "lanczos": 32}
REFERENCE = ("taylor", 64)


def run_energy(ctx, nw: int, n_steps: int, fields, tau: float, e0: float, expm: str, order: int,
               propagator: str = "split2") -> float:
    """Mean over n_steps steps of the mixed estimate E_k of nw walkers started
    at the trial; fields(k) returns the fields [nw, G] of step k on ctx's device."""
    import torch
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    e_loc = torch.empty(nw, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    total = 0.0
    for k in range(n_steps):
        ctx.step(w, fields(k), tau, e0, expm=expm, order=order, measure=True, e_loc=e_loc, e_mix=e_mix,
                 propagator=propagator)
        total += float(e_mix[2])
    return total / n_steps


def k_min(ctx, nw: int, n_steps: int, fields, tau: float, e0: float, expm: str, eps: float = 1e-5,
          k_max: int | None = None, e_ref: float | None = None, propagator: str = "split2") -> dict:
    """Smallest order of `expm` whose run energy is within eps of the
    reference run's (computed here unless e_ref is given).  Returns
    {"k_min": k or None, "errors": [error at k = 1, 2, ...], "e_ref": e_ref}."""
    if e_ref is None:
        e_ref = run_energy(ctx, nw, n_steps, fields, tau, e0, *REFERENCE, propagator=propagator)
    top = K_MAX[expm] if k_max is None else min(k_max, K_MAX[expm])
    errors = []
    for k in range(1, top + 1):
        err = abs(run_energy(ctx, nw, n_steps, fields, tau, e0, expm, k, propagator=propagator) - e_ref)
        errors.append(err)
        if err < eps:  # a NaN energy (every walker removed) never passes
            return {"k_min": k, "errors": errors, "e_ref": e_ref}
    return {"k_min": None, "errors": errors, "e_ref": e_ref}


def sweep(ctx, nw: int, n_steps: int, fields_for_tau, taus, e0: float,
          methods=("taylor", "chebyshev", "krylov", "bkrylov", "lanczos"), eps: float = 1e-5,
          k_max: int | None = None) -> dict:
    """k_min of every method at every time step (the rows of Fig. 1 for one
    system).  fields_for_tau(tau) returns the fields callable of that tau's runs;
    k_max caps the orders tried (None: each action's largest)."""
    out = {}
    for tau in taus:
        fields = fields_for_tau(tau)
        e_ref = run_energy(ctx, nw, n_steps, fields, tau, e0, *REFERENCE)
        out[tau] = {"e_ref": e_ref}
        for m in methods:
            out[tau][m] = k_min(ctx, nw, n_steps, fields, tau, e0, m, eps=eps, k_max=k_max, e_ref=e_ref)["k_min"]
    return out

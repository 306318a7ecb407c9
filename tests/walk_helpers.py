"""Shared drivers for the parity tests: the same seeded system and fields go
through the CUDA library (via the C ABI binding) and through the CPU oracle."""
import math

import numpy as np
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import make_fields


def oracle_setup(sys_, tau, trial=None, na=None, nb=None):
    trial = sys_.trial if trial is None else trial
    na = sys_.na if na is None else na
    nb = sys_.nb if nb is None else nb
    ham = R.make_hamiltonian(sys_.h1, sys_.L, trial, na, nb, sys_.e_const)
    Lbar = R.mean_field_shift(ham)
    hpp, ec = R.propagation_h1(ham, Lbar)
    B = R.half_step_propagator(hpp, tau)
    return ham, Lbar, ec, B


def near_ties(info, tau, e0, eps=1e-9):
    """Decisions whose argument lies within eps (relative) of its threshold (reading R9)."""
    f = info.f.abs()
    fac = info.factor
    n = int(((f - 1.0).abs() < eps).sum())
    n += int(((fac - 10.0).abs() < 10 * eps).sum())
    n += int((torch.cos(info.dtheta).abs() < eps).sum())
    return n


def oracle_walk(sys_, nw, steps, tau, e0, expm, order, reortho_every, seed, dead=(),
                trial=None, na=None, nb=None, psi0=None, lo0=None, W0=None, field_fn=None,
                propagator="split2"):
    ham, Lbar, ec, B = oracle_setup(sys_, tau, trial, na, nb)
    if psi0 is None:
        psi, lo, W = R.init_walkers(ham, nw)
    else:
        psi, lo, W = psi0.clone(), lo0.clone(), W0.clone()
    for d in dead:
        W[d] = 0.0
    out = []
    ties = 0
    for k in range(steps):
        x = make_fields(seed, k, nw, ham.G) if field_fn is None else field_fn(k)
        reo = reortho_every > 0 and (k + 1) % reortho_every == 0
        psi, lo, W, info = R.step(ham, psi, lo, W, x, tau, e0, method=expm, k=order, reortho=reo,
                                  B=B, L_bar=Lbar, ec=ec, propagator=propagator)
        ties += near_ties(info, tau, e0)
        El = R.local_energy(ham, psi)
        Ecap = R.energy_window(El, e0, tau, ham.na + ham.nb)
        emix, wsum = R.mixed_energy(W, Ecap)
        out.append(dict(psi=psi.clone(), lo=lo.clone(), W=W.clone(), El=El.clone(), emix=emix,
                        wsum=wsum))
    return out, ties


def gpu_walk(ctx, nw, steps, tau, e0, expm, order, reortho_every, seed, dead=(), record=None,
             state=None, field_fn=None, reuse_bias=False, propagator="split2"):
    """record: set of step indices to copy back (default: all)."""
    w = ctx.new_walkers(nw)
    if state is None:
        ctx.init_walkers(w)
    else:
        w.psi.copy_(state["psi"])
        w.weight.copy_(state["W"])
        w.logovl.copy_(state["lo"])
        w.status.zero_()
    for d in dead:
        w.weight[d] = 0.0
    e_loc = torch.empty(nw, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    out = []
    for k in range(steps):
        x = make_fields(seed, k, nw, ctx.G) if field_fn is None else field_fn(k)
        x = torch.as_tensor(np.ascontiguousarray(x), device=ctx.device)
        reo = reortho_every > 0 and (k + 1) % reortho_every == 0
        ctx.step(w, x, tau, e0, expm=expm, order=order, reortho=reo, measure=True,
                 e_loc=e_loc, e_mix=e_mix, reuse_bias=reuse_bias, propagator=propagator)
        if record is None or k in record:
            torch.cuda.synchronize()
            out.append(dict(k=k, psi=w.psi.cpu().to(torch.complex128).transpose(1, 2).contiguous(),
                            lo=torch.complex(w.logovl[:, 0], w.logovl[:, 1]).cpu(),
                            W=w.weight.cpu().clone(), status=w.status.cpu().clone(),
                            El=torch.complex(e_loc[:, 0], e_loc[:, 1]).cpu(),
                            emix=e_mix.cpu().clone()))
    ctx.sync()
    return out, w


def compare(g, r, rtol, alive=None, what=""):
    """Per-walker relative comparison of walkers, weights, log-overlaps, E_L."""
    W = r["W"]
    live = (W > 0) if alive is None else alive
    idx = torch.nonzero(live).flatten().tolist()
    assert len(idx) > 0
    worst = {}
    for w in idx:
        e_psi = float((g["psi"][w] - r["psi"][w]).norm() / r["psi"][w].norm())
        e_W = abs(float(g["W"][w] - W[w])) / max(abs(float(W[w])), 1e-300)
        d = complex(g["lo"][w] - r["lo"][w])
        e_lo = max(abs(d.real) / max(1.0, abs(r["lo"][w].real)),
                   abs((d.imag + math.pi) % (2 * math.pi) - math.pi))
        e_E = abs(complex(g["El"][w] - r["El"][w])) / abs(complex(r["El"][w]))
        for k, v in (("psi", e_psi), ("W", e_W), ("logovl", e_lo), ("E_L", e_E)):
            worst[k] = max(worst.get(k, 0.0), v)
    for k, v in worst.items():
        assert v <= rtol, f"{what} {k}: relative error {v:.3e} > {rtol:.1e}"
    return worst


def oracle_energy_run(s, nw, tau, e0, n_steps, n_eq, order, reortho_every, pop_every, seed, fseed):
    """The protocol of energy.energy_run (update_e0=True) driven through the
    oracle: steps with E_L every step, the comb every pop_every steps with
    numbers from one PCG64(seed), E_0 updated at each comb.  Returns the
    per-step total weights and mixed estimates."""
    from paper_2403_02542_gb300 import energy as S
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

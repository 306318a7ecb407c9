"""Energy and its derivative along a one-parameter path of Hamiltonians, the
shape of a bond-length scan: h1(s) = h1 + s dH1, L(s) = L + s dL.

At every point the energy is J(s) = E_n, the mixed estimator after an n-step
fixed-field walk from the trial (the same fields, trial and E_0 at every s,
so the points are correlated), and its derivative
dJ/ds = sum dJ/dh1 * dH1 + sum dJ/dL * dL from the walk adjoint
(afqmc_walk_backward).  Central differences of J along the path are taken
beside it as a check.  The paper has no gradients; this uses the library's
adjoint of the fixed-field walk (Split-2 with the Taylor action, Sec. III.B,
Eq. taylor, or the Krylov action of Eqs. krylovsub-krylov by Arnoldi or by
the complex-symmetric Lanczos recurrence).
"""
from __future__ import annotations

import numpy as np
import torch

from .api import Context, walk_energy


def path_scan(system, fields: torch.Tensor, s_values, dH1: np.ndarray, dL: np.ndarray, tau: float, e0: float,
              order: int = 6, reortho_every: int = 0, ckpt_every: int = 10, precision: str = "mixed",
              fd_step: float | None = 1e-2, device="cuda", expm: str = "taylor"):
    """Returns a list of dicts {s, J, dJds, dJds_fd (or None), live} for every s."""
    out = []
    nw = int(fields.shape[1])
    for s in s_values:
        h1 = system.h1 + s * dH1
        L = system.L + s * dL
        c = Context(h1, L, system.trial, system.na, system.nb, system.e_const, precision=precision, device=device)
        try:
            w = c.new_walkers(nw)
            c.init_walkers(w)
            J, gh, gL = c.walk_backward(w, fields, tau, e0, order=order, reortho_every=reortho_every,
                                        ckpt_every=ckpt_every, expm=expm)
            dJds = float((gh.cpu().numpy() * dH1).sum() + (gL.cpu().numpy() * dL).sum())
            Jv, live = float(J[2]), float(J[3])
        finally:
            c.close()
        fd = None
        if fd_step:
            vals = []
            for sign in (1.0, -1.0):
                sp = s + sign * fd_step
                c = Context(system.h1 + sp * dH1, system.L + sp * dL, system.trial, system.na, system.nb,
                            system.e_const, precision=precision, device=device)
                try:
                    vals.append(float(walk_energy(c, nw, fields, tau, e0, order, reortho_every, expm)[2]))
                finally:
                    c.close()
            fd = (vals[0] - vals[1]) / (2.0 * fd_step)
        out.append({"s": float(s), "J": Jv, "dJds": dJds, "dJds_fd": fd, "live": live})
    torch.cuda.synchronize()
    return out

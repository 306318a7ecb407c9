"""A CPU stand-in for `Context` whose steps are the oracle's: the same
new_walkers / init_walkers / step(measure=True) / population_control calls,
walkers kept as oracle tensors.  Tests use it to exercise host-side drivers
(the accuracy study, the energy run) without a GPU, and to compute, through the
oracle, what the library should give."""
from types import SimpleNamespace

import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import make_fields


class OracleContext:
    def __init__(self, sys_):
        self.sys = sys_
        self.ham = R.make_hamiltonian(sys_.h1, sys_.L, sys_.trial, sys_.na, sys_.nb, sys_.e_const)
        self.L_bar = R.mean_field_shift(self.ham)
        self.hpp, self.ec = R.propagation_h1(self.ham, self.L_bar)
        self.G = self.ham.G
        self.device = torch.device("cpu")
        self._B = {}

    def new_walkers(self, n):
        return _Walkers(n)

    def init_walkers(self, w):
        w.psi, w.lo, w.W = R.init_walkers(self.ham, w.n)

    def step(self, w, fields, tau, e0, expm="krylov", order=10, reortho=False, measure=False, e_loc=None,
             e_mix=None, reuse_bias=False, propagator="split2"):
        if tau not in self._B:
            self._B[tau] = R.half_step_propagator(self.hpp, tau)
        w.psi, w.lo, w.W, _ = R.step(self.ham, w.psi, w.lo, w.W, torch.as_tensor(fields).cpu(), tau, e0,
                                     method=expm, k=order, reortho=reortho, B=self._B[tau], L_bar=self.L_bar,
                                     ec=self.ec, propagator=propagator)
        if measure:
            El = R.local_energy(self.ham, w.psi)
            Ecap = R.energy_window(El, e0, tau, self.ham.na + self.ham.nb)
            emix, wsum = R.mixed_energy(w.W, Ecap)
            if e_loc is not None:
                e_loc[:, 0] = El.real
                e_loc[:, 1] = El.imag
            if e_mix is not None:
                e_mix[1] = float(wsum)
                e_mix[2] = float(emix)

    def local_energy(self, w, e0, tau, e_loc=None, e_mix=None):
        El = R.local_energy(self.ham, w.psi)
        emix, wsum = R.mixed_energy(w.W, R.energy_window(El, e0, tau, self.ham.na + self.ham.nb))
        if e_loc is None:
            e_loc = torch.empty(w.n, 2, dtype=torch.float64)
        if e_mix is None:
            e_mix = torch.zeros(4, dtype=torch.float64)
        e_loc[:, 0] = El.real
        e_loc[:, 1] = El.imag
        e_mix[1] = float(wsum)
        e_mix[2] = float(emix)
        return e_loc, e_mix

    def population_control(self, w, u, index_out=None):
        w.psi, w.lo, w.W, idx = R.population_control(w.psi, w.lo, w.W, u)
        if index_out is not None:
            index_out.copy_(idx)


class _Walkers(SimpleNamespace):
    """Oracle walkers (psi, log-overlap, weights); `weight` names W as the
    library's walker set does."""

    def __init__(self, n):
        super().__init__(n=n, psi=None, lo=None, W=None)

    @property
    def weight(self):
        return self.W


def field_fn(seed, nw, G, device=None):
    """fields(k) of one seeded run (make_fields), on `device` when given."""
    def f(k):
        x = torch.as_tensor(make_fields(seed, k, nw, G))
        return x.to(device) if device is not None else x
    return f

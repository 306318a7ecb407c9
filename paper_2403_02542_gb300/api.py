"""Python face of the walker-step library: device buffers from PyTorch,
everything else through the C ABI (include/afqmc.h)."""
from __future__ import annotations

import ctypes
import json
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

# walker updates of Sec. III built in the library
PROPAGATORS = {"split2": L.AFQMC_SPLIT2, "split1": L.AFQMC_SPLIT1, "taylor": L.AFQMC_TAYLORPROP,
               "cn": L.AFQMC_CN}
# actions of the one-body exponential of Sec. IV built in the library
EXPMS = {"taylor": L.AFQMC_EXPM_TAYLOR, "krylov": L.AFQMC_EXPM_KRYLOV, "bkrylov": L.AFQMC_EXPM_BLOCK_KRYLOV,
         "chebyshev": L.AFQMC_EXPM_CHEBYSHEV, "lanczos": L.AFQMC_EXPM_LANCZOS}


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


@dataclass
class WalkerSet:
    """Caller-owned device buffers of a walker population.

    psi     [Nw, nc, N] complex128 (FP64 context) or complex64 (mixed);
            psi[w, j, p] is coefficient p of orbital j (alpha j < na).
    weight  [Nw] float64
    logovl  [Nw, 2] float64 (Re, Im of log <Psi_T|Psi>)
    status  [Nw] int32 (AFQMC_W_* bits)
    """

    psi: torch.Tensor
    weight: torch.Tensor
    logovl: torch.Tensor
    status: torch.Tensor

    @property
    def n(self) -> int:
        return self.psi.shape[0]

    def c_struct(self) -> L.Walkers:
        return L.Walkers(self.n, _ptr(self.psi), _ptr(self.weight), _ptr(self.logovl),
                         _ptr(self.status))


class Context:
    """One Hamiltonian + trial determinant on one GPU (afqmc_create)."""

    def __init__(self, h1, chol, trial, na: int, nb: int, e_const: float = 0.0,
                 precision: str = "fp64", device: str | torch.device = "cuda",
                 stream: torch.cuda.Stream | None = None):
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("the walker step runs on a CUDA device only")
        h1 = np.ascontiguousarray(h1, dtype=np.float64)
        chol = np.ascontiguousarray(chol, dtype=np.float64)
        # trial arrives as [N, na+nb] (columns = orbitals); the ABI wants orbital-major
        trial_om = np.ascontiguousarray(np.asarray(trial, dtype=np.float64).T)
        self.N = h1.shape[0]
        self.G = chol.shape[0]
        self.na, self.nb = int(na), int(nb)
        self.nc = self.na + self.nb
        self.precision = precision
        self.ctype = torch.complex128 if precision == "fp64" else torch.complex64
        prec = {"fp64": L.AFQMC_FP64, "mixed": L.AFQMC_MIXED}[precision]
        self._stream = stream
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = L.lib().afqmc_create(ctypes.byref(handle), self.N, self.na, self.nb, self.G,
                                      h1.ctypes.data, chol.ctypes.data, trial_om.ctypes.data,
                                      float(e_const), prec, self._stream_ptr())
        L.check(st, "afqmc_create")
        self._h = handle

    def _stream_ptr(self):
        s = self._stream if self._stream is not None else torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def _bind_stream(self):
        L.check(L.lib().afqmc_set_stream(self._h, self._stream_ptr()), "afqmc_set_stream")

    def close(self):
        if getattr(self, "_h", None):
            L.lib().afqmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def new_walkers(self, n: int) -> WalkerSet:
        d = self.device
        return WalkerSet(
            psi=torch.empty(n, self.nc, self.N, dtype=self.ctype, device=d),
            weight=torch.empty(n, dtype=torch.float64, device=d),
            logovl=torch.empty(n, 2, dtype=torch.float64, device=d),
            status=torch.zeros(n, dtype=torch.int32, device=d),
        )

    def set_tau(self, tau: float):
        L.check(L.lib().afqmc_set_tau(self._h, float(tau)), "afqmc_set_tau")

    def init_walkers(self, w: WalkerSet):
        self._bind_stream()
        cw = w.c_struct()
        L.check(L.lib().afqmc_walkers_init(self._h, ctypes.byref(cw)), "afqmc_walkers_init")

    def step(self, w: WalkerSet, fields: torch.Tensor, tau: float, e0: float,
             expm: str = "krylov", order: int = 10, reortho: bool = False,
             measure: bool = False, e_loc: torch.Tensor | None = None,
             e_mix: torch.Tensor | None = None, reuse_bias: bool = False, propagator: str = "split2"):
        """One walker step (afqmc_step).  fields: device [Nw, G] float64.
        reuse_bias: take the force bias from the previous measurement of the
        same, unchanged walkers (see afqmc_step_params in the header).
        propagator: "split2" (default), "split1", "taylor" (the Taylor
        propagator; expm must then be "taylor") or "cn" (Crank-Nicolson;
        expm and order are not used)."""
        assert fields.dtype == torch.float64 and fields.is_cuda and fields.is_contiguous()
        self._bind_stream()
        p = L.StepParams(float(tau), float(e0), PROPAGATORS[propagator],
                         EXPMS[expm],
                         int(order), int(bool(reortho)), int(bool(measure)), int(bool(reuse_bias)))
        cw = w.c_struct()
        L.check(L.lib().afqmc_step(self._h, ctypes.byref(cw), fields.data_ptr(), ctypes.byref(p),
                                   _ptr(e_loc), _ptr(e_mix)), "afqmc_step")

    def local_energy(self, w: WalkerSet, e0: float, tau: float, e_loc=None, e_mix=None):
        """E_L per walker [Nw, 2] and (sum W E_cap, sum W, E_k, live) [4]."""
        if e_loc is None:
            e_loc = torch.empty(w.n, 2, dtype=torch.float64, device=self.device)
        if e_mix is None:
            e_mix = torch.empty(4, dtype=torch.float64, device=self.device)
        self._bind_stream()
        cw = w.c_struct()
        L.check(L.lib().afqmc_local_energy(self._h, ctypes.byref(cw), float(e0), float(tau),
                                           e_loc.data_ptr(), e_mix.data_ptr()), "afqmc_local_energy")
        return e_loc, e_mix

    def population_control(self, w: WalkerSet, u: float, index_out: torch.Tensor | None = None):
        """Comb resampling with uniform u in [0, 1) (afqmc_population_control)."""
        self._bind_stream()
        cw = w.c_struct()
        L.check(L.lib().afqmc_population_control(self._h, ctypes.byref(cw), float(u), _ptr(index_out)),
                "afqmc_population_control")

    def sync(self):
        L.check(L.lib().afqmc_sync(self._h), "afqmc_sync")

    def energy_backward(self, w: WalkerSet, e0: float, tau: float, dJ: float = 1.0):
        """(dE_k/dh1 [N,N], dE_k/dL [G,N,N]) at fixed walkers (afqmc_energy_backward)."""
        gh = torch.empty(self.N, self.N, dtype=torch.float64, device=self.device)
        gL = torch.empty(self.G, self.N, self.N, dtype=torch.float64, device=self.device)
        self._bind_stream()
        cw = w.c_struct()
        L.check(L.lib().afqmc_energy_backward(self._h, ctypes.byref(cw), float(e0), float(tau), float(dJ),
                                              gh.data_ptr(), gL.data_ptr()), "afqmc_energy_backward")
        return gh, gL

    def walk_backward(self, w: WalkerSet, fields: torch.Tensor, tau: float, e0: float, order: int = 6,
                      reortho_every: int = 0, ckpt_every: int = 10, dJ: float = 1.0, grad_psi0: bool = False,
                      expm: str = "taylor"):
        """Gradient of the mixed estimator after a fixed-field walk (afqmc_walk_backward).

        `w` holds the walkers at step 0 (left unchanged); `fields` is a device
        tensor [n_steps, Nw, G] of the walk's auxiliary fields; `expm` is
        "taylor" (order = Taylor order), "krylov" (Arnoldi) or "lanczos"
        (order = Krylov dimension), the action of e^A in every step.  Returns
        (e_mix [4], dJ/dh1 [N,N], dJ/dL [G,N,N]) and, with grad_psi0=True, the
        derivative G [Nw, na+nb, N] (the walkers' complex type) with
        dJ = Re sum G * dPsi_0 as well.  In a mixed context the walk and its
        reverse run on complex64 walkers (FP32 contractions, FP64 overlaps,
        determinants and gradient sums).
        """
        f = fields.to(device=self.device, dtype=torch.float64).contiguous()
        if f.dim() != 3 or f.shape[1] != w.n or f.shape[2] != self.G:
            raise ValueError("fields must be [n_steps, n_walkers, G]")
        if expm not in ("taylor", "krylov", "lanczos"):
            raise ValueError("the walk adjoint takes expm='taylor', 'krylov' or 'lanczos'")
        p = L.WalkAdjointParams(int(f.shape[0]), int(order), int(reortho_every), int(ckpt_every),
                                float(tau), float(e0), float(dJ), EXPMS[expm])
        J = torch.empty(4, dtype=torch.float64, device=self.device)
        gh = torch.empty(self.N, self.N, dtype=torch.float64, device=self.device)
        gL = torch.empty(self.G, self.N, self.N, dtype=torch.float64, device=self.device)
        gp = torch.empty(w.n, self.nc, self.N, dtype=self.ctype, device=self.device) if grad_psi0 else None
        self._bind_stream()
        cw = w.c_struct()
        L.check(L.lib().afqmc_walk_backward(self._h, ctypes.byref(cw), f.data_ptr(), ctypes.byref(p), J.data_ptr(),
                                            gh.data_ptr(), gL.data_ptr(), gp.data_ptr() if gp is not None else None),
                "afqmc_walk_backward")
        if grad_psi0:
            return J, gh, gL, gp
        return J, gh, gL

    # ------------------------------------------------------------------ tuning
    def tune_key(self, n_walkers: int) -> str:
        return f"N{self.N}_na{self.na}_nb{self.nb}_G{self.G}_{self.precision}_w{n_walkers}"

    def autotune(self, n_walkers: int, cache: str | None = None) -> list:
        """Pick the GEMM tile variant of every call site (afqmc_autotune); with
        `cache` (a JSON file) a table measured earlier for the same shape is reused."""
        table = (ctypes.c_int32 * 4)()
        key = self.tune_key(n_walkers)
        if cache and os.path.exists(cache):
            with open(cache) as f:
                known = json.load(f)
            if key in known:
                for i, v in enumerate(known[key]):
                    table[i] = int(v)
                L.check(L.lib().afqmc_tune_set(self._h, table), "afqmc_tune_set")
                return list(table)
        self._bind_stream()
        L.check(L.lib().afqmc_autotune(self._h, int(n_walkers), table), "afqmc_autotune")
        if cache:
            known = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    known = json.load(f)
            known[key] = list(table)
            with open(cache, "w") as f:
                json.dump(known, f, indent=1, sort_keys=True)
        return list(table)

    def tune_table(self) -> list:
        table = (ctypes.c_int32 * 4)()
        L.check(L.lib().afqmc_tune_get(self._h, table), "afqmc_tune_get")
        return list(table)

    def profile(self, enable: bool, classes=None):
        """Start (clearing) or stop per-kernel-class event timing: every class
        (afqmc_profile), or only the named ones of L.KERNEL_CLASSES
        (afqmc_profile_mask)."""
        if classes is None or not enable:
            L.check(L.lib().afqmc_profile(self._h, int(bool(enable))), "afqmc_profile")
            return
        mask = 0
        for name in classes:
            mask |= 1 << L.KERNEL_CLASSES.index(name)
        L.check(L.lib().afqmc_profile_mask(self._h, mask), "afqmc_profile_mask")

    def profile_read(self) -> dict:
        """{class: (total ms, launches)} accumulated since profile(True)."""
        ms = (ctypes.c_double * 7)()
        n = (ctypes.c_uint64 * 7)()
        L.check(L.lib().afqmc_profile_read(self._h, ms, n), "afqmc_profile_read")
        return {name: (ms[i], int(n[i])) for i, name in enumerate(L.KERNEL_CLASSES)}

    @property
    def launch_count(self) -> int:
        return int(L.lib().afqmc_launch_count(self._h))


def host_eigh(a: np.ndarray):
    """afqmc_host_eigh: (evals, evecs) of a real symmetric matrix."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    n = a.shape[0]
    ev = np.empty(n)
    V = np.empty((n, n))
    L.check(L.lib().afqmc_host_eigh(n, a.ctypes.data, ev.ctypes.data, V.ctypes.data),
            "afqmc_host_eigh")
    return ev, V


class Batch:
    """Several contexts stepped as one CUDA graph (afqmc_batch_*)."""

    def __init__(self, contexts: list):
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        h = ctypes.c_void_p()
        L.check(L.lib().afqmc_batch_create(ctypes.byref(h), arr, len(self.contexts)), "afqmc_batch_create")
        self._h = h

    def step(self, walker_sets, fields, tau, e0, expm="krylov", order=10, reortho=False, measure=False,
             e_loc=None, e_mix=None, stream: torch.cuda.Stream | None = None, reuse_bias=False,
             propagator="split2"):
        n = len(self.contexts)
        taus = tau if isinstance(tau, (list, tuple)) else [tau] * n
        e0s = e0 if isinstance(e0, (list, tuple)) else [e0] * n
        ws = (L.Walkers * n)(*[w.c_struct() for w in walker_sets])
        fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in fields])
        ex = EXPMS[expm]
        pr = PROPAGATORS[propagator]
        ps = (L.StepParams * n)(*[L.StepParams(float(taus[i]), float(e0s[i]), pr, ex, int(order),
                                               int(bool(reortho)), int(bool(measure)), int(bool(reuse_bias)))
                                  for i in range(n)])
        el = (ctypes.c_void_p * n)(*[None if e_loc is None or e_loc[i] is None else e_loc[i].data_ptr()
                                     for i in range(n)])
        em = (ctypes.c_void_p * n)(*[None if e_mix is None or e_mix[i] is None else e_mix[i].data_ptr()
                                     for i in range(n)])
        dev = self.contexts[0].device
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        L.check(L.lib().afqmc_batch_step(self._h, ws, fp, ps, el, em, s.cuda_stream), "afqmc_batch_step")

    def close(self):
        if getattr(self, "_h", None):
            L.lib().afqmc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MixedEnergy(torch.autograd.Function):
    """E_k(h1, L) at fixed walkers as a differentiable function: the forward
    runs afqmc_local_energy on a context built from (h1, L), the backward
    afqmc_energy_backward.  Inputs: h1 [N,N] and L [G,N,N] float64 tensors;
    `walkers` a dict with psi [Nw, nc, N] complex128, weight [Nw], logovl
    [Nw, 2] on the device; trial [N, nc]; na, nb; e0; tau."""

    @staticmethod
    def forward(ctx, h1, chol, walkers, trial, na, nb, e0, tau):
        c = Context(h1.detach().cpu().numpy(), chol.detach().cpu().numpy(), trial, na, nb, precision="fp64",
                    device=walkers["psi"].device)
        w = WalkerSet(walkers["psi"], walkers["weight"], walkers["logovl"],
                      torch.zeros(walkers["psi"].shape[0], dtype=torch.int32, device=walkers["psi"].device))
        _, e_mix = c.local_energy(w, e0, tau)
        ctx.state = (c, w, e0, tau)
        return e_mix[2].detach().to(h1.device)

    @staticmethod
    def backward(ctx, grad_out):
        c, w, e0, tau = ctx.state
        gh, gL = c.energy_backward(w, e0, tau, float(grad_out))
        return gh.to(grad_out.device), gL.to(grad_out.device), None, None, None, None, None, None


def walk_energy(ctx: "Context", n_walkers: int, fields: torch.Tensor, tau: float, e0: float, order: int = 6,
                reortho_every: int = 0, expm: str = "taylor") -> torch.Tensor:
    """J = E_n after n fixed-field steps (Split-2 + Taylor of the given order,
    or Krylov of that dimension) from walkers at the trial, by plain
    afqmc_step calls with the local energy measured at the last step.
    Returns e_mix [4] = (sum W Ebar_L, sum W, J, live walkers)."""
    w = ctx.new_walkers(n_walkers)
    ctx.init_walkers(w)
    e_loc = torch.empty(n_walkers, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    n = int(fields.shape[0])
    for k in range(n):
        ctx.step(w, fields[k], tau, e0, expm=expm, order=order,
                 reortho=bool(reortho_every) and (k + 1) % reortho_every == 0, measure=(k == n - 1),
                 e_loc=e_loc, e_mix=e_mix)
    return e_mix


class WalkEnergy(torch.autograd.Function):
    """J(h1, L) = E_n, the mixed estimator after an n-step fixed-field walk
    from walkers at the trial, as a differentiable function (the energy
    derivatives of a bond-length scan).  The forward is the walk itself
    (afqmc_step, Split-2 + Taylor of the given order or Krylov (Arnoldi or
    Lanczos) of that dimension, re-orthonormalisation every reortho_every steps); the
    backward is afqmc_walk_backward on a
    context built from the same (h1, L), which recomputes the walk from
    checkpoints every ckpt_every steps and returns dJ/dh1 and dJ/dL scaled by
    the incoming gradient.  The auxiliary fields, the trial, e0 and tau are
    fixed inputs (no gradient).

    apply(h1 [N,N] float64, L [G,N,N] float64, fields [n, Nw, G] float64 on
          the device, trial [N, na+nb], na, nb, e0, tau, order, reortho_every,
          ckpt_every, precision ("fp64" or "mixed"), e_const, expm ("taylor",
          "krylov" or "lanczos")) -> J (0-dim)"""

    @staticmethod
    def forward(ctx, h1, chol, fields, trial, na, nb, e0, tau, order=6, reortho_every=0, ckpt_every=10,
                precision="fp64", e_const=0.0, expm="taylor"):
        dev = fields.device
        c = Context(h1.detach().cpu().numpy(), chol.detach().cpu().numpy(), trial, na, nb, e_const,
                    precision=precision, device=dev)
        try:
            e_mix = walk_energy(c, int(fields.shape[1]), fields, tau, e0, order, reortho_every, expm)
            J = e_mix[2].clone()
            torch.cuda.synchronize(dev)
        finally:
            c.close()
        ctx.args = (h1.detach(), chol.detach(), fields, trial, na, nb, e0, tau, order, reortho_every, ckpt_every,
                    precision, e_const, expm)
        return J.to(h1.device)

    @staticmethod
    def backward(ctx, grad_out):
        h1, chol, fields, trial, na, nb, e0, tau, order, r, ckpt, precision, e_const, expm = ctx.args
        dev = fields.device
        c = Context(h1.cpu().numpy(), chol.cpu().numpy(), trial, na, nb, e_const, precision=precision, device=dev)
        try:
            w = c.new_walkers(int(fields.shape[1]))
            c.init_walkers(w)
            _, gh, gL = c.walk_backward(w, fields, tau, e0, order=order, reortho_every=r, ckpt_every=ckpt,
                                        dJ=float(grad_out), expm=expm)
            torch.cuda.synchronize(dev)
        finally:
            c.close()
        return (gh.to(h1.device), gL.to(chol.device)) + (None,) * 12

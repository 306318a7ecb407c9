"""Adjoint of the fixed-field walk (afqmc_walk_backward) against torch
autograd through the CPU oracle's walk (oracle.walk_objective, reading R10),
against central differences of the GPU forward, and for the invariances the
method fixes: checkpoint spacing does not change a bit of the result, and the
gradient with respect to the initial walkers is orthogonal to their gauge
directions.  Gradients are compared symmetrised (the derivative along
symmetric perturbations, which is what the library returns)."""
import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import config_system, make_fields, make_system, CONFIGS

pytestmark = pytest.mark.gpu
CT, RT = torch.complex128, torch.float64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


class _Sys:
    """Closed-shell synthetic system with the trial cut to na alpha, nb beta orbitals."""

    def __init__(self, N, na, nb, G, seed):
        base = make_system(N, na, na, G, rho=0.8, seed=seed)
        self.h1, self.L, self.e_const = base.h1, base.L, base.e_const
        self.trial = np.concatenate([base.trial[:, :na], base.trial[:, na:na + nb]], axis=1)
        self.na, self.nb, self.N, self.G = na, nb, N, G


def _sym(x):
    return 0.5 * (x + x.transpose(-1, -2))


def _e0(s):
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb, s.e_const)
    return float(R.local_energy(ham, ham.trial.to(CT)).real)


def _gpu(s, nw, fields, tau, e0, order, r, ckpt, dead=(), psi_grad=False, h1=None, L=None, precision="fp64",
         expm="taylor"):
    from paper_2403_02542_gb300.api import Context
    ctx = Context(s.h1 if h1 is None else h1, s.L if L is None else L, s.trial, s.na, s.nb, s.e_const,
                  precision=precision)
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    for d in dead:
        w.weight[d] = 0.0
    f = torch.as_tensor(np.stack(fields), device=ctx.device)
    out = ctx.walk_backward(w, f, tau, e0, order=order, reortho_every=r, ckpt_every=ckpt, grad_psi0=psi_grad,
                            expm=expm)
    torch.cuda.synchronize()
    # the initial walkers are left unchanged
    assert torch.all(w.weight.cpu()[list(set(range(nw)) - set(dead))] == 1.0)
    res = [t.cpu() for t in out]
    ctx.close()
    return res


def _plain_J(s, nw, fields, tau, e0, order, r, h1=None, L=None):
    """J after the walk by plain afqmc_step calls (E_L measured at the last step)."""
    from paper_2403_02542_gb300.api import Context
    ctx = Context(s.h1 if h1 is None else h1, s.L if L is None else L, s.trial, s.na, s.nb, s.e_const,
                  precision="fp64")
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    e_loc = torch.empty(nw, 2, dtype=RT, device=ctx.device)
    e_mix = torch.empty(4, dtype=RT, device=ctx.device)
    n = len(fields)
    for k, x in enumerate(fields):
        ctx.step(w, torch.as_tensor(x, device=ctx.device), tau, e0, expm="taylor", order=order,
                 reortho=bool(r) and (k + 1) % r == 0, measure=(k == n - 1), e_loc=e_loc, e_mix=e_mix)
    v = float(e_mix[2])
    ctx.close()
    return v


def _oracle(s, nw, fields, tau, e0, order, r, dead=(), method="taylor"):
    h1 = torch.tensor(s.h1, dtype=RT, requires_grad=True)
    L = torch.tensor(s.L, dtype=RT, requires_grad=True)
    ham = R.Hamiltonian(h1, L, torch.as_tensor(s.trial, dtype=RT), s.na, s.nb, s.e_const)
    psi0 = torch.as_tensor(s.trial, dtype=RT).to(CT).unsqueeze(0).repeat(nw, 1, 1).requires_grad_(True)
    W0 = torch.ones(nw, dtype=RT)
    for d in dead:
        W0[d] = 0.0
    J, W, _ = R.walk_objective(ham, psi0, W0, fields, tau, e0, k=order, reortho_every=r, method=method)
    gh, gL, gp = torch.autograd.grad(J, [h1, L, psi0])
    return float(J), _sym(gh), _sym(gL), gp.conj(), W


def _close(a, b, rtol):
    scale = float(b.abs().max())
    err = float((a - b).abs().max())
    assert err <= rtol * max(scale, 1e-300), (err, scale)


# FP64 gradient bar, entry by entry: |a - b| <= 1e-10 |b| + 1e-14 max|b|.  The
# absolute floor covers entries that are small because their terms cancel:
# such an entry is a sum of terms as large as the largest entry, added in a
# different order by the oracle's autograd and the hand-written reverse pass,
# so its rounding is a few 1e-16 of the largest entry times the growth over
# the steps, whatever its own size.
GRAD_RTOL, GRAD_FLOOR = 1e-10, 1e-14


def _close_entrywise(a, b, what=""):
    a = a.to(torch.complex128) if a.is_complex() else a
    scale = float(b.abs().max())
    d = (a - b).abs()
    bound = GRAD_RTOL * b.abs() + GRAD_FLOOR * scale
    big = b.abs() >= 1e-6 * scale
    worst_rel = float((d[big] / b.abs()[big]).max()) if bool(big.any()) else 0.0
    print(f"{what}: worst relative error {worst_rel:.2e} over entries >= 1e-6 of the largest; "
          f"worst error / largest entry {float(d.max()) / max(scale, 1e-300):.2e}")
    assert bool((d <= bound).all()), (what, float((d - bound).max()), scale)


@pytest.mark.parametrize("N,na,nb,G,nw,steps,r,ckpt,dead", [
    (10, 2, 2, 12, 5, 6, 2, 3, (1,)),
    (14, 3, 2, 20, 6, 7, 3, 2, ()),
    (24, 3, 3, 40, 4, 5, 0, 10, (3,)),
    (12, 2, 0, 16, 3, 4, 1, 1, ()),
])
def test_walk_adjoint_matches_oracle_autograd(N, na, nb, G, nw, steps, r, ckpt, dead):
    s = _Sys(N, na, nb, G, seed=N + steps)
    tau, order = 0.05, 6
    e0 = _e0(s)
    fields = [make_fields(N, k, nw, G) for k in range(steps)]
    J_ref, gh_ref, gL_ref, gp_ref, W_ref = _oracle(s, nw, fields, tau, e0, order, r, dead)
    assert int((W_ref > 0).sum()) == nw - len(dead)   # no walker killed on the way
    J, gh, gL, gp = _gpu(s, nw, fields, tau, e0, order, r, ckpt, dead, psi_grad=True)
    assert abs(float(J[2]) - J_ref) <= 1e-10 * abs(J_ref)
    _close_entrywise(gh, gh_ref, "dJ/dh1")
    _close_entrywise(gL, gL_ref, "dJ/dL")
    _close_entrywise(gp, gp_ref.transpose(1, 2), "dJ/dPsi0")
    assert torch.equal(gh, gh.T) and torch.equal(gL, gL.transpose(1, 2))


@pytest.mark.parametrize("N,na,nb,G,nw,steps,r,ckpt,dead,k", [
    (10, 2, 2, 12, 5, 6, 2, 3, (1,), 6),
    (14, 3, 2, 20, 6, 5, 3, 2, (), 10),
    (10, 2, 1, 12, 3, 4, 0, 10, (), 12),     # dimension above N: the whole space, k = N
    (24, 3, 3, 40, 4, 4, 1, 1, (2,), 4),
])
def test_walk_adjoint_krylov_matches_oracle_autograd(N, na, nb, G, nw, steps, r, ckpt, dead, k):
    """The Krylov action of Eqs. krylovsub-krylov in every step: FP64
    gradients entry by entry against autograd through the oracle's Arnoldi
    steps, norms and small exponential (torch.linalg.matrix_exp)."""
    s = _Sys(N, na, nb, G, seed=3 * N + steps)
    tau = 0.05
    e0 = _e0(s)
    fields = [make_fields(N, 50 + kk, nw, G) for kk in range(steps)]
    J_ref, gh_ref, gL_ref, gp_ref, W_ref = _oracle(s, nw, fields, tau, e0, k, r, dead, method="krylov")
    assert int((W_ref > 0).sum()) == nw - len(dead)
    J, gh, gL, gp = _gpu(s, nw, fields, tau, e0, k, r, ckpt, dead, psi_grad=True, expm="krylov")
    assert abs(float(J[2]) - J_ref) <= 1e-10 * abs(J_ref)
    _close_entrywise(gh, gh_ref, "dJ/dh1")
    _close_entrywise(gL, gL_ref, "dJ/dL")
    _close_entrywise(gp, gp_ref.transpose(1, 2), "dJ/dPsi0")
    assert torch.equal(gh, gh.T) and torch.equal(gL, gL.transpose(1, 2))


@pytest.mark.parametrize("N,na,nb,G,nw,steps,r,ckpt,dead,k", [
    (10, 2, 2, 12, 5, 6, 2, 3, (1,), 6),
    (24, 3, 3, 40, 4, 4, 1, 2, (), 8),
])
def test_walk_adjoint_krylov_mixed_matches_oracle_autograd(N, na, nb, G, nw, steps, r, ckpt, dead, k):
    s = _Sys(N, na, nb, G, seed=3 * N + steps)
    tau = 0.05
    e0 = _e0(s)
    fields = [make_fields(N, 50 + kk, nw, G) for kk in range(steps)]
    J_ref, gh_ref, gL_ref, gp_ref, W_ref = _oracle(s, nw, fields, tau, e0, k, r, dead, method="krylov")
    assert int((W_ref > 0).sum()) == nw - len(dead)
    J, gh, gL, gp = _gpu(s, nw, fields, tau, e0, k, r, ckpt, dead, psi_grad=True, precision="mixed",
                         expm="krylov")
    assert gp.dtype == torch.complex64
    assert abs(float(J[2]) - J_ref) <= MIXED_J_TOL
    _close(gh, gh_ref, MIXED_GRAD_RTOL)
    _close(gL, gL_ref, MIXED_GRAD_RTOL)
    _close(gp.to(CT), gp_ref.transpose(1, 2), MIXED_GRAD_RTOL)


def test_walk_adjoint_krylov_is_independent_of_checkpoint_spacing():
    """Recomputing the Arnoldi steps from checkpoints changes no bit."""
    s = _Sys(14, 3, 2, 20, seed=1401)
    tau, nw, steps, k = 0.05, 6, 6, 8
    e0 = _e0(s)
    fields = [make_fields(14, 70 + kk, nw, s.G) for kk in range(steps)]
    a = _gpu(s, nw, fields, tau, e0, k, 2, 1, psi_grad=True, expm="krylov")
    b = _gpu(s, nw, fields, tau, e0, k, 2, 4, psi_grad=True, expm="krylov")
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("N,na,nb,G,nw,steps,r,ckpt,dead,k", [
    (10, 2, 2, 12, 5, 6, 2, 3, (1,), 4),
    (14, 3, 2, 20, 6, 5, 3, 2, (), 10),
    (10, 2, 1, 12, 3, 4, 0, 10, (), 12),     # dimension above N: k = N
    (24, 3, 3, 40, 4, 4, 1, 1, (2,), 5),
])
def test_walk_adjoint_lanczos_matches_oracle_autograd(N, na, nb, G, nw, steps, r, ckpt, dead, k):
    """The complex-symmetric Lanczos action in every step: FP64 gradients
    entry by entry against autograd through the oracle's three-term
    recurrence (bilinear forms, principal square roots) and small
    exponential.  In the first case the Lanczos gradient differs from the
    Arnoldi one by far more than the bar, so the comparison sees which
    reverse pass ran."""
    s = _Sys(N, na, nb, G, seed=5 * N + steps)
    tau = 0.05
    e0 = _e0(s)
    fields = [make_fields(N, 90 + kk, nw, G) for kk in range(steps)]
    J_ref, gh_ref, gL_ref, gp_ref, W_ref = _oracle(s, nw, fields, tau, e0, k, r, dead, method="lanczos")
    assert int((W_ref > 0).sum()) == nw - len(dead)
    J, gh, gL, gp = _gpu(s, nw, fields, tau, e0, k, r, ckpt, dead, psi_grad=True, expm="lanczos")
    assert abs(float(J[2]) - J_ref) <= 1e-10 * abs(J_ref)
    _close_entrywise(gh, gh_ref, "dJ/dh1")
    _close_entrywise(gL, gL_ref, "dJ/dL")
    _close_entrywise(gp, gp_ref.transpose(1, 2), "dJ/dPsi0")
    assert torch.equal(gh, gh.T) and torch.equal(gL, gL.transpose(1, 2))
    if k == 4:
        _, gh_a, _, _, _ = _oracle(s, nw, fields, tau, e0, k, r, dead, method="krylov")
        assert float((gh_a - gh_ref).abs().max()) > 1e3 * GRAD_RTOL * float(gh_ref.abs().max())


def test_walk_adjoint_lanczos_is_independent_of_checkpoint_spacing():
    """Recomputing the Lanczos steps from checkpoints changes no bit."""
    s = _Sys(14, 3, 2, 20, seed=1402)
    tau, nw, steps, k = 0.05, 6, 6, 8
    e0 = _e0(s)
    fields = [make_fields(14, 170 + kk, nw, s.G) for kk in range(steps)]
    a = _gpu(s, nw, fields, tau, e0, k, 2, 1, psi_grad=True, expm="lanczos")
    b = _gpu(s, nw, fields, tau, e0, k, 2, 4, psi_grad=True, expm="lanczos")
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_walk_adjoint_matches_oracle_autograd_mid_size():
    """N = 48, 8+8 electrons, 160 vectors, 16 walkers, 10 steps, QR every 5,
    checkpoints every 5: FP64 gradients entry by entry against autograd
    through the oracle's walk."""
    s = _Sys(48, 8, 8, 160, seed=4810)
    tau, order, nw, steps, r = 0.05, 6, 16, 10, 5
    e0 = _e0(s)
    fields = [make_fields(48, k, nw, s.G) for k in range(steps)]
    J_ref, gh_ref, gL_ref, gp_ref, W_ref = _oracle(s, nw, fields, tau, e0, order, r)
    assert int((W_ref > 0).sum()) == nw
    J, gh, gL, gp = _gpu(s, nw, fields, tau, e0, order, r, 5, psi_grad=True)
    assert abs(float(J[2]) - J_ref) <= 1e-10 * abs(J_ref)
    _close_entrywise(gh, gh_ref, "dJ/dh1")
    _close_entrywise(gL, gL_ref, "dJ/dL")
    _close_entrywise(gp, gp_ref.transpose(1, 2), "dJ/dPsi0")


def test_walk_adjoint_is_independent_of_checkpoint_spacing():
    s = _Sys(12, 2, 2, 18, seed=5)
    tau, nw, steps = 0.05, 5, 8
    e0 = _e0(s)
    fields = [make_fields(7, k, nw, s.G) for k in range(steps)]
    ref = _gpu(s, nw, fields, tau, e0, 6, 3, steps, psi_grad=True)
    for ckpt in (1, 3):
        got = _gpu(s, nw, fields, tau, e0, 6, 3, ckpt, psi_grad=True)
        for a, b in zip(got, ref):
            assert torch.equal(a, b), ckpt


def test_walk_adjoint_gauge_invariance():
    """J(Psi_0 M) = J(Psi_0): the derivative G with respect to the initial
    orbitals satisfies Psi_0,s^T G_s = 0 for each spin block."""
    s = _Sys(16, 3, 2, 24, seed=9)
    tau, nw, steps = 0.05, 6, 6
    e0 = _e0(s)
    fields = [make_fields(3, k, nw, s.G) for k in range(steps)]
    _, _, _, gp = _gpu(s, nw, fields, tau, e0, 6, 2, 2, psi_grad=True)
    psi0 = torch.as_tensor(s.trial, dtype=RT).to(CT)          # [N, nc]
    G = gp.transpose(1, 2)                                     # [nw, N, nc]
    for sl in (slice(0, 3), slice(3, 5)):
        Z = psi0[:, sl].T.unsqueeze(0) @ G[:, :, sl]
        assert float(Z.abs().max()) <= 1e-11 * float(G.abs().max()) * 100


def test_walk_adjoint_central_differences():
    """Directional derivatives along random symmetric dH1, dL (h = 1e-5) of the
    GPU forward value J against the GPU gradient."""
    s = _Sys(20, 3, 3, 30, seed=4)
    tau, nw, steps, r = 0.05, 8, 6, 2
    e0 = _e0(s)
    fields = [make_fields(11, k, nw, s.G) for k in range(steps)]
    _, gh, gL = _gpu(s, nw, fields, tau, e0, 6, r, 3)
    rng = np.random.default_rng(2)
    dH = rng.standard_normal(s.h1.shape); dH = 0.5 * (dH + dH.T)
    dL = rng.standard_normal(s.L.shape); dL = 0.5 * (dL + dL.transpose(0, 2, 1))
    eps = 1e-5

    def J(h1, L):
        return _plain_J(s, nw, fields, tau, e0, 6, r, h1=h1, L=L)

    fd_h = (J(s.h1 + eps * dH, s.L) - J(s.h1 - eps * dH, s.L)) / (2 * eps)
    fd_L = (J(s.h1, s.L + eps * dL) - J(s.h1, s.L - eps * dL)) / (2 * eps)
    assert abs(fd_h - float((gh.numpy() * dH).sum())) <= 1e-6 * max(1.0, abs(fd_h))
    assert abs(fd_L - float((gL.numpy() * dL).sum())) <= 1e-6 * max(1.0, abs(fd_L))


def test_walk_adjoint_full_size_directional_derivative():
    """The differentiation workload at full size (N=96, 15+15 electrons, 480
    vectors, 512 walkers, 100 steps, Taylor-6, QR every 10 steps, checkpoints
    every 10): the gradient against a central difference of J along one random
    symmetric direction of h1 and of L."""
    cfg = CONFIGS["grad"]
    s = config_system("grad")
    tau, nw, steps = cfg["tau"], cfg["walkers"], cfg["steps"]
    e0 = _e0(s)
    fields = [make_fields(2024, k, nw, s.G) for k in range(steps)]
    Jv, gh, gL = _gpu(s, nw, fields, tau, e0, cfg["order"], cfg["reortho"], 10)
    assert float(Jv[3]) > 0.5 * nw
    assert abs(float(Jv[2]) - _plain_J(s, nw, fields, tau, e0, cfg["order"], cfg["reortho"])) <= 1e-13 * abs(
        float(Jv[2]))
    rng = np.random.default_rng(6)
    dH = rng.standard_normal(s.h1.shape); dH = 0.5 * (dH + dH.T)
    dL = rng.standard_normal(s.L.shape); dL = 0.5 * (dL + dL.transpose(0, 2, 1))
    dH *= 1e-2 / np.abs(dH).max()
    dL *= 1e-2 * np.abs(s.L).max() / np.abs(dL).max()
    eps = 1e-5

    def J(h1, L):
        return _plain_J(s, nw, fields, tau, e0, cfg["order"], cfg["reortho"], h1=h1, L=L)

    fd = (J(s.h1 + eps * dH, s.L + eps * dL) - J(s.h1 - eps * dH, s.L - eps * dL)) / (2 * eps)
    an = float((gh.numpy() * dH).sum() + (gL.numpy() * dL).sum())
    assert abs(fd - an) <= 1e-5 * max(abs(fd), 1e-3), (fd, an)


def test_walk_adjoint_argument_checks():
    from paper_2403_02542_gb300 import _lib as Lb
    from paper_2403_02542_gb300.api import Context
    s = _Sys(8, 1, 1, 6, seed=1)
    ctx = Context(s.h1, s.L, s.trial, 1, 1, precision="fp64")
    w = ctx.new_walkers(2)
    ctx.init_walkers(w)
    f = torch.zeros(2, 2, s.G, dtype=RT, device=ctx.device)
    with pytest.raises(Lb.AfqmcError):
        ctx.walk_backward(w, f, 0.05, -1.0, order=0)
    with pytest.raises(Lb.AfqmcError):
        ctx.walk_backward(w, f, -0.05, -1.0)
    with pytest.raises(Lb.AfqmcError):
        ctx.walk_backward(w, f, 0.05, -1.0, ckpt_every=0)
    mixed = Context(s.h1, s.L, s.trial, 1, 1, precision="mixed")
    wm = mixed.new_walkers(2)
    mixed.init_walkers(wm)
    with pytest.raises(Lb.AfqmcError):
        mixed.walk_backward(wm, f, 0.05, -1.0, order=33)
    J, gh, gL, gp = mixed.walk_backward(wm, f, 0.05, -1.0, grad_psi0=True)
    assert gp.dtype == torch.complex64 and gh.dtype == RT and gL.shape == (s.G, 8, 8)
    assert bool(torch.isfinite(gh).all()) and bool(torch.isfinite(gL).all())
    mixed.close()
    e = ctx.new_walkers(0)
    J, gh, gL = ctx.walk_backward(e, torch.zeros(2, 0, s.G, dtype=RT, device=ctx.device), 0.05, -1.0)
    assert torch.all(gh == 0) and torch.all(gL == 0)


# ---------------------------------------------------------------- mixed precision
# Complex64 walkers: the walk and its reverse run with FP32 contractions (the
# step's own tensor-core field and Taylor products forward, SIMT FP32 in the
# recomputed steps and the reverse), FP64 overlaps, determinants, weights and
# gradient sums.  Tolerances: J is an energy and takes the mixed energy bar
# (1e-4 Ha); a gradient entry carries the FP32 relative rounding of the
# contractions it passes through (about 6e-8 times a growth factor of a few
# hundred over the Taylor terms, steps and walker sums), so 1e-4 of the
# largest entry bounds it with room, and 3e-6 of the largest entry is far
# below any sign or index mistake, which would change entries at O(1).

MIXED_J_TOL = 1e-4        # Ha
MIXED_GRAD_RTOL = 1e-4    # of the largest entry


@pytest.mark.parametrize("N,na,nb,G,nw,steps,r,ckpt,dead", [
    (10, 2, 2, 12, 5, 6, 2, 3, (1,)),
    (14, 3, 2, 20, 6, 7, 3, 2, ()),
    (24, 3, 3, 40, 4, 5, 0, 10, (3,)),
    (12, 2, 0, 16, 3, 4, 1, 1, ()),
])
def test_walk_adjoint_mixed_matches_oracle_autograd(N, na, nb, G, nw, steps, r, ckpt, dead):
    s = _Sys(N, na, nb, G, seed=N + steps)
    tau, order = 0.05, 6
    e0 = _e0(s)
    fields = [make_fields(N, k, nw, G) for k in range(steps)]
    J_ref, gh_ref, gL_ref, gp_ref, W_ref = _oracle(s, nw, fields, tau, e0, order, r, dead)
    assert int((W_ref > 0).sum()) == nw - len(dead)
    J, gh, gL, gp = _gpu(s, nw, fields, tau, e0, order, r, ckpt, dead, psi_grad=True, precision="mixed")
    assert gp.dtype == torch.complex64
    assert abs(float(J[2]) - J_ref) <= MIXED_J_TOL
    _close(gh, gh_ref, MIXED_GRAD_RTOL)
    _close(gL, gL_ref, MIXED_GRAD_RTOL)
    _close(gp.to(CT), gp_ref.transpose(1, 2), MIXED_GRAD_RTOL)
    assert torch.equal(gh, gh.T) and torch.equal(gL, gL.transpose(1, 2))


@pytest.mark.parametrize("N,na,nb,G,nw,steps,r,ckpt,dead,k", [
    (10, 2, 2, 12, 5, 6, 2, 3, (1,), 6),
    (24, 3, 3, 40, 4, 4, 1, 2, (), 8),
])
def test_walk_adjoint_lanczos_mixed_matches_oracle_autograd(N, na, nb, G, nw, steps, r, ckpt, dead, k):
    """Complex64 walkers with the Lanczos action: the recurrence's scalars in
    FP32 forward and reverse, the gradient sums in FP64."""
    s = _Sys(N, na, nb, G, seed=5 * N + steps)
    tau = 0.05
    e0 = _e0(s)
    fields = [make_fields(N, 90 + kk, nw, G) for kk in range(steps)]
    J_ref, gh_ref, gL_ref, gp_ref, W_ref = _oracle(s, nw, fields, tau, e0, k, r, dead, method="lanczos")
    assert int((W_ref > 0).sum()) == nw - len(dead)
    J, gh, gL, gp = _gpu(s, nw, fields, tau, e0, k, r, ckpt, dead, psi_grad=True, precision="mixed",
                         expm="lanczos")
    assert gp.dtype == torch.complex64
    assert abs(float(J[2]) - J_ref) <= MIXED_J_TOL
    _close(gh, gh_ref, MIXED_GRAD_RTOL)
    _close(gL, gL_ref, MIXED_GRAD_RTOL)
    _close(gp.to(CT), gp_ref.transpose(1, 2), MIXED_GRAD_RTOL)


def test_walk_adjoint_mixed_is_independent_of_checkpoint_spacing():
    """The recomputed segments replay the same deterministic complex64 steps,
    so the checkpoint spacing changes no bit of the mixed result either."""
    s = _Sys(12, 2, 2, 18, seed=5)
    tau, nw, steps = 0.05, 5, 8
    e0 = _e0(s)
    fields = [make_fields(7, k, nw, s.G) for k in range(steps)]
    ref = _gpu(s, nw, fields, tau, e0, 6, 3, steps, psi_grad=True, precision="mixed")
    for ckpt in (1, 3):
        got = _gpu(s, nw, fields, tau, e0, 6, 3, ckpt, psi_grad=True, precision="mixed")
        for a, b in zip(got, ref):
            assert torch.equal(a, b), ckpt


def test_walk_adjoint_mixed_full_size_against_fp64():
    """The differentiation workload at full size (N=96, 15+15 electrons, 480
    vectors, 512 walkers, 100 steps, Taylor-6, QR every 10 steps): the mixed
    J and gradients against the FP64 ones (pinned to autograd through the
    oracle and to central differences above), entry by entry."""
    cfg = CONFIGS["grad"]
    s = config_system("grad")
    tau, nw, steps = cfg["tau"], cfg["walkers"], cfg["steps"]
    e0 = _e0(s)
    fields = [make_fields(2024, k, nw, s.G) for k in range(steps)]
    J64, gh64, gL64 = _gpu(s, nw, fields, tau, e0, cfg["order"], cfg["reortho"], 10)
    J32, gh32, gL32 = _gpu(s, nw, fields, tau, e0, cfg["order"], cfg["reortho"], 10, precision="mixed")
    assert float(J32[3]) == float(J64[3])
    assert abs(float(J32[2]) - float(J64[2])) <= MIXED_J_TOL
    _close(gh32, gh64, MIXED_GRAD_RTOL)
    _close(gL32, gL64, MIXED_GRAD_RTOL)


def test_walk_energy_autograd_function_matches_the_oracle():
    """WalkEnergy: forward = the walk through afqmc_step, backward =
    afqmc_walk_backward.  J and the gradients that torch autograd returns
    through it equal the oracle's walk objective and its autograd gradients
    (FP64, entry by entry at the FP64 gradient bar)."""
    from paper_2403_02542_gb300.api import WalkEnergy
    s = _Sys(12, 2, 2, 16, seed=31)
    tau, order, nw, steps, r = 0.05, 6, 6, 6, 2
    e0 = _e0(s)
    fields = [make_fields(31, k, nw, s.G) for k in range(steps)]
    J_ref, gh_ref, gL_ref, _, W_ref = _oracle(s, nw, fields, tau, e0, order, r)
    assert int((W_ref > 0).sum()) == nw
    h1 = torch.tensor(s.h1, dtype=RT, requires_grad=True)
    L = torch.tensor(s.L, dtype=RT, requires_grad=True)
    f = torch.as_tensor(np.stack(fields), device="cuda")
    J = WalkEnergy.apply(h1, L, f, s.trial, s.na, s.nb, e0, tau, order, r, 2, "fp64", s.e_const)
    assert abs(float(J) - J_ref) <= 1e-10 * abs(J_ref)
    gh, gL = torch.autograd.grad(J, [h1, L])
    _close_entrywise(gh.cpu(), gh_ref, "WalkEnergy dJ/dh1")
    _close_entrywise(gL.cpu(), gL_ref, "WalkEnergy dJ/dL")
    # the incoming gradient scales the result
    J2 = WalkEnergy.apply(h1, L, f, s.trial, s.na, s.nb, e0, tau, order, r, 2, "fp64", s.e_const)
    gh2, = torch.autograd.grad(3.0 * J2, [h1])
    assert torch.allclose(gh2, 3.0 * gh, rtol=1e-14, atol=0.0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("mixed", 2e-3)])
def test_path_scan_derivative_against_central_differences(precision, tol):
    """A three-point scan h1(s) = h1 + s dH1, L(s) = L + s dL: the adjoint
    derivative dJ/ds at every point against central differences of J(s)
    (FP64: 1e-6 relative; mixed: FP32 noise in J over the step 1e-2 bounds
    the difference, 2e-3 of max(|dJ/ds|, 1))."""
    from paper_2403_02542_gb300.scan import path_scan
    s = _Sys(16, 3, 3, 24, seed=41)
    tau, order, nw, steps, r = 0.05, 6, 8, 6, 3
    e0 = _e0(s)
    rng = np.random.default_rng(41)
    dH = rng.standard_normal(s.h1.shape); dH = 0.01 * (dH + dH.T)
    dL = rng.standard_normal(s.L.shape); dL = 0.01 * np.abs(s.L).max() * (dL + dL.transpose(0, 2, 1))
    f = torch.as_tensor(np.stack([make_fields(41, k, nw, s.G) for k in range(steps)]), device="cuda")
    pts = path_scan(s, f, [-0.05, 0.0, 0.05], dH, dL, tau, e0, order=order, reortho_every=r, ckpt_every=3,
                    precision=precision, fd_step=1e-2 if precision == "mixed" else 1e-4)
    for p in pts:
        assert p["live"] == nw
        assert abs(p["dJds"] - p["dJds_fd"]) <= tol * max(abs(p["dJds"]), 1.0), p
    assert len({round(p["J"], 12) for p in pts}) == 3     # the path moves the energy

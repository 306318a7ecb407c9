"""Block-Krylov exponential (Eq. bkrylov, reading R20) of the CUDA library
against the CPU oracle on the same seeded systems and common random fields:
FP64 element by element (1e-10 relative, as the other FP64 parity tests),
complex64 walkers within the mixed energy bar (1e-4 Ha per walker), the
batched graph against plain steps, and the argument checks."""
import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import config_system, make_fields, make_system
from walk_helpers import compare, gpu_walk, oracle_walk

pytestmark = pytest.mark.gpu
RTOL = 1e-10
E_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _e0(s, trial, na, nb):
    ham = R.make_hamiltonian(s.h1, s.L, trial, na, nb)
    return float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)


@pytest.mark.parametrize("N,na,nb,G,nw,steps,k,reo", [
    (12, 2, 2, 16, 5, 4, 3, 2),    # several blocks, QR every 2 steps
    (30, 4, 3, 48, 6, 3, 4, 0),    # unequal spins: different block sizes
    (16, 4, 4, 20, 4, 3, 4, 0),    # k n = N: the block space is the whole space
    (14, 3, 0, 18, 3, 3, 5, 0),    # no beta electrons; k clamped to N / n = 4
    (72, 5, 5, 150, 7, 2, 4, 3),   # several tiles with ragged tails
])
def test_block_krylov_fp64_matches_oracle(N, na, nb, G, nw, steps, k, reo):
    from paper_2403_02542_gb300.api import Context
    nmax = max(na, nb)
    s = make_system(N, nmax, nmax, G, rho=0.8 if G < 100 else 1e-5 ** (1 / G), seed=N * 7 + k)
    trial = np.concatenate([s.trial[:, :na], s.trial[:, :nb]], axis=1)
    tau = 0.05
    e0 = _e0(s, trial, na, nb)
    ref, ties = oracle_walk(s, nw, steps, tau, e0, "bkrylov", k, reo, seed=k + 5, trial=trial, na=na, nb=nb)
    assert ties == 0
    ctx = Context(s.h1, s.L, trial, na, nb, s.e_const, precision="fp64")
    got, _ = gpu_walk(ctx, nw, steps, tau, e0, "bkrylov", k, reo, seed=k + 5)
    for g, r in zip(got, ref):
        compare(g, r, RTOL, what=f"block Krylov k={k} step {g['k']}")
    ctx.close()


@pytest.mark.parametrize("cfg,nw,k", [("large", 6, 4), ("small", 9, 2)])
def test_block_krylov_mixed_step_from_oracle_state(cfg, nw, k):
    """Complex64 walkers: one step from an oracle state (after 2 oracle steps)
    on the large workload (N=128, 20+20, 640 vectors) and the small one."""
    from paper_2403_02542_gb300.api import Context
    s = config_system(cfg)
    tau = 0.05
    e0 = _e0(s, s.trial, s.na, s.nb)
    ref, ties = oracle_walk(s, nw, 3, tau, e0, "bkrylov", k, 0, seed=31)
    assert ties == 0
    state, nxt = ref[1], ref[2]
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="mixed")
    w = ctx.new_walkers(nw)
    w.psi.copy_(state["psi"].transpose(1, 2).to(torch.complex64))
    w.weight.copy_(state["W"])
    w.logovl.copy_(torch.stack([state["lo"].real, state["lo"].imag], 1))
    w.status.zero_()
    x = torch.as_tensor(make_fields(31, 2, nw, s.G), device=ctx.device)
    e_loc = torch.empty(nw, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    ctx.step(w, x, tau, e0, expm="bkrylov", order=k, measure=True, e_loc=e_loc, e_mix=e_mix)
    torch.cuda.synchronize()
    El = torch.complex(e_loc[:, 0], e_loc[:, 1]).cpu()
    live = nxt["W"] > 0
    assert bool(live.all())
    dE = float((El - nxt["El"]).abs().max())
    dW = float(((w.weight.cpu() - nxt["W"]).abs() / nxt["W"]).max())
    g = w.psi.cpu().to(torch.complex128).transpose(1, 2)
    dpsi = float(((g - nxt["psi"]).flatten(1).norm(dim=1) / nxt["psi"].flatten(1).norm(dim=1)).max())
    print(f"block Krylov mixed vs oracle ({cfg}): max|dE_L| = {dE:.2e} Ha, max rel dW = {dW:.2e}, "
          f"max rel dPsi = {dpsi:.2e}")
    assert dE <= E_TOL
    assert dW <= 1e-4 and dpsi <= 1e-4
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_block_krylov_batch_graph_equals_plain_steps(precision):
    from paper_2403_02542_gb300.api import Batch, Context
    systems = [make_system(20, 3, 3, 30, rho=0.8, seed=5), make_system(34, 4, 4, 60, rho=0.9, seed=6)]
    nws = [5, 3]
    tau = 0.05
    e0s = [_e0(s, s.trial, s.na, s.nb) for s in systems]
    plain, batched = [], []
    for i, s in enumerate(systems):
        ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision=precision)
        got, _ = gpu_walk(ctx, nws[i], 3, tau, e0s[i], "bkrylov", 3, 0, seed=40 + i)
        plain.append(got[-1])
        ctx.close()
    ctxs = [Context(s.h1, s.L, s.trial, s.na, s.nb, precision=precision) for s in systems]
    ws = [c.new_walkers(n) for c, n in zip(ctxs, nws)]
    for c, w in zip(ctxs, ws):
        c.init_walkers(w)
    batch = Batch(ctxs)
    for step in range(3):
        fields = [torch.as_tensor(make_fields(40 + i, step, nws[i], systems[i].G), device=ctxs[i].device)
                  for i in range(2)]
        batch.step(ws, fields, tau, e0s, expm="bkrylov", order=3)
    torch.cuda.synchronize()
    for i in range(2):
        g = ws[i].psi.cpu().to(torch.complex128).transpose(1, 2)
        assert torch.equal(g, plain[i]["psi"]), i
        assert torch.equal(ws[i].weight.cpu(), plain[i]["W"]), i
    batch.close()
    for c in ctxs:
        c.close()


def test_block_krylov_argument_checks():
    from paper_2403_02542_gb300 import _lib as Lb
    from paper_2403_02542_gb300.api import Context
    s = make_system(12, 2, 2, 10, rho=0.8, seed=1)
    ctx = Context(s.h1, s.L, s.trial, 2, 2, precision="fp64")
    w = ctx.new_walkers(2)
    ctx.init_walkers(w)
    x = torch.zeros(2, s.G, dtype=torch.float64, device=ctx.device)
    for order in (0, 17):
        with pytest.raises(Lb.AfqmcError):
            ctx.step(w, x, 0.05, -1.0, expm="bkrylov", order=order)
    ctx.close()
    # (k n)^2 + 3 (k n) n entries beyond one block's shared memory
    big = make_system(120, 50, 50, 10, rho=0.8, seed=2)
    ctx = Context(big.h1, big.L, big.trial, 50, 50, precision="mixed")
    w = ctx.new_walkers(1)
    ctx.init_walkers(w)
    x = torch.zeros(1, big.G, dtype=torch.float64, device=ctx.device)
    with pytest.raises(Lb.AfqmcError):
        ctx.step(w, x, 0.05, -1.0, expm="bkrylov", order=3)
    ctx.step(w, x, 0.05, -1.0, expm="bkrylov", order=1)   # one block fits
    ctx.sync()
    ctx.close()

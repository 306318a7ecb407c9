"""Complex-symmetric Lanczos action (reading R30; the Krylov space of Eq.
krylovsub built by the three-term recurrence with the bilinear form u^T v)
in the CUDA library against the CPU oracle on the same seeded systems and
common random fields: FP64 element by element (1e-10 relative, as the other
FP64 parity tests) with the Split-2 and Split-1 propagators, at full
dimension equal to the Arnoldi action, complex64 walkers within the mixed
energy bar (1e-4 Ha per walker), the batched graph bit for bit equal to
plain steps, and the argument checks."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import config_system, make_system
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


def _e0(s):
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb)
    return float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)


@pytest.mark.parametrize("N,na,nb,G,nw,k,reo,prop", [
    (40, 4, 4, 70, 6, 6, 2, "split2"),
    (40, 4, 4, 70, 6, 10, 0, "split1"),
    (72, 5, 5, 150, 5, 8, 1, "split2"),     # several tiles with ragged tails
    (18, 2, 2, 24, 3, 18, 0, "split2"),     # k = N: the whole space
    (14, 3, 1, 20, 4, 20, 0, "split2"),     # k > N is taken as N; uneven spins
    (40, 4, 4, 70, 5, 1, 0, "split2"),      # k = 1: e^{alpha_0} psi
])
def test_lanczos_fp64_matches_oracle(N, na, nb, G, nw, k, reo, prop):
    from paper_2403_02542_gb300.api import Context
    base = make_system(N, na, na, G, rho=0.85 if G < 100 else 1e-5 ** (1 / G), seed=N + k)
    trial = np.concatenate([base.trial[:, :na], base.trial[:, na:na + nb]], axis=1)
    s = dataclasses.replace(base, trial=trial, na=na, nb=nb)
    tau = 0.05
    e0 = _e0(s)
    ref, ties = oracle_walk(s, nw, 3, tau, e0, "lanczos", k, reo, seed=61 + k, propagator=prop)
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    got, _ = gpu_walk(ctx, nw, 3, tau, e0, "lanczos", k, reo, seed=61 + k, propagator=prop)
    for g, r in zip(got, ref):
        compare(g, r, RTOL, what=f"Lanczos k={k} {prop} step {g['k']}")
    ctx.close()


def test_lanczos_equals_arnoldi_at_full_dimension():
    """k = N: both recurrences span the whole space, so the GPU Lanczos and
    Arnoldi steps give the same walkers, weights and energies to 1e-10."""
    from paper_2403_02542_gb300.api import Context
    s = make_system(20, 3, 3, 36, rho=0.85, seed=20)
    e0 = _e0(s)
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    a, _ = gpu_walk(ctx, 5, 3, 0.05, e0, "lanczos", 20, 0, seed=3)
    b, _ = gpu_walk(ctx, 5, 3, 0.05, e0, "krylov", 20, 0, seed=3)
    for x, y in zip(a, b):
        compare(x, y, RTOL, what=f"Lanczos vs Arnoldi step {x['k']}")
    ctx.close()


def test_lanczos_mixed_large_workload_energy():
    """Complex64 walkers on the large workload (N=128, 20+20, 640 vectors,
    tensor-core products): E_L after two Split-2 steps with Lanczos of
    dimension 10 within 1e-4 Ha of the oracle."""
    from paper_2403_02542_gb300.api import Context
    s = config_system("large")
    tau = 0.05
    e0 = _e0(s)
    nw = 4
    ref, ties = oracle_walk(s, nw, 2, tau, e0, "lanczos", 10, 0, seed=63)
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="mixed")
    got, _ = gpu_walk(ctx, nw, 2, tau, e0, "lanczos", 10, 0, seed=63)
    dE = max(float((g["El"] - r["El"]).abs().max()) for g, r in zip(got, ref))
    print(f"Lanczos mixed vs oracle: max|dE_L| = {dE:.2e} Ha")
    assert dE <= E_TOL
    ctx.close()


def test_lanczos_batched_graph_equals_plain_steps():
    import test_batch as TB
    for precision in ("fp64", "mixed"):
        systems = TB._setup(precision)
        got = TB._batch_walk(systems, expm="lanczos")
        ref = TB._eager_walk(systems, expm="lanczos")
        for k in range(TB.STEPS):
            for i in range(len(systems)):
                for a, b in zip(got[k][i]["raw"], ref[k][i]["raw"]):
                    assert torch.equal(a, b), (precision, k, i)
        for (_, _, _, c) in systems:
            c.close()


def test_lanczos_argument_checks():
    from paper_2403_02542_gb300 import _lib as Lb
    from paper_2403_02542_gb300.api import Context
    s = make_system(12, 2, 2, 10, rho=0.8, seed=1)
    ctx = Context(s.h1, s.L, s.trial, 2, 2, precision="fp64")
    w = ctx.new_walkers(2)
    ctx.init_walkers(w)
    x = torch.zeros(2, s.G, dtype=torch.float64, device=ctx.device)
    for order in (0, 33):
        with pytest.raises(Lb.AfqmcError):
            ctx.step(w, x, 0.05, -1.0, expm="lanczos", order=order)
    with pytest.raises(Lb.AfqmcError):
        ctx.step(w, x, 0.05, -1.0, expm="lanczos", order=4, propagator="taylor")
    for expm in ("bkrylov", "chebyshev"):   # the walk adjoint takes taylor, krylov and lanczos
        with pytest.raises(ValueError):
            ctx.walk_backward(w, x[None], 0.05, -1.0, order=4, expm=expm)
    J, gh, gL = ctx.walk_backward(w, x[None], 0.05, -1.0, order=4, expm="lanczos")
    assert bool(torch.isfinite(gh).all()) and bool(torch.isfinite(gL).all())
    ctx.step(w, x, 0.05, -1.0, expm="lanczos", order=32)
    ctx.close()

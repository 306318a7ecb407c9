"""The Split-1 propagator (Sec. III.A: the interaction exponential first, then
the whole one-body step e^{-tau h''} as two half steps), the Taylor
propagator (Sec. III.C: the Taylor series of e^{A - tau h''}, no splitting)
and the Crank-Nicolson propagator (Sec. III.D: (1 - X/2)^{-1} (1 + X/2) with
X = A - tau h'') of the CUDA library against the CPU oracle on the same seeded systems and common
random fields: FP64 element by element (1e-10 relative, as the other FP64
parity tests), complex64 walkers within the mixed energy bar (1e-4 Ha per
walker), and the argument checks."""
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


@pytest.mark.parametrize("expm,order,reo", [("krylov", 8, 2), ("taylor", 6, 0), ("bkrylov", 3, 0)])
def test_split1_fp64_matches_oracle(expm, order, reo):
    from paper_2403_02542_gb300.api import Context
    s = make_system(40, 4, 4, 70, rho=0.85, seed=11)
    tau = 0.05
    e0 = _e0(s)
    ref, ties = oracle_walk(s, 6, 3, tau, e0, expm, order, reo, seed=17, propagator="split1")
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    got, _ = gpu_walk(ctx, 6, 3, tau, e0, expm, order, reo, seed=17, propagator="split1")
    for g, r in zip(got, ref):
        compare(g, r, RTOL, what=f"Split-1 {expm} step {g['k']}")
    # the two propagators differ at this time step
    two, _ = gpu_walk(ctx, 6, 1, tau, e0, expm, order, 0, seed=17)
    assert float((two[0]["psi"] - got[0]["psi"]).abs().max()) > 1e-6
    ctx.close()


def test_split1_mixed_large_workload_energy():
    """Complex64 walkers on the large workload (N=128, 20+20, 640 vectors):
    E_L after two Split-1 steps within 1e-4 Ha of the oracle."""
    from paper_2403_02542_gb300.api import Context
    s = config_system("large")
    tau = 0.05
    e0 = _e0(s)
    nw = 4
    ref, ties = oracle_walk(s, nw, 2, tau, e0, "krylov", 10, 0, seed=23, propagator="split1")
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="mixed")
    got, _ = gpu_walk(ctx, nw, 2, tau, e0, "krylov", 10, 0, seed=23, propagator="split1")
    dE = max(float((g["El"] - r["El"]).abs().max()) for g, r in zip(got, ref))
    print(f"Split-1 mixed vs oracle: max|dE_L| = {dE:.2e} Ha")
    assert dE <= E_TOL
    ctx.close()


@pytest.mark.parametrize("order,reo", [(6, 2), (10, 0)])
def test_taylor_propagator_fp64_matches_oracle(order, reo):
    from paper_2403_02542_gb300.api import Context
    s = make_system(40, 4, 4, 70, rho=0.85, seed=12)
    tau = 0.05
    e0 = _e0(s)
    ref, ties = oracle_walk(s, 6, 3, tau, e0, "taylor", order, reo, seed=19, propagator="taylor")
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    got, _ = gpu_walk(ctx, 6, 3, tau, e0, "taylor", order, reo, seed=19, propagator="taylor")
    for g, r in zip(got, ref):
        compare(g, r, RTOL, what=f"Taylor propagator k={order} step {g['k']}")
    ctx.close()


def test_taylor_propagator_mixed_large_workload_energy():
    """Complex64 walkers on the large workload (N=128, 20+20, 640 vectors):
    E_L after two steps of the Taylor propagator (order 8) within 1e-4 Ha of
    the oracle."""
    from paper_2403_02542_gb300.api import Context
    s = config_system("large")
    tau = 0.05
    e0 = _e0(s)
    nw = 4
    ref, ties = oracle_walk(s, nw, 2, tau, e0, "taylor", 8, 0, seed=29, propagator="taylor")
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="mixed")
    got, _ = gpu_walk(ctx, nw, 2, tau, e0, "taylor", 8, 0, seed=29, propagator="taylor")
    dE = max(float((g["El"] - r["El"]).abs().max()) for g, r in zip(got, ref))
    print(f"Taylor propagator mixed vs oracle: max|dE_L| = {dE:.2e} Ha")
    assert dE <= E_TOL
    ctx.close()


def test_taylor_propagator_needs_the_taylor_action():
    from paper_2403_02542_gb300 import _lib as Lb
    from paper_2403_02542_gb300.api import Context
    s = make_system(12, 2, 2, 10, rho=0.8, seed=1)
    ctx = Context(s.h1, s.L, s.trial, 2, 2, precision="fp64")
    w = ctx.new_walkers(2)
    ctx.init_walkers(w)
    x = torch.zeros(2, s.G, dtype=torch.float64, device=ctx.device)
    for expm in ("krylov", "bkrylov"):
        with pytest.raises(Lb.AfqmcError):
            ctx.step(w, x, 0.05, -1.0, expm=expm, order=4, propagator="taylor")
    ctx.step(w, x, 0.05, -1.0, expm="taylor", order=4, propagator="taylor")
    ctx.sync()
    ctx.close()


@pytest.mark.parametrize("N,n,G,nw,reo", [(40, 4, 70, 6, 2), (72, 5, 150, 5, 0)])
def test_crank_nicolson_fp64_matches_oracle(N, n, G, nw, reo):
    from paper_2403_02542_gb300.api import Context
    s = make_system(N, n, n, G, rho=0.85 if G < 100 else 1e-5 ** (1 / G), seed=N + 3)
    tau = 0.05
    e0 = _e0(s)
    ref, ties = oracle_walk(s, nw, 3, tau, e0, "taylor", 1, reo, seed=53, propagator="cn")
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    got, _ = gpu_walk(ctx, nw, 3, tau, e0, "taylor", 1, reo, seed=53, propagator="cn")
    for g, r in zip(got, ref):
        compare(g, r, RTOL, what=f"Crank-Nicolson N={N} step {g['k']}")
    ctx.close()


def test_crank_nicolson_mixed_large_workload_energy():
    """Complex64 walkers on the large workload (N=128, 20+20, 640 vectors):
    E_L after two Crank-Nicolson steps within 1e-4 Ha of the oracle."""
    from paper_2403_02542_gb300.api import Context
    s = config_system("large")
    tau = 0.05
    e0 = _e0(s)
    nw = 4
    ref, ties = oracle_walk(s, nw, 2, tau, e0, "taylor", 1, 0, seed=59, propagator="cn")
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, precision="mixed")
    got, _ = gpu_walk(ctx, nw, 2, tau, e0, "taylor", 1, 0, seed=59, propagator="cn")
    dE = max(float((g["El"] - r["El"]).abs().max()) for g, r in zip(got, ref))
    print(f"Crank-Nicolson mixed vs oracle: max|dE_L| = {dE:.2e} Ha")
    assert dE <= E_TOL
    ctx.close()

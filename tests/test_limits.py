"""The library at the limits of its C ABI against the CPU oracle: the largest
system afqmc_create accepts (N = 512 orbitals, 80 + 80 electrons), where the
mixed path takes its fallbacks (SIMT exchange for n > 64, SIMT A*V for
2 nc > 240), with the Krylov and Lanczos actions and a re-orthonormalisation;
the walk adjoint's own limit (max(na, nb) <= 64) reported as ENOTSUP; and
empty walker sets, which every entry point accepts without touching them."""
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import make_system
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


@pytest.fixture(scope="module")
def largest():
    s = make_system(512, 80, 80, 24, rho=0.9, seed=512)
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb)
    e0 = float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)
    return s, e0


@pytest.mark.parametrize("expm", ["krylov", "lanczos"])
def test_largest_system_fp64_matches_oracle(largest, expm):
    from paper_2403_02542_gb300.api import Context
    s, e0 = largest
    ref, ties = oracle_walk(s, 2, 2, 0.05, e0, expm, 4, 2, seed=512)
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    got, _ = gpu_walk(ctx, 2, 2, 0.05, e0, expm, 4, 2, seed=512)
    for g, r in zip(got, ref):
        compare(g, r, RTOL, what=f"N=512, 80+80, {expm}, step {g['k']}")
    ctx.close()


def test_largest_system_mixed_energy(largest):
    from paper_2403_02542_gb300.api import Context
    s, e0 = largest
    ref, ties = oracle_walk(s, 2, 2, 0.05, e0, "krylov", 4, 2, seed=512)
    assert ties == 0
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="mixed")
    got, _ = gpu_walk(ctx, 2, 2, 0.05, e0, "krylov", 4, 2, seed=512)
    dE = max(float((g["El"] - r["El"]).abs().max()) for g, r in zip(got, ref))
    print(f"N=512, 80+80, mixed vs oracle: max|dE_L| = {dE:.2e} Ha")
    assert dE <= E_TOL
    ctx.close()


def test_walk_adjoint_limit_is_reported(largest):
    from paper_2403_02542_gb300 import _lib as Lb
    from paper_2403_02542_gb300.api import Context
    s, e0 = largest
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    w = ctx.new_walkers(2)
    ctx.init_walkers(w)
    f = torch.zeros(1, 2, s.G, dtype=torch.float64, device=ctx.device)
    with pytest.raises(Lb.AfqmcError) as exc:
        ctx.walk_backward(w, f, 0.05, e0, order=4)
    assert exc.value.status == Lb.AFQMC_ENOTSUP
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_empty_walker_sets(precision):
    """Zero walkers: steps, energies, population control and both adjoints
    return without launching anything on them; the gradients come back zero."""
    from paper_2403_02542_gb300.api import Context
    s = make_system(16, 2, 2, 20, rho=0.8, seed=16)
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision=precision)
    w = ctx.new_walkers(0)
    ctx.init_walkers(w)
    x = torch.zeros(0, s.G, dtype=torch.float64, device=ctx.device)
    for expm in ("taylor", "krylov", "lanczos", "bkrylov", "chebyshev"):
        ctx.step(w, x, 0.05, -1.0, expm=expm, order=2)
    ctx.local_energy(w, -1.0, 0.05)
    ctx.population_control(w, 0.5)
    gh, gL = ctx.energy_backward(w, -1.0, 0.05)
    assert float(gh.abs().max()) == 0.0 and float(gL.abs().max()) == 0.0
    J, gh, gL = ctx.walk_backward(w, torch.zeros(1, 0, s.G, dtype=torch.float64, device=ctx.device), 0.05, -1.0)
    assert float(gh.abs().max()) == 0.0 and float(gL.abs().max()) == 0.0
    torch.cuda.synchronize()
    ctx.close()

"""Force bias taken from the previous measurement (afqmc_step_params.reuse_bias).

<L_g> = sum_s tr(Lh_gs Theta_s) of the walkers at the start of a step is the
trace the previous local-energy evaluation of the same walkers computed (Theta
is invariant under the re-orthonormalisation in between).  Checks: oracle
parity with the option on (FP64 1e-10, mixed 1e-4 Ha on E_L); agreement with
the recomputed force bias; bit identity with the option off whenever the
stored traces are not valid (no measurement, or a population control in
between); graph replay bit-identical to eager steps."""
import numpy as np
import pytest
import torch

from oracle import afqmc_ref as R
from paper_2403_02542_gb300.inputs import make_fields, make_system
from walk_helpers import compare, gpu_walk, near_ties, oracle_walk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ctx(s, precision):
    from paper_2403_02542_gb300.api import Context
    return Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision=precision)


def _e0(s):
    ham = R.make_hamiltonian(s.h1, s.L, s.trial, s.na, s.nb)
    return float(R.local_energy(ham, ham.trial.to(torch.complex128)).real)


def test_reuse_bias_fp64_matches_oracle():
    s = make_system(24, 3, 3, 40, rho=0.85, seed=31)
    e0, tau, nw, steps = _e0(s), 0.05, 7, 8
    ref, ties = oracle_walk(s, nw, steps, tau, e0, "krylov", 6, 3, seed=77)
    assert ties == 0
    got, _ = gpu_walk(_ctx(s, "fp64"), nw, steps, tau, e0, "krylov", 6, 3, seed=77, reuse_bias=True)
    for g, r in zip(got, ref):
        compare(g, r, 1e-10, what=f"step {g['k']}")


def test_reuse_bias_mixed_matches_oracle():
    s = make_system(32, 4, 4, 60, rho=0.9, seed=32)
    e0, tau, nw, steps = _e0(s), 0.05, 6, 6
    ref, ties = oracle_walk(s, nw, steps, tau, e0, "krylov", 8, 3, seed=78)
    assert ties == 0
    got, _ = gpu_walk(_ctx(s, "mixed"), nw, steps, tau, e0, "krylov", 8, 3, seed=78, reuse_bias=True)
    for g, r in zip(got, ref):
        live = r["W"] > 0
        dE = (g["El"] - r["El"]).abs()[live]
        assert float(dE.max()) <= 1e-4, (g["k"], float(dE.max()))


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_reuse_bias_agrees_with_recomputed_bias(precision, rtol):
    s = make_system(40, 5, 5, 90, rho=0.9, seed=33)
    e0, tau, nw, steps = _e0(s), 0.05, 9, 5
    a, _ = gpu_walk(_ctx(s, precision), nw, steps, tau, e0, "krylov", 8, 2, seed=79, reuse_bias=True)
    b, _ = gpu_walk(_ctx(s, precision), nw, steps, tau, e0, "krylov", 8, 2, seed=79, reuse_bias=False)
    for g, r in zip(a, b):
        compare(g, r, rtol, what=f"{precision} step {g['k']}")


def _run(ctx, w, fields, tau, e0, measure, reuse, pop_after=None):
    e_loc = torch.empty(w.n, 2, dtype=torch.float64, device=ctx.device)
    e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
    out = []
    for k, x in enumerate(fields):
        ctx.step(w, x, tau, e0, expm="krylov", order=6, reortho=(k % 3 == 2), measure=measure[k],
                 e_loc=e_loc, e_mix=e_mix, reuse_bias=reuse)
        if pop_after is not None and k == pop_after:
            ctx.population_control(w, 0.5)
        torch.cuda.synchronize()
        out.append((w.psi.cpu().clone(), w.weight.cpu().clone(), w.logovl.cpu().clone()))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("measure,pop_after", [([False, False, False, False], None), ([True, True], 0)])
def test_reuse_bias_is_inert_without_valid_traces(precision, measure, pop_after):
    """Unmeasured steps, or a population control after the measured step,
    leave nothing to reuse: every step is bit-identical to one without the
    option."""
    s = make_system(20, 3, 3, 30, rho=0.85, seed=34)
    e0, tau, nw = _e0(s), 0.05, 6
    ctx = _ctx(s, precision)
    fields = [torch.as_tensor(make_fields(5, k, nw, s.G), device=ctx.device) for k in range(len(measure))]
    runs = []
    for reuse in (True, False):
        w = ctx.new_walkers(nw)
        ctx.init_walkers(w)
        runs.append(_run(ctx, w, fields, tau, e0, measure, reuse, pop_after))
    for k in range(len(measure)):
        for a, b in zip(runs[0][k], runs[1][k]):
            assert torch.equal(a, b), (precision, k)


def test_reuse_bias_graph_replay_is_bit_identical():
    from paper_2403_02542_gb300.api import Batch
    s = make_system(24, 3, 3, 40, rho=0.85, seed=35)
    e0, tau, nw = _e0(s), 0.05, 5
    res = []
    for graph in (False, True):
        ctx = _ctx(s, "mixed")
        w = ctx.new_walkers(nw)
        ctx.init_walkers(w)
        e_loc = torch.empty(nw, 2, dtype=torch.float64, device=ctx.device)
        e_mix = torch.empty(4, dtype=torch.float64, device=ctx.device)
        x = torch.empty(nw, s.G, dtype=torch.float64, device=ctx.device)
        batch = Batch([ctx]) if graph else None
        out = []
        for k in range(6):
            x.copy_(torch.as_tensor(make_fields(9, k, nw, s.G)))
            if graph:
                batch.step([w], [x], tau, e0, expm="krylov", order=6, reortho=(k % 3 == 2), measure=True,
                           e_loc=[e_loc], e_mix=[e_mix], reuse_bias=True)
            else:
                ctx.step(w, x, tau, e0, expm="krylov", order=6, reortho=(k % 3 == 2), measure=True,
                         e_loc=e_loc, e_mix=e_mix, reuse_bias=True)
            torch.cuda.synchronize()
            out.append((w.psi.cpu().clone(), w.weight.cpu().clone(), e_loc.cpu().clone()))
        if batch:
            batch.close()
        res.append(out)
    for a, b in zip(res[0], res[1]):
        for x, y in zip(a, b):
            assert torch.equal(x, y)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_reuse_bias_after_workspace_growth(precision):
    """afqmc_local_energy, then a first Krylov step (its basis needs a larger
    workspace, which frees the stored traces): the step must recompute the
    force bias, i.e. equal the step without the option bit for bit."""
    s = make_system(66, 11, 11, 330, rho=1e-5 ** (1 / 330), seed=36)
    e0, tau, nw = _e0(s), 0.05, 9
    out = []
    for reuse in (True, False):
        ctx = _ctx(s, precision)
        w = ctx.new_walkers(nw)
        ctx.init_walkers(w)
        el = torch.empty(nw, 2, dtype=torch.float64, device=ctx.device)
        em = torch.empty(4, dtype=torch.float64, device=ctx.device)
        ctx.local_energy(w, e0, tau, el, em)
        x = torch.as_tensor(make_fields(12, 0, nw, s.G), device=ctx.device)
        ctx.step(w, x, tau, e0, expm="krylov", order=10, measure=True, e_loc=el, e_mix=em, reuse_bias=reuse)
        torch.cuda.synchronize()
        out.append((w.psi.cpu().clone(), w.weight.cpu().clone(), el.cpu().clone()))
        ctx.close()
    for a, b in zip(*out):
        assert torch.equal(a, b)

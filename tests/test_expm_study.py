"""The accuracy study of Sec. IV.E (Fig. 1), `expm_study`: on the CPU its
driver runs on the oracle (tests/oracle_context.py) and is checked against the
definitions it states; on the GPU the library's k_min and run errors are
compared with the oracle's on the same seeded system and fields."""
import pytest
import torch

from oracle import afqmc_ref as R
from oracle_context import OracleContext, field_fn
from paper_2403_02542_gb300 import expm_study as S
from paper_2403_02542_gb300.inputs import make_system

NW, STEPS, TAU = 8, 10, 0.1


def _setup():
    s = make_system(16, 3, 3, 40, rho=0.9, seed=5)
    octx = OracleContext(s)
    e0 = float(R.local_energy(octx.ham, octx.ham.trial.to(torch.complex128)).real)
    return s, octx, e0


def test_order_limits_match_the_header():
    """The study tries each action up to the largest order afqmc_step accepts,
    as the header states it."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "afqmc.h")).read()
    for name, macro in (("taylor", "TAYLOR"), ("krylov", "KRYLOV"), ("chebyshev", "CHEBYSHEV"),
                        ("bkrylov", "BLOCK_KRYLOV"), ("lanczos", "LANCZOS")):
        m = re.search(r"AFQMC_EXPM_" + macro + r" \(order = [^)]*?(\d+) <= k <= (\d+)", hdr)
        assert m is not None, name
        assert S.K_MAX[name] == int(m.group(2)), name
    assert S.REFERENCE == ("taylor", S.K_MAX["taylor"])


def test_reference_run_is_the_exact_exponential():
    """The order-64 Taylor reference equals the run with the exact action
    (the oracle's eigendecomposition/matrix_exp) and with Krylov at dimension N."""
    s, octx, e0 = _setup()
    f = field_fn(100, NW, octx.G)
    e_ref = S.run_energy(octx, NW, STEPS, f, TAU, e0, *S.REFERENCE)
    e_exact = S.run_energy(octx, NW, STEPS, f, TAU, e0, "exact", 0)
    e_kN = S.run_energy(octx, NW, STEPS, f, TAU, e0, "krylov", 16)
    assert abs(e_ref - e_exact) <= 1e-12 * abs(e_exact)
    assert abs(e_kN - e_exact) <= 1e-11 * abs(e_exact)


def test_k_min_is_the_first_order_within_eps():
    s, octx, e0 = _setup()
    f = field_fn(100, NW, octx.G)
    e_ref = S.run_energy(octx, NW, STEPS, f, TAU, e0, *S.REFERENCE)
    prev = 0
    for eps in (1e-3, 1e-5, 1e-8):
        for m in ("taylor", "krylov"):
            r = S.k_min(octx, NW, STEPS, f, TAU, e0, m, eps=eps, e_ref=e_ref)
            k = r["k_min"]
            assert k is not None and len(r["errors"]) == k
            assert r["errors"][-1] < eps and all(e >= eps for e in r["errors"][:-1])
            if m == "krylov":
                assert k >= prev        # a tighter eps never needs fewer products
                prev = k
    r = S.k_min(octx, NW, STEPS, f, TAU, e0, "taylor", eps=1e-14, k_max=2, e_ref=e_ref)
    assert r["k_min"] is None and len(r["errors"]) == 2


def test_krylov_needs_no_more_products_than_the_polynomials():
    """Fig. 1's ordering on this synthetic system at tau = 0.1: the Krylov
    actions reach 1e-5 Ha with no more A|Psi> products than Taylor or Chebyshev."""
    s, octx, e0 = _setup()
    res = S.sweep(octx, NW, STEPS, lambda tau: field_fn(100, NW, octx.G), (TAU,), e0)[TAU]
    assert res["krylov"] <= res["taylor"] and res["krylov"] <= res["chebyshev"]
    assert res["bkrylov"] <= res["taylor"] and res["bkrylov"] <= res["chebyshev"]


@pytest.mark.gpu
def test_library_k_min_matches_the_oracle():
    """FP64 library runs against the oracle runs: every run error within 1e-8 Ha
    and the same k_min for each action (orders whose error lies within 1e-8 of
    eps would be ties; none occurs on this system)."""
    from paper_2403_02542_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_02542_gb300.api import Context
    s, octx, e0 = _setup()
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64")
    fo = field_fn(100, NW, octx.G)
    fg = field_fn(100, NW, ctx.G, device=ctx.device)
    e_ref_o = S.run_energy(octx, NW, STEPS, fo, TAU, e0, *S.REFERENCE)
    e_ref_g = S.run_energy(ctx, NW, STEPS, fg, TAU, e0, *S.REFERENCE)
    assert abs(e_ref_g - e_ref_o) <= 1e-10 * abs(e_ref_o)
    for m in ("taylor", "chebyshev", "krylov", "bkrylov"):
        ro = S.k_min(octx, NW, STEPS, fo, TAU, e0, m, e_ref=e_ref_o)
        rg = S.k_min(ctx, NW, STEPS, fg, TAU, e0, m, e_ref=e_ref_g)
        assert all(abs(e - 1e-5) > 1e-8 for e in ro["errors"]), m
        assert rg["k_min"] == ro["k_min"], m
        for a, b in zip(rg["errors"], ro["errors"]):
            assert abs(a - b) <= 1e-8, m
    ctx.close()

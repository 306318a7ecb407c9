"""C ABI checks that need no GPU: the library builds and loads, exports every
symbol the header declares, validates arguments before touching the device,
and its host Jacobi eigensolver is correct."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2403_02542_gb300 import _lib as L
from paper_2403_02542_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(afqmc_\w+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "afqmc_step" in names and "afqmc_create" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    # and the binding declares them all
    assert names <= set(L.SIGNATURES)


def test_strerror(lib):
    assert lib.afqmc_strerror(L.AFQMC_OK) == b"ok"
    assert lib.afqmc_strerror(L.AFQMC_EDOM) == b"non-finite input"
    assert lib.afqmc_strerror(99) == b"unknown status"


def _create(lib, N=4, na=1, nb=1, G=3, h1=None, chol=None, trial=None, prec=0):
    h1 = np.eye(N) if h1 is None else h1
    chol = np.zeros((G, N, N)) if chol is None else chol
    trial = np.eye(na + nb, N) if trial is None else trial
    out = ctypes.c_void_p()
    return lib.afqmc_create(ctypes.byref(out), N, na, nb, G, h1.ctypes.data, chol.ctypes.data,
                            trial.ctypes.data, 0.0, prec, None), out


def test_create_rejects_bad_sizes_without_touching_the_device(lib):
    for kw in (dict(N=0), dict(na=0, nb=0), dict(na=5, N=4), dict(G=0), dict(N=600), dict(na=81, N=200)):
        st, out = _create(lib, **kw)
        assert st == L.AFQMC_EINVAL, kw
        assert not out.value
    st, _ = _create(lib, prec=7)
    assert st == L.AFQMC_EINVAL
    out = ctypes.c_void_p()
    assert lib.afqmc_create(ctypes.byref(out), 4, 1, 1, 3, None, None, None, 0.0, 0, None) == L.AFQMC_EINVAL


def test_create_rejects_non_finite_input(lib):
    h1 = np.eye(4)
    h1[1, 2] = np.nan
    st, out = _create(lib, h1=h1)
    assert st == L.AFQMC_EDOM and not out.value
    chol = np.zeros((3, 4, 4))
    chol[2, 0, 0] = np.inf
    assert _create(lib, chol=chol)[0] == L.AFQMC_EDOM


def test_null_context_calls_fail_cleanly(lib):
    assert lib.afqmc_set_tau(None, 0.1) == L.AFQMC_EINVAL
    assert lib.afqmc_sync(None) == L.AFQMC_EINVAL
    assert lib.afqmc_launch_count(None) == 0
    lib.afqmc_destroy(None)
    p = L.StepParams(0.1, 0.0, 0, 0, 4, 0, 0, 0)
    w = L.Walkers(1, None, None, None, None)
    assert lib.afqmc_step(None, ctypes.byref(w), None, ctypes.byref(p), None, None) == L.AFQMC_EINVAL


def test_host_eigh_against_numpy(lib):
    from paper_2403_02542_gb300.api import host_eigh
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 40):
        a = rng.standard_normal((n, n))
        a = a + a.T
        ev, V = host_eigh(a)
        order = np.argsort(ev)
        assert np.allclose(np.sort(ev), np.linalg.eigvalsh(a), atol=1e-12 * max(1, np.abs(a).max()))
        assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)
        assert np.allclose(a @ V, V * ev[None, :], atol=1e-11)
    # degenerate spectrum
    a = np.diag([1.0, 1.0, 2.0])
    ev, V = host_eigh(a)
    assert np.allclose(np.sort(ev), [1, 1, 2])
    bad = np.array([[1.0, np.nan], [np.nan, 1.0]])
    ev = np.empty(2); V = np.empty((2, 2))
    assert lib.afqmc_host_eigh(2, bad.ctypes.data, ev.ctypes.data, V.ctypes.data) == L.AFQMC_EDOM


def test_product_path_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", "/nonexistent/libafqmc.so")
    with pytest.raises(RuntimeError, match="missing"):
        L.lib()


def test_binding_constants_match_the_header():
    """Every enumerator and #define value of the header equals the binding's."""
    text = open(os.path.join(ROOT, "include", "afqmc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    values = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"(AFQMC_\w+)\s*=\s*(\d+)", body):
            values[name] = int(val)
    for name, val in re.findall(r"#define\s+(AFQMC_W_\w+)\s+(0x[0-9a-fA-F]+)u", text):
        values[name] = int(val, 16)
    assert values["AFQMC_EXPM_BLOCK_KRYLOV"] == 2 and values["AFQMC_MIXED"] == 1
    for name, val in values.items():
        if name.startswith("AFQMC_K_") and name != "AFQMC_K_COUNT":
            assert L.KERNEL_CLASSES[val] == name[len("AFQMC_K_"):].lower().replace("forcebias", "force_bias") \
                .replace("halfstep", "half_step"), name
        elif hasattr(L, name):
            assert getattr(L, name) == val, name
    assert values["AFQMC_K_COUNT"] == len(L.KERNEL_CLASSES)
    m = re.search(r"AFQMC_STATIC_SCRATCH_BYTES\s*\(\(unsigned long long\)(\d+)\s*<<\s*(\d+)\)", text)
    assert m and L.STATIC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2))


def test_binding_structs_match_the_header():
    """The ctypes mirrors of the header's parameter structs list the same
    fields, in the same order, with the same C types (so the offsets agree)."""
    text = open(os.path.join(ROOT, "include", "afqmc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    ctype = {"int": ctypes.c_int, "double": ctypes.c_double, "void*": ctypes.c_void_p,
             "uint32_t*": ctypes.c_void_p, "double*": ctypes.c_void_p}
    for cname, pyname in (("afqmc_walkers", "Walkers"), ("afqmc_step_params", "StepParams"),
                          ("afqmc_walk_adjoint_params", "WalkAdjointParams")):
        m = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + cname + r"\s*;", text)
        assert m, cname
        fields = []
        for decl in m.group(1).split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            mm = re.match(r"(?:const )?(\w+)\s*(\**)\s*(\w+)$", decl)
            assert mm, (cname, decl)
            fields.append((mm.group(3), ctype[mm.group(1) + mm.group(2)]))
        assert [(n, t) for n, t in getattr(L, pyname)._fields_] == fields, cname

"""The C-ABI library loads and exports every entry point include/wpccc.h declares (no GPU needed).

Only argument checking is exercised here: calls that fail validation queue no
GPU work, so they run on a machine without a GPU.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"WPCCC_API\s+[\w\s\*]+?\b(wpccc_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    path = os.path.join(ROOT, "paper_2403_04252_gb300", "libwpccc.so")
    if not os.path.exists(path):
        import __graft_entry__
        __graft_entry__.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"wpccc_basis_create", "wpccc_matrix_elements", "wpccc_solve", "wpccc_propagate",
            "wpccc_probabilities"} <= names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    import paper_2403_04252_gb300 as w
    assert set(w.EXPORTED) == _declared()


def test_argument_errors_without_gpu(lib):
    lib.wpccc_last_error.restype = C.c_char_p
    lib.wpccc_solve.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                C.c_void_p]
    assert lib.wpccc_solve(0, 1, None, None, None, None, 0, None) == 1          # EINVAL: N < 1
    assert b"N out of range" in lib.wpccc_last_error()
    assert lib.wpccc_solve(10, -1, None, None, None, None, 0, None) == 1        # EINVAL: batch < 0
    assert lib.wpccc_solve(10, 1, None, None, None, None, 0, None) == 1         # EINVAL: null pointers
    assert lib.wpccc_solve(10, 0, None, None, None, None, 0, None) == 0         # empty batch: nothing to do
    assert lib.wpccc_probabilities(-1, 4, None, None, None) == 1
    assert lib.wpccc_basis_create(None, 0, None) == 1
    assert lib.wpccc_basis_destroy(None) == 0


def test_null_handles_are_argument_errors_without_gpu(lib):
    # every entry point that takes a basis or a batch handle rejects a null one before any CUDA call
    EINVAL = 1
    lib.wpccc_last_error.restype = C.c_char_p
    P = C.c_void_p
    calls = {
        "wpccc_basis_info": ([P, P, P], [None, None, None]),
        "wpccc_matrix_elements": ([P, C.c_double, C.c_double, C.c_int, P, P, P, P],
                                  [None, 1.0, 1.0, 1, None, None, None, None]),
        "wpccc_matrix_elements_precision": ([P, C.c_double, C.c_double, C.c_int, P, P, P, C.c_int, P],
                                            [None, 1.0, 1.0, 1, None, None, None, 4, None]),
        "wpccc_matrix_elements_noalloc": ([P, C.c_double, C.c_double, C.c_int, P, P, P, P],
                                          [None, 1.0, 1.0, 1, None, None, None, None]),
        "wpccc_propagate": ([P, P, C.c_int, C.c_int, P, P], [None, None, 0, 0, None, None]),
        "wpccc_propagate_adjoint": ([P, P, C.c_int, P, C.c_int, P, P, P, P],
                                    [None, None, 1, None, 1, None, None, None, None]),
        "wpccc_basis_set_solve_mode": ([P, C.c_int], [None, 0]),
        "wpccc_basis_set_refine_iters": ([P, C.c_int], [None, 1]),
        "wpccc_basis_set_rk4_layout": ([P, C.c_int], [None, 0]),
        "wpccc_basis_set_workspace_limit": ([P, C.c_size_t], [None, 1 << 30]),
        "wpccc_basis_set_tangents": ([P, C.c_int, P, P, P, P, P], [None, 1, None, None, None, None, None]),
        "wpccc_profile_enable": ([P, C.c_int], [None, 1]),
        "wpccc_profile_read": ([P, P, P], [None, None, None]),
        "wpccc_batch_create": ([C.c_int, P, P, C.c_int, P, C.c_int, P], [0, None, None, 0, None, 0, None]),
        "wpccc_batch_launch": ([P, P], [None, None]),
        "wpccc_batch_status": ([P, P], [None, None]),
        "wpccc_batch_info": ([P, P, P], [None, None, None]),
    }
    for name, (types, args) in calls.items():
        f = getattr(lib, name)
        f.argtypes = types
        assert f(*args) == EINVAL, name
        assert name.encode() in lib.wpccc_last_error() or b"null" in lib.wpccc_last_error(), name
    lib.wpccc_batch_destroy.argtypes = [P]
    assert lib.wpccc_batch_destroy(None) == 0


def test_non_finite_inputs_are_argument_errors_without_gpu():
    # corrupt tables are refused at basis creation, before any device work: a NaN radial value, an
    # infinite state energy, a NaN quadrature weight
    import numpy as np
    import wpccc_inputs as wi
    import paper_2403_04252_gb300 as w

    def corrupt(kind):
        b = wi.make_basis(1.0, 1.0, 2, 1, 1, 2.0, True, Nr=200, Geta=8, Gtau=8)
        if kind == "f":
            b.T.f = b.T.f.copy()
            b.T.f[1, 50] = np.nan
        elif kind == "eps":
            b.P.st_eps = b.P.st_eps.copy()
            b.P.st_eps[2] = np.inf
        else:
            b.quad.ws = b.quad.ws.copy()
            b.quad.ws[3] = np.nan
        return b

    for kind, words in (("f", b"radial table"), ("eps", b"state energy"), ("quad", b"quadrature")):
        with pytest.raises(w.WpcccError) as e:
            w.Basis(corrupt(kind))
        assert e.value.status == w.EINVAL, kind
        assert words in w._lib.wpccc_last_error(), kind


def test_binding_constants_match_header():
    # every status code and #define the binding mirrors has the header's value
    import paper_2403_04252_gb300 as w
    src = open(os.path.join(ROOT, "include", "wpccc.h")).read()
    enum = {k: int(v) for k, v in re.findall(r"\bWPCCC_([A-Z]+)\s*=\s*(\d+)", src)}
    for name in ("OK", "EINVAL", "ENOMEM", "ESINGULAR", "ENONFINITE", "ECUDA", "EUNSUPPORTED", "ETIMEOUT",
                 "ENOCONV"):
        assert getattr(w, name) == enum[name], name
    defines = {k: v for k, v in re.findall(r"#define WPCCC_(\w+)\s+(\S.*)", src)}
    for name in ("LMAX", "NMAX", "MAX_PARAMS", "MAX_REFINE", "SOLVE_STAGE", "SOLVE_MATRIX", "SOLVE_SCHUR",
                 "RK4_AUTO", "RK4_SHARED", "RK4_GLOBAL", "SCHUR_UPDATE_AUTO", "SCHUR_UPDATE_TENSOR",
                 "SCHUR_UPDATE_CUDA_CORES"):
        assert getattr(w, name) == int(defines[name]), name
    assert w.NOALLOC_SCRATCH_BYTES == 64 << 20 and "64 << 20" in defines["NOALLOC_SCRATCH_BYTES"]
    assert len(w.PROF_CATEGORIES) == int(defines["PROF_N"])
    assert w.DEFAULT_WAIT_POLLS == 1 << 20 and "1L << 20" in defines["DEFAULT_WAIT_POLLS"]

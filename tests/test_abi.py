"""The C ABI library loads, exports every declared symbol, and validates
arguments on the host before touching the GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(tg_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_2602_05052_gb300 import build
    path = build.build_library()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n


def test_build_compiles_every_cuda_source():
    """Every translation unit under csrc/ is in the build's source list."""
    from paper_2602_05052_gb300 import build
    csrc = os.path.join(ROOT, "paper_2602_05052_gb300", "csrc")
    assert sorted(f for f in os.listdir(csrc) if f.endswith(".cu")) == sorted(build.SOURCES)


def test_status_strings(L):
    L.tg_status_string.restype = C.c_char_p
    assert L.tg_status_string(0) == b"TG_OK"
    assert L.tg_status_string(8) == b"TG_ERR_UNSUPPORTED"


def test_quadrature_rules_match_the_oracle(L):
    import oracle as O
    for el in (0, 1, 2, 3):
        nq = L.tg_quadrature(el, None, None)
        w = (C.c_double * nq)()
        x = (C.c_double * (3 * nq))()
        L.tg_quadrature(el, w, x)
        ow, ox = O.quadrature(min(el, 2))
        d = ox.shape[1]
        assert np.allclose(np.array(w[:]), ow, rtol=0, atol=1e-15)
        assert np.allclose(np.array(x[: nq * d]).reshape(nq, d), ox, rtol=0, atol=1e-15)
    # the quadrilateral's 2 x 2 Gauss rule against the quad oracle's
    from oracle import quad as Q
    pts, ow = Q.gauss2()
    w = (C.c_double * 4)()
    x = (C.c_double * 8)()
    assert L.tg_quadrature(4, w, x) == 4
    assert np.allclose(np.array(w[:]), ow, rtol=0, atol=1e-15)
    assert np.allclose(np.array(x[:]).reshape(4, 2), np.array(pts), rtol=0, atol=1e-15)


def test_host_validation_without_gpu(L):
    vp = C.c_void_p
    out = vp()
    L.tg_build_pattern.argtypes = [vp, C.c_int64, C.c_int64, C.c_int32, vp, C.POINTER(vp)]
    assert L.tg_build_pattern(None, 0, 10, 0, None, None) == 1            # no output handle
    assert L.tg_build_pattern(None, 0, 10, 7, None, C.byref(out)) == 1    # bad element kind
    assert L.tg_build_pattern(None, 5, 10, 0, None, C.byref(out)) == 1    # cells missing
    assert L.tg_build_pattern(None, 0, 0, 0, None, C.byref(out)) == 1     # no nodes
    assert L.tg_build_pattern(vp(16), 1 << 29, 10, 0, None, C.byref(out)) == 4  # index overflow
    L.tg_assemble_bilinear.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, C.c_double, vp, vp]
    assert L.tg_assemble_bilinear(None, 0, None, None, 1, 0.0, None, None) == 1
    L.tg_assemble_backward.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, C.c_double] + [vp] * 7
    assert L.tg_assemble_backward(None, 0, None, None, 1, 0.0, None, None, None, None, None, None, None) == 1
    L.tg_batch_create.argtypes = [vp, C.c_int32, C.POINTER(vp)]
    assert L.tg_batch_create(None, 0, C.byref(out)) == 1
    L.tg_diag_fma_rate.argtypes = [C.c_int32, vp, vp]
    assert L.tg_diag_fma_rate(1, None, None) == 1
    L.tg_diag_grid_barrier_timeout.argtypes = [C.c_int32, vp]
    assert L.tg_diag_grid_barrier_timeout(0, None) == 1
    assert L.tg_diag_grid_barrier_timeout((1 << 22) + 1, None) == 1
    L.tg_cg_solve.argtypes = [vp, C.c_int32, vp, vp, vp, vp, C.c_double, C.c_int32, vp, vp, vp]
    assert L.tg_cg_solve(None, 1, None, None, None, None, 1e-10, 10, None, None, None) == 1
    L.tg_residual.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, C.c_double, vp, vp, C.c_int32, vp, vp, vp, vp]
    assert L.tg_residual(None, 0, None, None, 1, 0.0, None, None, 2, None, None, None, None) == 1
    L.tg_semilinear_residual.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, C.c_double, vp, vp, C.c_int32, vp, vp,
                                         vp, vp, vp, vp]
    assert L.tg_semilinear_residual(None, 0, None, None, 1, 0.0, None, None, 2, None, None, None, None, None,
                                    None) == 1
    L.tg_pattern_layouts.argtypes = [vp, vp]
    flags = C.c_uint32(7)
    assert L.tg_pattern_layouts(None, C.byref(flags)) == 1 and flags.value == 7
    L.tg_build_facets.argtypes = [vp, vp, C.c_int64, vp, C.POINTER(vp)]
    assert L.tg_build_facets(None, None, 0, None, C.byref(out)) == 1
    assert L.tg_build_facets(None, None, 0, None, None) == 1
    L.tg_assemble_facets.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, vp, C.c_int32, vp, vp, vp]
    assert L.tg_assemble_facets(None, 0, None, None, 3, None, 3, None, None, None) == 1
    L.tg_assemble_simp.argtypes = [vp, C.c_int32, vp, vp] + [C.c_double] * 4 + [vp, vp]
    assert L.tg_assemble_simp(None, 0, None, None, 1.0, 2.0, 3.0, 0.3, None, None) == 1
    L.tg_simp_sensitivity.argtypes = [vp, C.c_int32, vp, vp] + [C.c_double] * 4 + [vp, vp, vp]
    assert L.tg_simp_sensitivity(None, 0, None, None, 1.0, 2.0, 3.0, 0.3, None, None, None) == 1
    L.tg_quadrature.argtypes = [C.c_int32, vp, vp]
    assert L.tg_quadrature(4, None, None) == 4   # the 2 x 2 Gauss rule of the quadrilateral
    assert L.tg_quadrature(5, None, None) == 0


def test_python_binding_imports_without_gpu():
    import paper_2602_05052_gb300 as tg
    assert tg.lib() is not None
    w, x = tg.tg_quadrature(tg.P2_TRI)
    assert abs(w.sum() - 0.5) < 1e-15

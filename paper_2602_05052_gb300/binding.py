"""Thin ctypes binding of libtg.so (argument marshalling only).

Every function carries the name of the C entry point it calls and takes
torch tensors that already live on the GPU; all computation happens in the
library's CUDA kernels.  There is no CPU fallback: if the library is not
built, importing raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from .build import LIB

P1_TRI, P2_TRI, P1_TET, P1_TET_VEC3, Q1_QUAD_VEC2 = 0, 1, 2, 3, 4
# Pattern.layouts flags (include/tg.h)
LAYOUT_ROW_BLOCKS, LAYOUT_FANS, LAYOUT_ELEM_POS, LAYOUT_EDGE_MASKS = 1, 2, 4, 8
F32, F64 = 0, 1
PER_ELEMENT, PER_QP, PER_NODE, CONSTANT = 0, 1, 2, 3
NV = {P1_TRI: 3, P2_TRI: 6, P1_TET: 4, P1_TET_VEC3: 4, Q1_QUAD_VEC2: 4}
DIM = {P1_TRI: 2, P2_TRI: 2, P1_TET: 3, P1_TET_VEC3: 3, Q1_QUAD_VEC2: 2}
NQ = {P1_TRI: 3, P2_TRI: 6, P1_TET: 4, P1_TET_VEC3: 4, Q1_QUAD_VEC2: 4}

STATUS = ["TG_OK", "TG_ERR_INVALID_ARG", "TG_ERR_INDEX_RANGE", "TG_ERR_DEGENERATE_ELEMENT", "TG_ERR_INDEX_OVERFLOW",
          "TG_ERR_OUT_OF_MEMORY", "TG_ERR_CUDA", "TG_ERR_TIMEOUT", "TG_ERR_UNSUPPORTED"]


class TGError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{where}: {name}" + (f" ({detail})" if detail else ""))


_lib = None
vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(f"{LIB} is missing: build it with `python -m paper_2602_05052_gb300.build` "
                          "(or __graft_entry__.build()); there is no fallback path")
    L = C.CDLL(LIB)
    sig = {
        "tg_status_string": (C.c_char_p, [i32]),
        "tg_last_error_message": (C.c_char_p, []),
        "tg_quadrature": (i32, [i32, vp, vp]),
        "tg_build_pattern": (i32, [vp, i64, i64, i32, vp, C.POINTER(vp)]),
        "tg_pattern_info": (i32, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                  C.POINTER(i32)]),
        "tg_pattern_shape": (i32, [vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i64), C.POINTER(i32),
                                   C.POINTER(i32)]),
        "tg_pattern_row_blocks": (i32, [vp, C.POINTER(i32), C.POINTER(i64)]),
        "tg_pattern_layouts": (i32, [vp, C.POINTER(C.c_uint32)]),
        "tg_get_device_status": (i32, [vp, C.POINTER(i64)]),
        "tg_pattern_destroy": (None, [vp]),
        "tg_assemble_bilinear": (i32, [vp, i32, vp, vp, i32, dbl, vp, vp]),
        "tg_assemble_bilinear_atomic": (i32, [vp, i32, vp, vp, i32, dbl, vp, vp]),
        "tg_assemble_elasticity": (i32, [vp, i32, vp, vp, vp, i32, vp, vp]),
        "tg_assemble_load": (i32, [vp, i32, vp, vp, i32, i32, vp, vp]),
        "tg_assemble_system": (i32, [vp, i32, vp, vp, i32, dbl, vp, i32, vp, vp, vp]),
        "tg_assemble_backward": (i32, [vp, i32, vp, vp, i32, dbl, vp, vp, vp, vp, vp, vp, vp]),
        "tg_assemble_load_backward": (i32, [vp, i32, vp, vp, i32, i32, vp, vp, vp, i32, vp]),
        "tg_assemble_elasticity_backward": (i32, [vp, i32, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp]),
        "tg_residual": (i32, [vp, i32, vp, vp, i32, dbl, vp, vp, i32, vp, vp, vp, vp]),
        "tg_semilinear_residual": (i32, [vp, i32, vp, vp, i32, dbl, vp, vp, i32, C.POINTER(dbl), vp, vp, vp, vp,
                                         vp]),
        "tg_assemble_simp": (i32, [vp, i32, vp, vp, dbl, dbl, dbl, dbl, vp, vp]),
        "tg_simp_sensitivity": (i32, [vp, i32, vp, vp, dbl, dbl, dbl, dbl, vp, vp, vp]),
        "tg_reaction_points": (i32, [vp, i32, vp, C.POINTER(dbl), vp, vp]),
        "tg_diag_wait_timeout": (i32, [vp, i32, vp]),
        "tg_diag_grid_barrier_timeout": (i32, [i32, vp]),
        "tg_build_facets": (i32, [vp, vp, i64, vp, C.POINTER(vp)]),
        "tg_assemble_facets": (i32, [vp, i32, vp, vp, i32, vp, i32, vp, vp, vp]),
        "tg_facets_shape": (i32, [vp, C.POINTER(i64), C.POINTER(i64)]),
        "tg_facets_destroy": (None, [vp]),
        "tg_spmv": (i32, [vp, i32, vp, vp, vp, vp]),
        "tg_csr_outer": (i32, [vp, i32, vp, vp, dbl, vp, vp]),
        "tg_scale_masked": (i32, [i32, vp, vp, dbl, vp, i64, vp]),
        "tg_cg_solve": (i32, [vp, i32, vp, vp, vp, vp, dbl, i32, C.POINTER(i32), C.POINTER(dbl), vp]),
        "tg_cg_solve_noalloc": (i32, [vp, i32, vp, vp, vp, vp, dbl, i32, C.POINTER(i32), C.POINTER(dbl), vp]),
        "tg_batch_create": (i32, [C.POINTER(vp), i32, C.POINTER(vp)]),
        "tg_batch_assemble": (i32, [vp, i32, C.POINTER(vp), C.POINTER(vp), i32, C.POINTER(dbl), C.POINTER(vp), vp]),
        "tg_batch_set_schedule": (i32, [vp, i32, i32, i32]),
        "tg_batch_get_schedule": (i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
        "tg_batch_autotune": (i32, [vp, i32, C.POINTER(vp), C.POINTER(vp), i32, C.POINTER(dbl), C.POINTER(vp), i32,
                                    C.POINTER(C.c_float), vp]),
        "tg_batch_destroy": (None, [vp]),
        "tg_diag_fma_rate": (i32, [i32, C.POINTER(dbl), vp]),
        "tg_diag_recip": (i32, [vp, vp, i64, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(st: int, where: str):
    if st != 0:
        msg = lib().tg_last_error_message()
        raise TGError(st, where, msg.decode() if msg else "")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _ptr(t, dtype=None, name="tensor", n=None, cur=None):
    """Raw device pointer of a tensor argument after checking it: a
    contiguous CUDA tensor of the expected dtype on the current device (cur,
    looked up when not given), with exactly n elements when n is given (the
    library reads and writes raw pointers, so a short or misplaced buffer
    must be refused here)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    cur = torch.cuda.current_device() if cur is None else cur
    if t.get_device() != cur:
        raise ValueError(f"{name} is on {t.device}, the current device is cuda:{cur}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _n_x(p):
    """Elements of the coordinate array of pattern p's mesh: [N][d]."""
    return p.n_nodes * DIM[p.el]


def _n_coef(p, layout, ncomp=1, n_per_elem=None, per_node=True):
    """Elements of a coefficient array of the given layout on pattern p
    (None for a layout the library rejects itself: PER_NODE where only
    per_node=True admits it, or an unknown value)."""
    if layout == PER_QP:
        return p.n_elems * (n_per_elem or NQ[p.el]) * ncomp
    if layout == PER_ELEMENT:
        return p.n_elems * ncomp
    if layout == PER_NODE and per_node:
        return p.n_nodes * ncomp
    if layout == CONSTANT:
        return ncomp
    return None


def _out(arg, make):
    """Output argument: True allocates, False/None skips, a tensor is filled."""
    if arg is True:
        return make()
    if arg is None or arg is False:
        return None
    return arg


class _DevView:
    """__cuda_array_interface__ view of a library-owned device buffer."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 2, "strides": None}


def tg_quadrature(el: int):
    L = lib()
    nq = L.tg_quadrature(el, None, None)
    w = (C.c_double * nq)()
    x = (C.c_double * (nq * 3))()
    L.tg_quadrature(el, w, x)
    d = DIM[el]
    import numpy as np
    return np.array(w[:]), np.array(x[: nq * d]).reshape(nq, d)


class Pattern:
    """Owns a tg_pattern handle (tg_build_pattern / tg_pattern_destroy)."""

    def __init__(self, handle, device):
        self.handle = handle
        self.device = device
        L = lib()
        el, E, N, mrl, mdeg = i32(), i64(), i64(), i32(), i32()
        _check(L.tg_pattern_shape(handle, C.byref(el), C.byref(E), C.byref(N), C.byref(mrl), C.byref(mdeg)),
               "tg_pattern_shape")
        self.el, self.n_elems, self.n_nodes = el.value, E.value, N.value
        self.max_row_len, self.max_degree = mrl.value, mdeg.value
        nr, nnz, rp, ci, es, ss = i64(), i64(), vp(), vp(), vp(), i32()
        _check(L.tg_pattern_info(handle, C.byref(nr), C.byref(nnz), C.byref(rp), C.byref(ci), C.byref(es),
                                 C.byref(ss)), "tg_pattern_info")
        self.n_rows, self.nnz = nr.value, nnz.value
        rb, nb = i32(), i64()
        _check(L.tg_pattern_row_blocks(handle, C.byref(rb), C.byref(nb)), "tg_pattern_row_blocks")
        self.rows_per_block, self.n_blocks = rb.value, nb.value
        lf = C.c_uint32()
        _check(L.tg_pattern_layouts(handle, C.byref(lf)), "tg_pattern_layouts")
        self.layouts = lf.value
        self._rp, self._ci, self._es, self.slot_stride = rp.value, ci.value, es.value, ss.value

    def _view(self, ptr, n):
        if n == 0:
            return torch.empty(0, dtype=torch.int32, device=self.device)
        t = torch.as_tensor(_DevView(ptr, n, "<i4"), device=self.device)
        return t

    @property
    def row_ptr(self):
        return self._view(self._rp, self.n_rows + 1)

    @property
    def col_idx(self):
        return self._view(self._ci, self.nnz)

    @property
    def elem_slot(self):
        return self._view(self._es, self.n_elems * self.slot_stride)

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.tg_pattern_destroy(h)


def tg_build_pattern(cells: torch.Tensor, n_nodes: int, el: int, stream=None) -> Pattern:
    if cells.dim() != 2 or cells.shape[1] != NV[el]:
        raise ValueError("cells must be [E, nv]")
    h = vp()
    _check(lib().tg_build_pattern(_ptr(cells, torch.int32, "cells"), cells.shape[0], int(n_nodes), el,
                                  _stream(stream), C.byref(h)), "tg_build_pattern")
    return Pattern(h, cells.device)


def tg_get_device_status(p: Pattern):
    bad = i64()
    st = lib().tg_get_device_status(p.handle, C.byref(bad))
    return st, bad.value


def tg_assemble_bilinear(p: Pattern, coords, kappa, layout: int, c: float = 0.0, vals_out=None, stream=None):
    if vals_out is None:
        vals_out = torch.empty(p.nnz, dtype=coords.dtype, device=coords.device)
    dt = _dt(coords)
    _check(lib().tg_assemble_bilinear(p.handle, dt, _ptr(coords, coords.dtype, "coords", _n_x(p)),
                                      _ptr(kappa, coords.dtype, "kappa", _n_coef(p, layout, per_node=False)), layout, float(c),
                                      _ptr(vals_out, coords.dtype, "vals_out", p.nnz), _stream(stream)),
           "tg_assemble_bilinear")
    return vals_out


def tg_assemble_bilinear_atomic(p: Pattern, coords, kappa, layout: int, c: float = 0.0, vals_out=None, stream=None):
    if vals_out is None:
        vals_out = torch.empty(p.nnz, dtype=coords.dtype, device=coords.device)
    _check(lib().tg_assemble_bilinear_atomic(p.handle, _dt(coords), _ptr(coords, coords.dtype, "coords", _n_x(p)),
                                             _ptr(kappa, coords.dtype, "kappa", _n_coef(p, layout, per_node=False)), layout,
                                             float(c), _ptr(vals_out, coords.dtype, "vals_out", p.nnz),
                                             _stream(stream)),
           "tg_assemble_bilinear_atomic")
    return vals_out


def tg_assemble_elasticity(p: Pattern, coords, lam, mu, layout: int, vals_out=None, stream=None):
    if vals_out is None:
        vals_out = torch.empty(p.nnz, dtype=coords.dtype, device=coords.device)
    _check(lib().tg_assemble_elasticity(p.handle, _dt(coords), _ptr(coords, coords.dtype, "coords", _n_x(p)),
                                        _ptr(lam, coords.dtype, "lam", _n_coef(p, layout, per_node=False)),
                                        _ptr(mu, coords.dtype, "mu", _n_coef(p, layout, per_node=False)), layout,
                                        _ptr(vals_out, coords.dtype, "vals_out", p.nnz), _stream(stream)),
           "tg_assemble_elasticity")
    return vals_out


def tg_assemble_load(p: Pattern, coords, f, layout: int, ncomp: int = 1, F_out=None, stream=None):
    if F_out is None:
        F_out = torch.empty(p.n_nodes * ncomp, dtype=coords.dtype, device=coords.device)
    _check(lib().tg_assemble_load(p.handle, _dt(coords), _ptr(coords, coords.dtype, "coords", _n_x(p)),
                                  _ptr(f, coords.dtype, "f", _n_coef(p, layout, ncomp)), layout, int(ncomp),
                                  _ptr(F_out, coords.dtype, "F_out", p.n_nodes * ncomp), _stream(stream)),
           "tg_assemble_load")
    return F_out


def tg_assemble_system(p: Pattern, coords, kappa, kappa_layout: int, c: float, f, f_layout: int, vals=True, F=True,
                       stream=None):
    """Returns (vals [nnz], F [N]): the bilinear values and the load vector in one call (pass tensors to fill)."""
    dt = coords.dtype
    vals = _out(vals, lambda: torch.empty(p.nnz, dtype=dt, device=coords.device))
    F = _out(F, lambda: torch.empty(p.n_nodes, dtype=dt, device=coords.device))
    _check(lib().tg_assemble_system(p.handle, _dt(coords), _ptr(coords, dt, "coords", _n_x(p)),
                                    _ptr(kappa, dt, "kappa", _n_coef(p, kappa_layout, per_node=False)), kappa_layout, float(c),
                                    _ptr(f, dt, "f", _n_coef(p, f_layout)), f_layout,
                                    _ptr(vals, dt, "vals", p.nnz), _ptr(F, dt, "F", p.n_nodes), _stream(stream)),
           "tg_assemble_system")
    return vals, F


def tg_assemble_backward(p: Pattern, coords, kappa, layout: int, c: float = 0.0, grad_vals=None, lam=None, U=None,
                         grad_kappa=True, grad_coords=True, grad_c=True, stream=None):
    """Returns (grad_kappa, grad_coords [N, d], grad_c [1]); pass False to skip one."""
    dt = coords.dtype
    dev = coords.device
    gk = _out(grad_kappa, lambda: torch.empty_like(kappa))
    gx = _out(grad_coords, lambda: torch.empty_like(coords))
    gc = _out(grad_c, lambda: torch.empty(1, dtype=dt, device=dev))
    nk = _n_coef(p, layout, per_node=False)
    _check(lib().tg_assemble_backward(p.handle, _dt(coords), _ptr(coords, dt, "coords", _n_x(p)),
                                      _ptr(kappa, dt, "kappa", nk), layout, float(c),
                                      _ptr(grad_vals, dt, "grad_vals", p.nnz), _ptr(lam, dt, "lam", p.n_rows),
                                      _ptr(U, dt, "U", p.n_rows), _ptr(gk, dt, "grad_kappa", nk),
                                      _ptr(gx, dt, "grad_coords", _n_x(p)), _ptr(gc, dt, "grad_c", 1),
                                      _stream(stream)), "tg_assemble_backward")
    return gk, gx, gc


def tg_assemble_load_backward(p: Pattern, coords, f, layout: int, ncomp: int, grad_F, grad_f=True,
                              grad_coords=True, accumulate: bool = False, stream=None):
    """Returns (grad_f, grad_coords); pass False to skip one, or tensors to fill."""
    dt = coords.dtype
    gf = _out(grad_f, lambda: torch.empty_like(f))
    gx = _out(grad_coords, lambda: torch.empty_like(coords))
    nf = _n_coef(p, layout, ncomp)
    _check(lib().tg_assemble_load_backward(p.handle, _dt(coords), _ptr(coords, dt, "coords", _n_x(p)),
                                           _ptr(f, dt, "f", nf), layout, int(ncomp),
                                           _ptr(grad_F, dt, "grad_F", p.n_nodes * ncomp), _ptr(gf, dt, "grad_f", nf),
                                           _ptr(gx, dt, "grad_coords", _n_x(p)), int(bool(accumulate)),
                                           _stream(stream)),
           "tg_assemble_load_backward")
    return gf, gx


def tg_assemble_elasticity_backward(p: Pattern, coords, lam, mu, layout: int, grad_vals=None, lam_adj=None, U=None,
                                    grad_lam=True, grad_mu=True, grad_coords=True, stream=None):
    """Returns (grad_lam, grad_mu, grad_coords [N, 3]); pass False to skip one."""
    dt = coords.dtype
    gl = _out(grad_lam, lambda: torch.empty_like(lam))
    gm = _out(grad_mu, lambda: torch.empty_like(mu))
    gx = _out(grad_coords, lambda: torch.empty_like(coords))
    nc = _n_coef(p, layout, per_node=False)
    _check(lib().tg_assemble_elasticity_backward(p.handle, _dt(coords), _ptr(coords, dt, "coords", _n_x(p)),
                                                 _ptr(lam, dt, "lam", nc), _ptr(mu, dt, "mu", nc), layout,
                                                 _ptr(grad_vals, dt, "grad_vals", p.nnz),
                                                 _ptr(lam_adj, dt, "lam_adj", p.n_rows), _ptr(U, dt, "U", p.n_rows),
                                                 _ptr(gl, dt, "grad_lam", nc), _ptr(gm, dt, "grad_mu", nc),
                                                 _ptr(gx, dt, "grad_coords", _n_x(p)), _stream(stream)),
           "tg_assemble_elasticity_backward")
    return gl, gm, gx


def tg_residual(p: Pattern, coords, kappa, layout: int, c: float, x, f=None, f_layout: int = PER_NODE, dirichlet=None,
                y=None, loss=True, stream=None):
    """Matrix-free y = K x - F (F omitted when f is None); returns (y, loss [1] or None)."""
    dt = coords.dtype
    if y is None:
        y = torch.empty_like(x)
    ls = _out(loss, lambda: torch.empty(1, dtype=dt, device=coords.device))
    _check(lib().tg_residual(p.handle, _dt(coords), _ptr(coords, dt, "coords", _n_x(p)),
                             _ptr(kappa, dt, "kappa", _n_coef(p, layout, per_node=False)), layout, float(c),
                             _ptr(x, dt, "x", p.n_nodes), _ptr(f, dt, "f", _n_coef(p, f_layout)), f_layout,
                             _ptr(dirichlet, torch.uint8, "dirichlet", p.n_nodes), _ptr(y, dt, "y", p.n_nodes),
                             _ptr(ls, dt, "loss", 1), _stream(stream)), "tg_residual")
    return y, ls


def tg_semilinear_residual(p: Pattern, coords, kappa, layout: int, c: float, x, reaction, f=None,
                           f_layout: int = PER_NODE, x_react=None, dirichlet=None, y=None, loss=True, stream=None):
    """y = K x + N(x) - F with the reaction r(u) = sum_k reaction[k] u^k (or,
    with x_react, its Jacobian at x_react applied to x); returns (y, loss)."""
    dt = coords.dtype
    if y is None:
        y = torch.empty_like(x)
    ls = _out(loss, lambda: torch.empty(1, dtype=dt, device=coords.device))
    r = (dbl * 4)(*[float(v) for v in reaction])
    _check(lib().tg_semilinear_residual(p.handle, _dt(coords), _ptr(coords, dt, "coords", _n_x(p)),
                                        _ptr(kappa, dt, "kappa", _n_coef(p, layout, per_node=False)), layout, float(c),
                                        _ptr(x, dt, "x", p.n_nodes), _ptr(f, dt, "f", _n_coef(p, f_layout)),
                                        f_layout, r, _ptr(x_react, dt, "x_react", p.n_nodes),
                                        _ptr(dirichlet, torch.uint8, "dirichlet", p.n_nodes),
                                        _ptr(y, dt, "y", p.n_nodes), _ptr(ls, dt, "loss", 1), _stream(stream)),
           "tg_semilinear_residual")
    return y, ls


def tg_assemble_simp(p: Pattern, coords, rho, e_min: float, e_max: float, penal: float, nu: float, vals_out=None,
                     stream=None):
    if vals_out is None:
        vals_out = torch.empty(p.nnz, dtype=coords.dtype, device=coords.device)
    _check(lib().tg_assemble_simp(p.handle, _dt(coords), _ptr(coords, coords.dtype, "coords", _n_x(p)),
                                  _ptr(rho, coords.dtype, "rho", p.n_elems), float(e_min), float(e_max), float(penal),
                                  float(nu), _ptr(vals_out, coords.dtype, "vals", p.nnz), _stream(stream)),
           "tg_assemble_simp")
    return vals_out


def tg_simp_sensitivity(p: Pattern, coords, rho, e_min: float, e_max: float, penal: float, nu: float, u, dc_out=None,
                        stream=None):
    if dc_out is None:
        dc_out = torch.empty_like(rho)
    _check(lib().tg_simp_sensitivity(p.handle, _dt(coords), _ptr(coords, coords.dtype, "coords", _n_x(p)),
                                     _ptr(rho, coords.dtype, "rho", p.n_elems), float(e_min), float(e_max),
                                     float(penal), float(nu), _ptr(u, coords.dtype, "u", p.n_rows),
                                     _ptr(dc_out, coords.dtype, "dc", p.n_elems), _stream(stream)),
           "tg_simp_sensitivity")
    return dc_out


def tg_reaction_points(p: Pattern, x, reaction, out=None, stream=None):
    """r(u_q) at the quadrature points of every element: [E * Q]."""
    if out is None:
        out = torch.empty(p.n_elems * NQ[p.el], dtype=x.dtype, device=x.device)
    r = (dbl * 4)(*[float(v) for v in reaction])
    _check(lib().tg_reaction_points(p.handle, _dt(x), _ptr(x, x.dtype, "x", p.n_nodes), r,
                                    _ptr(out, x.dtype, "out", p.n_elems * NQ[p.el]), _stream(stream)),
           "tg_reaction_points")
    return out


def tg_diag_wait_timeout(p: Pattern, max_tries: int = 1000, stream=None):
    _check(lib().tg_diag_wait_timeout(p.handle, int(max_tries), _stream(stream)), "tg_diag_wait_timeout")


def tg_diag_grid_barrier_timeout(max_polls: int = 1000, stream=None) -> int:
    """Runs the grid-barrier failure check and returns its status code
    (TG_ERR_TIMEOUT = 7 when the barrier gave up, as it should)."""
    return int(lib().tg_diag_grid_barrier_timeout(int(max_polls), _stream(stream)))


class Facets:
    """Owns a tg_facets handle (tg_build_facets / tg_facets_destroy); keeps
    its pattern alive."""

    def __init__(self, handle, pattern):
        self.handle = handle
        self.pattern = pattern
        F, M = i64(), i64()
        _check(lib().tg_facets_shape(handle, C.byref(F), C.byref(M)), "tg_facets_shape")
        self.n_facets, self.n_boundary_nodes = F.value, M.value

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.tg_facets_destroy(h)


def tg_build_facets(p: Pattern, facets: torch.Tensor, stream=None) -> Facets:
    if facets.dim() != 2 or facets.shape[1] != DIM[p.el]:
        raise ValueError("facets must be [F, d]")
    h = vp()
    _check(lib().tg_build_facets(p.handle, _ptr(facets, torch.int32, "facets"), facets.shape[0], _stream(stream),
                                 C.byref(h)), "tg_build_facets")
    return Facets(h, p)


def tg_assemble_facets(fc: Facets, coords, alpha=None, alpha_layout: int = CONSTANT, g=None, g_layout: int = CONSTANT,
                       vals=None, F=None, stream=None):
    """Adds the Robin matrix term to vals and the facet load to F (in place)."""
    dt = coords.dtype
    p, nqf = fc.pattern, DIM[fc.pattern.el]  # points per facet: 2 on an edge, 3 on a face
    n_fc = lambda lay: (fc.n_facets * nqf if lay == PER_QP else fc.n_facets if lay == PER_ELEMENT
                        else p.n_nodes if lay == PER_NODE else 1 if lay == CONSTANT else None)
    _check(lib().tg_assemble_facets(fc.handle, _dt(coords), _ptr(coords, dt, "coords", _n_x(p)),
                                    _ptr(alpha, dt, "alpha", n_fc(alpha_layout)), alpha_layout,
                                    _ptr(g, dt, "g", n_fc(g_layout)), g_layout, _ptr(vals, dt, "vals", p.nnz),
                                    _ptr(F, dt, "F", p.n_nodes), _stream(stream)), "tg_assemble_facets")
    return vals, F


def tg_csr_outer(p: Pattern, lam, U, alpha: float = 1.0, out=None, stream=None):
    if out is None:
        out = torch.empty(p.nnz, dtype=lam.dtype, device=lam.device)
    _check(lib().tg_csr_outer(p.handle, _dt(lam), _ptr(lam, lam.dtype, "lam", p.n_rows),
                              _ptr(U, lam.dtype, "U", p.n_rows), float(alpha), _ptr(out, lam.dtype, "out", p.nnz),
                              _stream(stream)), "tg_csr_outer")
    return out


def tg_scale_masked(x, alpha: float = 1.0, dirichlet=None, out=None, stream=None):
    """alpha * x with zeros on the rows where dirichlet != 0 (out may be x)."""
    if out is None:
        out = torch.empty_like(x)
    n = x.numel()
    _check(lib().tg_scale_masked(_dt(x), _ptr(x, x.dtype, "x"), _ptr(dirichlet, torch.uint8, "dirichlet", n),
                                 float(alpha), _ptr(out, x.dtype, "out", n), n, _stream(stream)),
           "tg_scale_masked")
    return out


def tg_spmv(p: Pattern, vals, x, y=None, stream=None):
    if y is None:
        y = torch.empty(p.n_rows, dtype=vals.dtype, device=vals.device)
    _check(lib().tg_spmv(p.handle, _dt(vals), _ptr(vals, vals.dtype, "vals", p.nnz),
                         _ptr(x, vals.dtype, "x", p.n_rows), _ptr(y, vals.dtype, "y", p.n_rows), _stream(stream)),
           "tg_spmv")
    return y


def tg_cg_solve(p: Pattern, vals, F, dirichlet=None, x=None, rtol: float = 1e-10, maxit: int = 100000, stream=None):
    if x is None:
        x = torch.zeros(p.n_rows, dtype=vals.dtype, device=vals.device)
    it, rr = i32(), dbl()
    _check(lib().tg_cg_solve(p.handle, _dt(vals), _ptr(vals, vals.dtype, "vals", p.nnz),
                             _ptr(F, vals.dtype, "F", p.n_rows), _ptr(dirichlet, torch.uint8, "dirichlet", p.n_rows),
                             _ptr(x, vals.dtype, "x", p.n_rows), float(rtol), int(maxit), C.byref(it), C.byref(rr),
                             _stream(stream)), "tg_cg_solve")
    return x, it.value, rr.value


TG_CG_NOALLOC_SCRATCH_BYTES = 16 << 20


def tg_cg_solve_noalloc(p: Pattern, vals, F, dirichlet=None, x=None, rtol: float = 1e-10, maxit: int = 100000,
                        stream=None):
    """tg_cg_solve with its work vectors in the library's fixed device
    scratch (no allocation; calls on one device must not overlap)."""
    if x is None:
        x = torch.zeros(p.n_rows, dtype=vals.dtype, device=vals.device)
    it, rr = i32(), dbl()
    _check(lib().tg_cg_solve_noalloc(p.handle, _dt(vals), _ptr(vals, vals.dtype, "vals", p.nnz),
                                     _ptr(F, vals.dtype, "F", p.n_rows),
                                     _ptr(dirichlet, torch.uint8, "dirichlet", p.n_rows),
                                     _ptr(x, vals.dtype, "x", p.n_rows), float(rtol), int(maxit), C.byref(it),
                                     C.byref(rr), _stream(stream)),
           "tg_cg_solve_noalloc")
    return x, it.value, rr.value


class Batch:
    """Owns a tg_batch handle (tg_batch_create / tg_batch_destroy)."""

    def __init__(self, handle, pats):
        self.handle = handle
        self.pats = pats  # keep the patterns alive

    def schedule(self):
        t, r, c = i32(), i32(), i32()
        _check(lib().tg_batch_get_schedule(self.handle, C.byref(t), C.byref(r), C.byref(c)), "tg_batch_get_schedule")
        return t.value, r.value, c.value

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.tg_batch_destroy(h)


def tg_batch_create(pats: list[Pattern]) -> Batch:
    arr = (vp * len(pats))(*[p.handle for p in pats])
    h = vp()
    _check(lib().tg_batch_create(arr, len(pats), C.byref(h)), "tg_batch_create")
    return Batch(h, list(pats))


def _ptr_array(ts, dtype, name, sizes=None):
    if sizes is not None and len(sizes) != len(ts):
        raise ValueError(f"{name}: {len(ts)} tensors for {len(sizes)} instances")
    cur = torch.cuda.current_device()
    return (vp * len(ts))(*[_ptr(t, dtype, name, None if sizes is None else sizes[k], cur) for k, t in enumerate(ts)])


def _batch_sizes(b: Batch, layout: int):
    """Expected element counts of every instance's coords, kappa and values."""
    return ([_n_x(q) for q in b.pats], [_n_coef(q, layout, per_node=False) for q in b.pats], [q.nnz for q in b.pats])


def tg_batch_assemble(b: Batch, coords: list, kappa: list, layout: int, c: list, vals_out: list, stream=None):
    dt = coords[0].dtype
    n = len(coords)
    nx, nk, nv = _batch_sizes(b, layout)
    _check(lib().tg_batch_assemble(b.handle, _dt(coords[0]), _ptr_array(coords, dt, "coords", nx),
                                   _ptr_array(kappa, dt, "kappa", nk), layout, (dbl * n)(*map(float, c)),
                                   _ptr_array(vals_out, dt, "vals_out", nv), _stream(stream)), "tg_batch_assemble")
    return vals_out


def tg_batch_set_schedule(b: Batch, threads: int, rows_per_item: int, ctas_per_sm: int = 0):
    _check(lib().tg_batch_set_schedule(b.handle, threads, rows_per_item, ctas_per_sm), "tg_batch_set_schedule")


def tg_batch_autotune(b: Batch, coords: list, kappa: list, layout: int, c: list, vals_out: list, reps: int = 5,
                      stream=None):
    dt = coords[0].dtype
    n = len(coords)
    ms = C.c_float()
    nx, nk, nv = _batch_sizes(b, layout)
    _check(lib().tg_batch_autotune(b.handle, _dt(coords[0]), _ptr_array(coords, dt, "coords", nx),
                                   _ptr_array(kappa, dt, "kappa", nk), layout, (dbl * n)(*map(float, c)),
                                   _ptr_array(vals_out, dt, "vals_out", nv), int(reps), C.byref(ms),
                                   _stream(stream)),
           "tg_batch_autotune")
    return ms.value


def tg_diag_recip(x, stream=None):
    """The FP64 reciprocal the P1 forward kernels take of |det J|, elementwise."""
    y = torch.empty_like(x)
    n = x.numel()
    _check(lib().tg_diag_recip(_ptr(x, torch.float64, "x", n), _ptr(y, torch.float64, "y", n), n, _stream(stream)),
           "tg_diag_recip")
    return y


def tg_diag_fma_rate(dtype=torch.float64, stream=None) -> float:
    out = dbl()
    _check(lib().tg_diag_fma_rate(F64 if dtype == torch.float64 else F32, C.byref(out), _stream(stream)),
           "tg_diag_fma_rate")
    return out.value

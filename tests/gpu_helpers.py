"""Shared helpers of the GPU parity tests (inputs on the device, oracle
inputs rounded the way an FP32 run sees them, error metrics)."""
from __future__ import annotations

import numpy as np
import torch

import meshgen as mg
import oracle as O

# relative Frobenius tolerances of the GPU result against the FP64 oracle
TOL = {torch.float64: 1e-12, torch.float32: 2e-6}


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host_as(a, dtype):
    """What the oracle sees for an input the GPU reads in `dtype`."""
    a = np.asarray(a, dtype=np.float64)
    return a.astype(np.float32).astype(np.float64) if dtype == torch.float32 else a


# every relative error computed during the session: (test id, value); the
# conftest prints the largest per test at the end of the run
ERRORS: list = []
CURRENT = {"test": None}


def rel_scalar(got, want):
    """|got - want| / |want| of a scalar (recorded like relfro)."""
    err = abs(float(got) - float(want)) / (abs(float(want)) if want != 0 else 1.0)
    ERRORS.append((CURRENT["test"], err))
    return err


# A loss sum_i y_i^2 whose vector y is within relative Frobenius error t of
# the oracle's is within 2 t + t^2 of the oracle's loss (|dL| <= 2 |y| |dy|
# + |dy|^2): twice the vector bounds.
LOSS_TOL = {torch.float64: 2e-12, torch.float32: 4e-6}


def relfro(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    n = np.linalg.norm(want)
    err = float(np.linalg.norm(got - want) / (n if n > 0 else 1.0))
    ERRORS.append((CURRENT["test"], err))
    return err


def jittered_tri(n, seed=3, hilbert=True):
    m = mg.jitter(mg.tri_grid(n), seed)
    return mg.hilbert_order(m) if hilbert else m


def jittered_tet(n, seed=4, frac=0.15):
    m = mg.kuhn_tet_grid(n)
    g = np.random.default_rng(seed)
    disp = g.uniform(-frac * m.h, frac * m.h, size=m.coords.shape)
    disp[m.boundary] = 0
    m.coords = m.coords + disp
    return m


def mesh_for(el, size="small"):
    if el == mg.P1_TRI:
        return jittered_tri(37 if size == "small" else 64)
    if el == mg.P2_TRI:
        return mg.hilbert_order(mg.p2_tri_grid(13 if size == "small" else 24, jitter_seed=5))
    m = jittered_tet(7 if size == "small" else 10)
    if el == mg.P1_TET_VEC3:
        m.el = mg.P1_TET_VEC3
    return m


def coef(layout, E, nq, seed, lo=0.5, hi=2.0):
    g = np.random.default_rng(seed)
    if layout == mg.PER_QP:
        return g.uniform(lo, hi, size=E * nq)
    if layout == mg.PER_ELEMENT:
        return g.uniform(lo, hi, size=E)
    return np.array([g.uniform(lo, hi)])

"""GB300-native Galerkin assembly (TensorGalerkin's Map-Reduce) on one GPU.

The compute lives in ``libtg.so`` (hand-written sm_103a CUDA behind a C
ABI, declared in ``include/tg.h``); ``binding`` marshals torch tensors into
its calls and ``autograd`` wraps them in ``torch.autograd.Function``s.
"""
from .binding import (CONSTANT, DIM, F32, F64, LAYOUT_EDGE_MASKS, LAYOUT_ELEM_POS, LAYOUT_FANS, LAYOUT_ROW_BLOCKS,
                      NQ, NV, P1_TET, P1_TET_VEC3, P1_TRI, P2_TRI, PER_ELEMENT, PER_NODE,
                      Q1_QUAD_VEC2, tg_assemble_simp, tg_simp_sensitivity,
                      PER_QP, Batch, Facets, Pattern, TGError, lib, tg_assemble_backward, tg_assemble_bilinear,
                      tg_assemble_bilinear_atomic, tg_assemble_elasticity, tg_assemble_facets, tg_build_facets, tg_assemble_elasticity_backward,
                      tg_assemble_load, tg_assemble_load_backward, tg_assemble_system, tg_batch_assemble,
                      tg_batch_autotune, tg_batch_create, tg_batch_set_schedule, tg_build_pattern, tg_cg_solve, tg_cg_solve_noalloc,
                      tg_csr_outer, tg_scale_masked,
                      tg_diag_fma_rate, tg_diag_grid_barrier_timeout, tg_diag_recip, tg_diag_wait_timeout, tg_reaction_points, tg_residual, tg_semilinear_residual, tg_get_device_status, tg_quadrature, tg_spmv)

__all__ = [n for n in dir() if n.startswith("tg_")] + [
    "Pattern", "Batch", "Facets", "TGError", "lib", "P1_TRI", "P2_TRI", "P1_TET", "P1_TET_VEC3", "Q1_QUAD_VEC2", "PER_ELEMENT", "PER_QP",
    "PER_NODE", "CONSTANT", "F32", "F64", "NV", "DIM", "NQ"] + [n for n in dir() if n.startswith("LAYOUT_")]

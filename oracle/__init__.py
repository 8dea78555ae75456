"""Plain FP64 CPU oracle for the PPCG eigensolver (Vecharynski, Yang, Pask, arXiv 1407.7506).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or execute anything under oracle/:
only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg use it. It shares no code
with the CUDA library: it reads only the seeded inputs from the standalone `workloads` module.
"""
from .ppcg import (  # noqa: F401
    apply_H, diag_H, assemble_H, precondition, project, cholqr, cholqr2, shifted_cholqr3,
    block_coefficients, block_update, rayleigh_ritz, residual, ppcg, PPCGResult, normalize_phase,
    subblocks, orth, energy_gradient, polar_coefficients, polar_terms, orth_polar, orthonormalize, POLAR_MAX_TERMS,
)

"""Write the stored expected values under tests/golden/ from the CPU oracle only.

  grid16_k64_dense_eigs.txt    the 72 smallest eigenvalues of the 16^3 uniform-potential operator (n = 4096) by
                           dense LAPACK eigh of the entry-by-entry assembled matrix (oracle.assemble_H):
                           the plain definition of the result (the k smallest eigenpairs, Section 2, eq. tracemin).
  grid32_k256_oracle_eigs.txt  the 256 smallest eigenpairs' values and residuals of the 32^3, 8-well operator
                           (n = 32768) from the oracle's Algorithm 3 run to max residual 1e-8.

Usage: python tests/golden/make_golden.py [grid16_k64] [grid32_k256]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
import oracle  # noqa: E402


def grid16_k64():
    w = wl.GRID16_K64
    V, _ = wl.make_inputs(w)
    t = time.time()
    ev = np.linalg.eigvalsh(oracle.assemble_H(V, w.N, w.h))[:72]
    with open(os.path.join(HERE, "grid16_k64_dense_eigs.txt"), "w") as f:
        f.write(f"# {w.name}: smallest 72 eigenvalues of H = -Laplacian_h + diag(V), N={w.N}, h={w.h}, seed={w.seed}\n")
        f.write("# dense LAPACK eigh of oracle.assemble_H (definition of the result, Section 2 eq. tracemin)\n")
        for x in ev:
            f.write(f"{x:.17e}\n")
    print("grid16_k64 done in %.1fs" % (time.time() - t))


def grid32_k256():
    w = wl.GRID32_K256
    V, X0 = wl.make_inputs(w)
    t = time.time()
    r = oracle.ppcg(V, w.N, w.h, w.k, w.sbsize, w.rr_period, X0, tol=w.tol, maxiter=5000)
    el = time.time() - t
    with open(os.path.join(HERE, "grid32_k256_oracle_eigs.txt"), "w") as f:
        f.write(f"# {w.name}: oracle PPCG (Algorithm 3), N={w.N}, k={w.k}, sbsize={w.sbsize}, rr_period={w.rr_period}, "
                f"tol={w.tol}, seed={w.seed}\n")
        f.write(f"# converged={r.converged} iters={r.iters} n_rr={r.n_rr} stats={r.stats} seconds={el:.1f}\n")
        f.write("# columns: Ritz value, residual norm ||H x - lambda x||\n")
        for lam, res in zip(r.lam, r.res):
            f.write(f"{lam:.17e} {res:.6e}\n")
    print("grid32_k256 done in %.1fs, iters %d" % (el, r.iters))


if __name__ == "__main__":
    which = sys.argv[1:] or ["grid16_k64", "grid32_k256"]
    if "grid16_k64" in which:
        grid16_k64()
    if "grid32_k256" in which:
        grid32_k256()

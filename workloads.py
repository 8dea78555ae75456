"""Seeded synthetic inputs for the PPCG eigensolver: potentials V and starting blocks X0.

This module is shared by the CPU oracle and the CUDA path. It holds none of the method's arithmetic:
it only draws random numbers and lays them out. The shapes follow the paper's setting (§6, Table "probs":
a Hermitian operator of order n_G ~ 2e5..2e6 and k ~ 2000 wanted eigenpairs) scaled to a real-space
stencil operator H = -Δ_h + diag(V) on an N x N x N periodic grid.

Layout: a grid function is a flat array of n = N^3 doubles with linear index p = i + N*j + N^2*l
(x fastest). A block of k vectors is an (n, k) array in Fortran (column-major) order.

Recipes (numpy default_rng with one seed per workload, 1001-1005; draw order: V, then X0):
  uniform      V_p ~ U[0, 1)
  wells        V = sum over w of -d_w * exp(-|r - c_w|^2 / (2 s_w^2)) + U[0, noise), with
               d_w ~ U[2, 6], s_w ~ U[2, 4] grid points, c_w ~ U[0, N)^3 and the periodic
               minimum-image distance |r - c|.
  separable    V(i, j, l) = V1(i) + V2(j) + V3(l), each V_d ~ U[0, 1)  (test-only recipe)
  zero         V = 0                                                  (test-only recipe)
X0 = standard_normal((n, k)) laid out column-major (real); complex X0 = real + 1j*imag from two draws.

The batched workload is a list of independent problems: from default_rng(1004) draw the 64 grid
sizes N_i ~ U{12..28} and then the 64 block sizes k_i ~ U{32..256}; problem i then draws V_i ~ U[0, 1) and its
X0_i from default_rng(1004 * 1000 + i) (V first, then X0).
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    N: int                 # grid points per axis (cubic grid)
    k: int                 # wanted eigenpairs
    sbsize: int            # sub-block size q
    rr_period: int = 5
    potential: str = "uniform"
    n_wells: int = 0
    noise: float = 0.1
    h: float = 1.0
    tol: float = 1e-8
    seed: int = 0
    dtype: str = "f64"     # "f64" real symmetric, "c128" complex Hermitian (Bloch)
    theta: tuple = (0.0, 0.0, 0.0)
    precision: str = "fp64"
    nbuf: int = 0          # buffer vectors (X gets k + nbuf columns; convergence is tested on the first k)

    @property
    def n(self) -> int:
        return self.N ** 3


# The workloads of the method's benchmark set: plain FP64 at two sizes, the mixed form at 48^3, and the complex
# Bloch recipe (its full 64^3, k = 2048 size does not converge within a benchmark run on one GPU, so it is also
# defined at smaller sizes: 48^3 with k = 512 and 32^3 with k = 128). The batched set is batch() below.
GRID16_K64 = Workload("grid16_k64_q1_uniform", N=16, k=64, sbsize=1, potential="uniform", seed=1001)
GRID32_K256 = Workload("grid32_k256_q4_wells8", N=32, k=256, sbsize=4, potential="wells", n_wells=8, seed=1002)
# nbuf = 50: the number of buffer vectors of every test in the paper's experiments (Section 6)
GRID48_K1024 = Workload("grid48_k1024_q8_wells32", N=48, k=1024, sbsize=8, potential="wells", n_wells=32,
                        seed=1003, precision="mixed", nbuf=50)
GRID64_K2048_BLOCH = Workload("grid64_k2048_q8_wells64_bloch", N=64, k=2048, sbsize=8, potential="wells",
                              n_wells=64, seed=1005, dtype="c128", theta=(0.3, 0.7, 1.1))
# the Bloch recipe at 48^3 with k = 512 and sbsize = 8: the wells keep the 64^3 recipe's density (64 x (48/64)^3 = 27)
GRID48_K512_BLOCH = Workload("grid48_k512_q8_wells27_bloch", N=48, k=512, sbsize=8, potential="wells", n_wells=27,
                             seed=1005, dtype="c128", theta=(0.3, 0.7, 1.1))
GRID32_K128_BLOCH = Workload("grid32_k128_q4_wells8_bloch", N=32, k=128, sbsize=4, potential="wells", n_wells=8,
                             seed=1005, dtype="c128", theta=(0.3, 0.7, 1.1))


def batch(count: int = 64, seed: int = 1004, n_range=(12, 28), k_range=(32, 256), sbsize: int = 4):
    """The batched workload: `count` independent uniform-potential problems of uneven size (64 problems, N in
    12..28, k in 32..256 with the defaults). Returns a list of Workloads; make_inputs(w) draws each problem's V
    and X0 from its own seed."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    ks = rng.integers(k_range[0], k_range[1] + 1, size=count)
    out = []
    for i in range(count):
        N, k = int(Ns[i]), int(ks[i])
        k = min(k, N ** 3 // 2)
        out.append(Workload(f"batch{seed}_{i}_grid{N}_k{k}", N=N, k=k, sbsize=min(sbsize, k), potential="uniform",
                            seed=seed * 1000 + i))
    return out


def potential(w: Workload, rng: np.random.Generator) -> np.ndarray:
    """Draw V (flat, length N^3, x fastest) for workload w from rng."""
    N = w.N
    if w.potential == "uniform":
        return rng.random(N ** 3)
    if w.potential == "zero":
        return np.zeros(N ** 3)
    if w.potential == "separable":
        v1, v2, v3 = rng.random(N), rng.random(N), rng.random(N)
        return (v1[:, None, None] + v2[None, :, None] + v3[None, None, :]).reshape(-1, order="F")
    if w.potential == "wells":
        ax = np.arange(N, dtype=np.float64)
        V = np.zeros((N, N, N))
        for _ in range(w.n_wells):
            depth = rng.uniform(2.0, 6.0)
            width = rng.uniform(2.0, 4.0)
            c = rng.uniform(0.0, N, size=3)
            d2 = np.zeros((N, N, N))
            for axis in range(3):
                d = ax - c[axis]
                d = d - N * np.round(d / N)          # minimum image
                shape = [1, 1, 1]
                shape[axis] = N
                d2 = d2 + (d * d).reshape(shape)
            V -= depth * np.exp(-d2 / (2.0 * width * width))
        V += rng.uniform(0.0, w.noise, size=(N, N, N))
        return V.reshape(-1, order="F")
    raise ValueError(f"unknown potential recipe {w.potential!r}")


def start_block(w: Workload, rng: np.random.Generator, ncols: int | None = None) -> np.ndarray:
    """Draw X0 (n x ncols, column-major; by default k + nbuf columns) for workload w from rng."""
    ncols = w.k + w.nbuf if ncols is None else ncols
    if w.dtype == "c128":
        re = rng.standard_normal((w.n, ncols))
        im = rng.standard_normal((w.n, ncols))
        return np.asfortranarray(re + 1j * im)
    return np.asfortranarray(rng.standard_normal((w.n, ncols)))


def make_inputs(w: Workload, ncols: int | None = None):
    """(V, X0) for workload w, drawn in the fixed order V then X0 from default_rng(w.seed)."""
    rng = np.random.default_rng(w.seed)
    V = potential(w, rng)
    X0 = start_block(w, rng, ncols)
    return V, X0


def small(name: str, N: int, k: int, sbsize: int, potential: str = "uniform", seed: int = 7, **kw) -> Workload:
    """A small workload for tests (sizes the oracle finishes in seconds)."""
    return Workload(name, N=N, k=k, sbsize=sbsize, potential=potential, seed=seed, **kw)

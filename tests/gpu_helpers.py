"""Helpers shared by the GPU tests: column-major blocks as torch tensors and a step-API handle."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1407_7506_gb300 as pk  # noqa: E402


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1407_7506_gb300 import build
    build.build()


def dev(A):
    """numpy (n, m) -> device tensor (m, n) holding the column-major block (ld = n)."""
    A = np.asarray(A, dtype=np.float64)
    if A.ndim == 1:
        A = A[:, None]
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda()


def host(T):
    """device tensor (m, n) -> numpy (n, m)."""
    torch.cuda.synchronize()
    return T.cpu().numpy().T.copy()


def ptr(t):
    return t.data_ptr() if t is not None else None


class Handle:
    """A ppcg handle used for the step-level entry points."""

    def __init__(self, V, N, kt, sbsize, nbuf=0, h=1.0, precision=0, fp64_gemm=0):
        self.V = torch.as_tensor(np.asarray(V, dtype=np.float64)).cuda()
        self.N, self.n = N, N ** 3
        op = pk.ppcg_operator(N, N, N, h, self.V.data_ptr(), (ctypes.c_double * 3)(0, 0, 0), 0)
        opt = pk.ppcg_options()
        opt.nbuf = nbuf
        opt.precision = precision
        opt.fp64_gemm = fp64_gemm
        nbytes = pk.ppcg_workspace_bytes(op, self.n, kt - nbuf, sbsize, opt)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.h = pk.ppcg_create(op, self.n, kt - nbuf, sbsize, 5, opt, torch.cuda.current_stream().cuda_stream,
                                self.ws.data_ptr(), nbytes)

    def close(self):
        if self.h:
            pk.ppcg_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

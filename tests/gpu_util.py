"""Helpers for the GPU parity tests: contexts on the current torch stream and
host/device transfers of complex fields."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def make_ctx(U, dims, m0, csw, **kw):
    torch = torch_cuda()
    from paper_2004_08146_gb300 import qcd
    ctx = qcd.Context(stream=torch.cuda.current_stream().cuda_stream, **kw)
    ctx.qcd_set_gauge(U, dims, m0, csw)
    return ctx


def dev(a, dtype=None):
    torch = torch_cuda()
    a = np.ascontiguousarray(a)
    if dtype is not None:
        a = a.astype(dtype)
    return torch.from_numpy(a.reshape(-1)).to("cuda")


def host(t):
    torch = torch_cuda()
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)

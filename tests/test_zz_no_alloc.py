"""The allocation-free variational-energy entry point, on the GPU.

nqs_variational_energy_noalloc is meant for callers that cannot allocate
device memory: code whose device memory is entirely owned by another
allocator, or that must keep device-wide synchronising allocation calls off
its hot path.  It keeps its partial sums in a fixed array inside the library
instead of a caller workspace.  These tests call it through the C ABI and
check it against nqs_variational_energy (the workspace form) on two calls in
a row, within the FP64 tolerance of the other parity tests.  The file is
named so that pytest collects it last.
"""

import ctypes
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


def _lib():
    import paper_2408_07625_gb300 as nqs
    lib = nqs.load_library()
    f = lib.nqs_variational_energy_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return nqs, lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _workspace_batch(nqs):
    """A staged one-sample batch: its workspace serves the workspace form."""
    ham = nqs.Hamiltonian(np.array([[0]], np.uint64), np.array([[1]], np.uint64), np.array([1.0]), 4)
    batch = nqs.Batch(ham, np.array([[3]], np.uint64))
    return ham, batch


def test_noalloc_matches_workspace_form_on_two_calls():
    nqs, lib = _lib()
    ham, batch = _workspace_batch(nqs)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(2024)
    # the second and later calls must not see an earlier call's partial sums;
    # 2^21 fills all 1024 partial-sum slots of the array, 2^21 - 1 leaves a ragged last one
    for n in (100_000, 777, 2 ** 21, 2 ** 21 - 1):
        a = torch.from_numpy(-2.0 * rng.integers(0, 5, n) + rng.normal(0.0, 0.3, n)).cuda()
        e = torch.from_numpy(rng.normal(50.0, 30.0, n)).cuda()
        want = torch.empty(3, dtype=torch.float64, device="cuda")
        got = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        assert lib.nqs_variational_energy(n, _p(a), _p(e), _p(batch.work), _p(want), stream) == 0
        assert lib.nqs_variational_energy_noalloc(n, _p(a), _p(e), _p(got), stream) == 0
        torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert abs(g[0] - w[0]) <= TOL64, (g, w)
        assert g[1] == w[1]
        assert abs(g[2] - w[2]) <= TOL64 * abs(w[2])
        # and the plain definition (Eq. variational_energy) in FP64 on the host
        an, en = a.cpu().numpy(), e.cpu().numpy()
        p = np.exp(2.0 * (an - an.max()))
        assert abs(g[0] - math.fsum(p * en) / math.fsum(p)) <= TOL64


def test_noalloc_rejects_batches_beyond_its_array():
    nqs, lib = _lib()
    n = 2 ** 21 + 1
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.full((3,), 7.0, dtype=torch.float64, device="cuda")
    rc = lib.nqs_variational_energy_noalloc(n, _p(a), _p(a), _p(out), None)
    torch.cuda.synchronize()
    assert rc == -4
    assert b"limit" in lib.nqs_last_error()
    assert torch.equal(out, torch.full((3,), 7.0, dtype=torch.float64, device="cuda"))

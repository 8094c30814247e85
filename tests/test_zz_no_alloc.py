"""The allocation-free entry point, idtx_cmi_ksg_noalloc, called through the C ABI.

Some callers cannot allocate device memory (their memory pool owns the
device, a cudaMalloc would synchronise the device on their path, or their
footprint must stay fixed after start-up).  This entry point serves them from
one fixed device array declared in the library.  These tests compare it with
the ordinary entry point, idtx_cmi_ksg, on two calls in a row (the array
keeps the previous call's contents, so the second call checks that nothing
stale leaks in), and check that a problem too large for the array is refused
with a clear error.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1807_10459_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_10459_gb300 as m
    from paper_1807_10459_gb300 import build
    build.build()
    lib = m.load()
    vp = ctypes.c_void_p
    lib.idtx_cmi_ksg_noalloc.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int,
                                         ctypes.c_int64, ctypes.c_int64,
                                         ctypes.POINTER(m.Settings), vp, vp]
    lib.idtx_cmi_ksg_noalloc.restype = ctypes.c_int
    return m, lib


def _noalloc(m, lib, x, y, z, k, n_surr, seed):
    n = x.shape[1]
    out = torch.empty(1 + n_surr, dtype=torch.float64, device="cuda")
    s = m.Settings(k, n_surr, seed, 0.05, 0, 0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.idtx_cmi_ksg_noalloc(x.data_ptr(), x.shape[0], y.data_ptr(), y.shape[0],
                                  None if z is None else z.data_ptr(),
                                  0 if z is None else z.shape[0], n, n, ctypes.byref(s),
                                  out.data_ptr(), stream)
    return rc, out


def test_matches_idtx_cmi_ksg_on_two_calls_in_a_row(lib):
    m, L = lib
    cases = [(synth.gaussian_problem(1000, 1, 1, 2, seed=41), 100, 7),
             (synth.gaussian_problem(3001, 2, 1, 3, seed=42), 40, 8)]
    for g, n_surr, seed in cases:
        x, y, z = (torch.from_numpy(a).cuda() for a in (g.x, g.y, g.z))
        rc, got = _noalloc(m, L, x, y, z, 4, n_surr, seed)
        assert rc == 0, L.idtx_last_error()
        ref = m.cmi_ksg(x, y, z, k=4, n_surr=n_surr, seed=seed)
        torch.cuda.synchronize()
        assert torch.max(torch.abs(got - ref)).item() < TOL


def test_refuses_a_problem_larger_than_its_scratch(lib):
    m, L = lib
    g = synth.gaussian_problem(60000, 1, 1, 2, seed=43)
    x, y, z = (torch.from_numpy(a).cuda() for a in (g.x, g.y, g.z))
    rc, _ = _noalloc(m, L, x, y, z, 4, 200, 1)
    assert rc == m.IDTX_EINVAL
    assert b"scratch" in L.idtx_last_error()
    # the entry point still works afterwards
    g = synth.gaussian_problem(500, 1, 1, 0, seed=44)
    x, y = torch.from_numpy(g.x).cuda(), torch.from_numpy(g.y).cuda()
    rc, got = _noalloc(m, L, x, y, None, 4, 10, 2)
    assert rc == 0
    ref = m.cmi_ksg(x, y, None, k=4, n_surr=10, seed=2)
    assert torch.max(torch.abs(got - ref)).item() < TOL

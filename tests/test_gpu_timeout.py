"""A bounded device wait that runs out returns IDTX_ETIMEOUT and leaves the
context usable (the time-out path of the C ABI's status codes).

The wait limit is set to 1 ns: the tile kernel's first wait for a staged
reference tile cannot finish in that time, so the call must report the
time-out; nothing waits without bound, and each aborting CTA still waits
for its own copies in flight before it exits.  The next call on the same
context, with the limit restored, must be oracle-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1807_10459_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def idtx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_10459_gb300 as m
    from paper_1807_10459_gb300 import build
    build.build()
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _exact(idtx, ctx, g, S, seed):
    cmi, eps, cnt = idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=4, n_surr=S, seed=seed,
                                 want_eps=True, want_counts=True, ctx=ctx)
    torch.cuda.synchronize()
    cmi, eps, cnt = cmi.cpu().numpy(), eps.cpu().numpy(), cnt.cpu().numpy()
    ref = oracle.cmi_surrogates(g.x, g.y, g.z, 4, S, seed)
    assert np.max(np.abs(cmi - ref)) < 1e-10
    n = g.x.shape[1]
    for s in (0, S):
        xs = g.x if s == 0 else g.x[:, oracle.perm(seed, s - 1, n)]
        e, a, b, c = oracle.ksg_counts(xs, g.y, g.z, 4)
        assert np.array_equal(eps[s], e)
        assert np.array_equal(cnt[s], np.stack([a, b, c]))


@pytest.mark.parametrize("batch", [False, True])
def test_tile_kernel_wait_runs_out_then_context_recovers(idtx, batch):
    g = synth.gaussian_problem(6000, 1, 1, 2, seed=61)
    S, seed = 40, 5
    ctx = idtx.Context(0)
    ctx.set_kernel(idtx.KERNEL_TILE)
    ctx.set_wait_limit_ns(1)
    with pytest.raises(idtx.IdtxError) as err:
        if batch:
            idtx.cmi_batch([dict(x=_dev(g.x), y=_dev(g.y), z=_dev(g.z), n_surr=S, seed=seed)],
                           k=4, ctx=ctx)
        else:
            idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=4, n_surr=S, seed=seed, ctx=ctx)
        torch.cuda.synchronize()
    assert err.value.code == idtx.IDTX_ETIMEOUT
    ctx.set_wait_limit_ns(0)
    _exact(idtx, ctx, g, S, seed)


def test_list_kernel_short_limit_is_exact_or_times_out(idtx):
    """The list kernel waits only when a warp's tile slot is still held; with
    a 1 ns bound a call either needs no such wait (and is exact) or reports
    the time-out -- and the context is exact afterwards either way."""
    g = synth.gaussian_problem(6000, 1, 1, 2, seed=62)
    S, seed = 40, 6
    ctx = idtx.Context(0)
    ctx.set_kernel(idtx.KERNEL_LIST)
    ctx.set_wait_limit_ns(1)
    try:
        _exact(idtx, ctx, g, S, seed)
    except idtx.IdtxError as e:
        assert e.code == idtx.IDTX_ETIMEOUT
    ctx.set_wait_limit_ns(0)
    _exact(idtx, ctx, g, S, seed)


def test_negative_limit_is_rejected(idtx):
    ctx = idtx.Context(0)
    with pytest.raises(idtx.IdtxError):
        ctx.set_wait_limit_ns(-1)

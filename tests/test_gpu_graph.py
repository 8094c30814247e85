"""CUDA-graph replay of idtx_cmi_batch: a repeated call with identical
arguments replays the captured graph and gives the same estimates as the
direct path, also after its inputs were overwritten in place and after other
calls used the context's scratch."""
import numpy as np
import pytest

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


def _probs(seed):
    shapes = [(600, 1, 1, 2), (900, 2, 1, 3), (300, 1, 2, 1)]
    return [synth.gaussian_problem(n, dx, dy, dz, seed=seed + i)
            for i, (n, dx, dy, dz) in enumerate(shapes)]


def _dev(probs, n_surr=7):
    return [dict(x=torch.from_numpy(p.x).cuda(), y=torch.from_numpy(p.y).cuda(),
                 z=torch.from_numpy(p.z).cuda(), n_surr=n_surr, seed=11 + i)
            for i, p in enumerate(probs)]


def _direct(idtx, dev):
    ctx = idtx.Context(0)
    return [o.cpu().numpy() for o in idtx.cmi_batch(dev, k=4, ctx=ctx)]


def _np(v):
    return v.cpu().numpy() if hasattr(v, "cpu") else v


def _same(a, b):
    return len(a) == len(b) and all(np.array_equal(_np(x), _np(y)) for x, y in zip(a, b))


def test_replay_matches_direct_path(idtx):
    dev = _dev(_probs(1))
    ref = _direct(idtx, dev)
    ctx = idtx.Context(0)
    ctx.set_graphs(True)
    first = idtx.cmi_batch(dev, k=4, ctx=ctx)          # captured
    launches = ctx.stats()["kernel_launches"]
    second = idtx.cmi_batch(dev, k=4, ctx=ctx)         # replayed: nothing enqueued by hand
    assert ctx.stats()["graph_launches"] == 2
    assert ctx.stats()["kernel_launches"] == launches
    assert _same(first, ref) and _same(second, ref)

    # new values in the same buffers: the replay computes on them
    new = _probs(50)
    for d, p in zip(dev, new):
        d["x"].copy_(torch.from_numpy(p.x))
        d["y"].copy_(torch.from_numpy(p.y))
        d["z"].copy_(torch.from_numpy(p.z))
    replay = idtx.cmi_batch(dev, k=4, ctx=ctx)
    assert ctx.stats()["graph_launches"] == 3
    assert _same(replay, _direct(idtx, dev))

    # another call on the context in between does not disturb the graph
    g = synth.gaussian_problem(1200, 1, 1, 4, seed=9)
    idtx.cmi_ksg(torch.from_numpy(g.x).cuda(), torch.from_numpy(g.y).cuda(),
                 torch.from_numpy(g.z).cuda(), k=4, n_surr=20, ctx=ctx)
    again = idtx.cmi_batch(dev, k=4, ctx=ctx)
    assert ctx.stats()["graph_launches"] == 4
    assert _same(again, replay)


def test_other_arguments_capture_a_new_graph(idtx):
    dev = _dev(_probs(2))
    ctx = idtx.Context(0)
    ctx.set_graphs(True)
    idtx.cmi_batch(dev, k=4, ctx=ctx)
    dev8 = _dev(_probs(2), n_surr=8)
    launches = ctx.stats()["kernel_launches"]
    out = idtx.cmi_batch(dev8, k=4, ctx=ctx)
    assert ctx.stats()["graph_launches"] == 2
    assert ctx.stats()["kernel_launches"] > launches   # a new capture enqueued the work
    assert _same(out, _direct(idtx, dev8))
    out = idtx.cmi_batch(dev, k=4, ctx=ctx)            # back to the first: recaptured
    assert _same(out, _direct(idtx, dev))


def test_profiling_and_disabling_bypass_graphs(idtx):
    dev = _dev(_probs(3))
    ctx = idtx.Context(0)
    ctx.set_graphs(True)
    ctx.set_profiling(True)
    idtx.cmi_batch(dev, k=4, ctx=ctx)
    assert ctx.stats()["graph_launches"] == 0
    ctx.set_profiling(False)
    ctx.set_graphs(False)
    out = idtx.cmi_batch(dev, k=4, ctx=ctx)
    assert ctx.stats()["graph_launches"] == 0
    assert _same(out, _direct(idtx, dev))

"""Network-inference variants the paper lists next to multivariate TE, through
the C ABI, against the oracle: bivariate TE of every source variable, and
multivariate MI inference (the greedy loop without target past).

Bar: estimates within 1e-10 nats, p-values and every decision identical.
"""
import numpy as np
import pytest

import oracle
from paper_1807_10459_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def idtx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_10459_gb300 as m
    from paper_1807_10459_gb300 import build
    build.build()
    return m


def _same(got, ref):
    (e1, p1), (e2, p2) = got, ref
    assert np.array_equal(np.isnan(p1), np.isnan(p2))
    ok = ~np.isnan(p2)
    assert np.array_equal(p1[ok], p2[ok])
    assert np.max(np.abs(e1[ok] - e2[ok])) < TOL
    assert np.all(np.isnan(e1[~ok]))


@pytest.mark.parametrize("n_past,lags", [(1, (1, 2)), (3, (1, 3)), (0, (1, 2)), (2, (2, 4))])
def test_bivariate_te_matches_oracle(idtx, n_past, lags):
    net = synth.var_network(n_nodes=5, order=3, T=900, density=0.4, weight=0.6, seed=31)
    for target in (0, 3):
        ref = oracle.bivariate_te(net.series, target, n_past, lags[0], lags[1], 4, 25, 9)
        got = idtx.bivariate_te(torch.from_numpy(net.series).cuda(), target, n_past, lags[0],
                                lags[1], k=4, n_surr=25, seed=9)
        _same(got, ref)


def test_bivariate_te_host_series_and_both_kernels(idtx):
    net = synth.var_network(n_nodes=4, order=2, T=1500, density=0.5, weight=0.6, seed=4)
    ref = oracle.bivariate_te(net.series, 1, 2, 1, 2, 4, 20, 3)
    for kern in (idtx.KERNEL_TILE, idtx.KERNEL_LIST):
        ctx = idtx.Context(0)
        ctx.set_kernel(kern)
        _same(idtx.bivariate_te(net.series, 1, 2, 1, 2, k=4, n_surr=20, seed=3, ctx=ctx), ref)


def test_multivariate_mi_inference_matches_oracle(idtx):
    """Multivariate MI network inference is the greedy loop with no target
    past: the first step is an MI (no conditioning), later steps condition on
    the selected sources only."""
    net = synth.var_network(n_nodes=5, order=2, T=1000, density=0.5, weight=0.6, seed=14)
    kw = dict(k=4, n_surr=20, alpha=0.05, seed=6, max_parents=4)
    for target in (1, 4):
        ref = oracle.select_target(net.series, target, 0, 1, 2, **kw)
        got = idtx.mte_select_target(net.series, target, 0, 1, 2, **kw)
        assert got["parents"] == ref["parents"]
        assert [s[:2] for s in got["steps"]] == [s[:2] for s in ref["steps"]]
        assert [s[3] for s in got["steps"]] == [s[3] for s in ref["steps"]]
        for a, b in zip(got["steps"], ref["steps"]):
            assert abs(a[2] - b[2]) < TOL


def test_bivariate_te_rejects_bad_arguments(idtx):
    net = synth.var_network(n_nodes=3, order=2, T=300, seed=2)
    with pytest.raises(idtx.IdtxError):
        idtx.bivariate_te(net.series[:1], 0, 1, 1, 2)       # no source process
    with pytest.raises(idtx.IdtxError):
        idtx.bivariate_te(net.series, 5, 1, 1, 2)           # target out of range


def _steps_equal(got, ref):
    assert [s[:2] for s in got] == [s[:2] for s in ref]
    assert [s[3] for s in got] == [s[3] for s in ref]
    for a, b in zip(got, ref):
        assert abs(a[2] - b[2]) < TOL


def test_target_past_selection_matches_oracle(idtx):
    net = synth.var_network(n_nodes=4, order=3, T=1200, density=0.5, weight=0.6, seed=23)
    kw = dict(k=4, n_surr=20, alpha=0.05, seed=3)
    for target in (0, 2):
        ref = oracle.select_past(net.series, target, 1, 4, max_past=4, **kw)
        got = idtx.mte_select_past(torch.from_numpy(net.series).cuda(), target, 1, 4,
                                   max_past=4, **kw)
        assert got["past"] == ref["past"]
        _steps_equal(got["steps"], ref["steps"])
        # then the sources, from that (non-uniform) past
        ref_s = oracle.select_sources(net.series, target, ref["past"], 1, 4, max_parents=4, **kw)
        got_s = idtx.mte_select_sources(net.series, target, got["past"], 1, 4, max_parents=4,
                                        **kw)
        assert got_s["parents"] == ref_s["parents"]
        _steps_equal(got_s["steps"], ref_s["steps"])


def test_sources_from_a_uniform_past_equal_select_target(idtx):
    net = synth.var_network(n_nodes=4, order=3, T=900, density=0.5, weight=0.6, seed=17)
    kw = dict(k=4, n_surr=15, alpha=0.05, seed=8, max_parents=4)
    for target, n_past in ((0, 2), (3, 3)):
        a = idtx.mte_select_target(net.series, target, n_past, 1, 3, **kw)
        past = [target * 3 + lag - 1 for lag in range(1, n_past + 1)]
        b = idtx.mte_select_sources(net.series, target, past, 1, 3, **kw)
        assert a["parents"] == b["parents"]
        assert [tuple(s) for s in a["steps"]] == [tuple(s) for s in b["steps"]]


@pytest.mark.parametrize("n,reps,dims", [(600, 20, (1, 1, 2)), (1000, 50, (2, 1, 3)),
                                         (240, 240, (1, 1, 1)), (3000, 60, (1, 1, 2))])
def test_replication_surrogates_match_oracle(idtx, n, reps, dims):
    g = synth.gaussian_problem(n, *dims, seed=n + reps)
    ref = oracle.cmi_surrogates_reps(g.x, g.y, g.z, 4, 12, 5, n_reps=reps)
    for kern in (idtx.KERNEL_TILE, idtx.KERNEL_LIST):
        ctx = idtx.Context(0)
        ctx.set_kernel(kern)
        got = idtx.cmi_ksg(torch.from_numpy(g.x).cuda(), torch.from_numpy(g.y).cuda(),
                           torch.from_numpy(g.z).cuda(), k=4, n_surr=12, seed=5, n_reps=reps,
                           ctx=ctx).cpu().numpy()
        assert np.max(np.abs(got - ref)) < TOL
    if reps == n:    # one sample per replication: the sample-level surrogates
        plain = idtx.cmi_ksg(g.x, g.y, g.z, k=4, n_surr=12, seed=5)
        assert np.array_equal(plain, idtx.cmi_ksg(g.x, g.y, g.z, k=4, n_surr=12, seed=5,
                                                  n_reps=reps))


def test_replication_count_must_divide_n(idtx):
    g = synth.gaussian_problem(300, 1, 1, 1, seed=1)
    with pytest.raises(idtx.IdtxError):
        idtx.cmi_ksg(g.x, g.y, g.z, k=4, n_surr=3, n_reps=7)

"""Tests after the greedy selection (pruning by the minimum statistic, omnibus
test, sequential maximum statistic) through the C ABI, against the oracle.

Bar: every decision (kept parents, significance, removal order) identical to
the oracle's; every statistic within 1e-10 nats; p-values equal (counts of
surrogates, compared in fp64 on both sides).
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


def _driven_system(T=1500, seed=3):
    """Node 0 driven at lag 1 by nodes 1 and 2; nodes 3, 4, 5 independent."""
    rng = np.random.default_rng(seed)
    x = np.zeros((6, T + 100))
    e = rng.standard_normal((6, T + 100))
    for t in range(1, T + 100):
        x[1, t] = 0.5 * x[1, t - 1] + e[1, t]
        x[2, t] = 0.5 * x[2, t - 1] + e[2, t]
        x[3:, t] = e[3:, t]
        x[0, t] = 0.3 * x[0, t - 1] + 0.6 * x[1, t - 1] + 0.6 * x[2, t - 1] + 0.5 * e[0, t]
    x = x[:, 100:]
    x = (x - x.mean(axis=1, keepdims=True)) / x.std(axis=1, keepdims=True)
    return x.astype(np.float32)


POST = dict(target=0, n_past=1, min_lag=1, max_lag=1, k=4, n_surr=40, alpha=0.05, seed=11)


def _ctx(idtx, kernel):
    ctx = idtx.Context(0)
    ctx.set_kernel(kernel)
    return ctx


@pytest.mark.parametrize("parents", [[1, 3, 2], [3, 4, 5], [2, 1], [4]])
def test_prune_matches_oracle(idtx, parents):
    s = _driven_system()
    ref = oracle.prune(s, parents=parents, **POST)
    for kern in (idtx.KERNEL_AUTO, idtx.KERNEL_TILE, idtx.KERNEL_LIST):
        got = idtx.mte_prune(torch.from_numpy(s).cuda(), parents=parents, ctx=_ctx(idtx, kern),
                             **POST)
        assert got["kept"] == ref["kept"]
        assert len(got["rounds"]) == len(ref["rounds"])
        for a, b in zip(got["rounds"], ref["rounds"]):
            assert (a[0], a[1], a[3]) == (b[0], b[1], b[3])
            assert abs(a[2] - b[2]) < TOL


@pytest.mark.parametrize("parents", [[1, 2], [3, 4], [1, 2, 3, 4], [5]])
def test_omnibus_matches_oracle(idtx, parents):
    s = _driven_system()
    ref = oracle.omnibus(s, parents=parents, **POST)
    got = idtx.mte_omnibus(torch.from_numpy(s).cuda(), parents=parents, **POST)
    assert got[1:] == ref[1:]
    assert abs(got[0] - ref[0]) < TOL
    # host series give the same result
    assert idtx.mte_omnibus(s, parents=parents, **POST) == got


@pytest.mark.parametrize("parents", [[1, 3, 2], [4, 5], [2]])
def test_seqmax_matches_oracle(idtx, parents):
    s = _driven_system()
    r_stats, r_p, r_sig = oracle.seqmax(s, parents=parents, **POST)
    for kern in (idtx.KERNEL_TILE, idtx.KERNEL_LIST):
        stats, p, sig = idtx.mte_seqmax(torch.from_numpy(s).cuda(), parents=parents,
                                        ctx=_ctx(idtx, kern), **POST)
        assert np.max(np.abs(stats - r_stats)) < TOL
        assert np.array_equal(p, r_p) and np.array_equal(sig, r_sig)


def test_selection_then_pruning_on_a_var_network(idtx):
    """The greedy loop, then pruning of what it selected, both against the oracle."""
    net = synth.var_network(n_nodes=5, order=2, T=1200, density=0.5, weight=0.6, seed=12)
    kw = dict(k=4, n_surr=20, alpha=0.05, seed=7)
    for target in (0, 2):
        sel = idtx.mte_select_target(net.series, target, 1, 1, 2, max_parents=5, **kw)
        ref_sel = oracle.select_target(net.series, target, 1, 1, 2, max_parents=5, **kw)
        assert sel["parents"] == ref_sel["parents"]
        if not sel["parents"]:
            continue
        got = idtx.mte_prune(net.series, target, 1, 1, 2, sel["parents"], **kw)
        ref = oracle.prune(net.series, target, 1, 1, 2, sel["parents"], **kw)
        assert got["kept"] == ref["kept"]
        assert [r[:2] for r in got["rounds"]] == [r[:2] for r in ref["rounds"]]


def test_bad_parent_lists_are_rejected(idtx):
    s = _driven_system(T=300)
    d = torch.from_numpy(s).cuda()
    bad = [dict(parents=[0]),              # the target's own lag 1 (target past)
           dict(parents=[1, 1]),           # repeated
           dict(parents=[7]),              # out of range
           dict(parents=[])]
    for b in bad:
        with pytest.raises(idtx.IdtxError):
            idtx.mte_prune(d, **dict(POST, **b))
    with pytest.raises(idtx.IdtxError):      # more parents than the omnibus kernel's X columns
        idtx.mte_omnibus(d, **dict(POST, parents=[1, 2, 3, 4, 5]))


@pytest.mark.slow
def test_full_size_post_selection_sampled(idtx):
    """The benchmarked network (10-node VAR(5), T=10000, target 0, history 3,
    lags 1..5, k=4, 200 surrogates): after the greedy selection, the
    leave-one-out statistic of every selected parent against the oracle's
    estimate (N = 9995)."""
    net = synth.var_network()
    s = torch.from_numpy(net.series).cuda()
    kw = dict(k=4, n_surr=200, alpha=0.05, seed=20181029)
    par = idtx.mte_select_target(s, 0, 3, 1, 5, max_parents=10, **kw)["parents"]
    assert len(par) >= 1
    stats, pvals, sig = idtx.mte_seqmax(s, 0, 3, 1, 5, par, **kw)
    L, T = 5, net.series.shape[1]
    col = lambda c: net.series[c // 5, L - (1 + c % 5):T - (1 + c % 5)]
    y = net.series[0, L:]
    past = [net.series[0, L - lag:T - lag] for lag in (1, 2, 3)]
    for i, c in enumerate(par):
        z = np.stack(past + [col(d) for j, d in enumerate(par) if j != i])
        assert abs(stats[i] - oracle.cmi_ksg(col(c)[None, :], y, z, 4)) < TOL

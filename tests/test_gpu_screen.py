"""GPU tests of the learned screen: its forward pass and gradient against the
fp64 oracle on the same bf16-rounded weights, deterministic training, and the
screened greedy step against the exact (batched) step."""
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


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 10)).astype(np.float32)
    x[:, 1] = 8.0 + rng.random(n)             # ln N-like column with a large offset
    t = (np.tanh(x[:, 0]) + 0.3 * x[:, 6] * x[:, 8] + 0.1 * x[:, 1]).astype(np.float32)
    return x, t


def _screen(idtx, seed):
    rng = np.random.default_rng(seed)
    sc = idtx.Screen(seed=seed)
    sc.params[:] += (rng.standard_normal(sc.params.size) * 0.05).astype(np.float32)
    sc.feat_mean[:] = np.array([0, 8.5, 0, 0, 0, 0, 0, 0, 0, 0], np.float32)
    sc.feat_scale[:] = np.array([1, 3.0, 1, 1, 1, 1, 1, 1, 1, 1], np.float32)
    return sc


def test_forward_matches_oracle(idtx):
    sc = _screen(idtx, 1)
    x, _ = _data(300, 2)
    got = idtx.screen_predict(sc, x)
    ref = oracle.mlp_forward(sc.params, 10, 64, sc.feat_mean, sc.feat_scale, x, bf16=True)
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("quantile", [0.0, 0.95])
def test_gradient_matches_oracle(idtx, quantile):
    sc = _screen(idtx, 3)
    x, t = _data(257, 4)
    loss, g = idtx.screen_loss_grad(sc, x, t, quantile=quantile)
    rl, rg = oracle.mlp_loss_grad(sc.params, 10, 64, sc.feat_mean, sc.feat_scale, x, t,
                                  bf16=True, quantile=quantile)
    assert abs(loss - rl) <= 1e-5 * max(1.0, rl)
    assert np.max(np.abs(g - rg)) <= 1e-4 * max(1.0, np.max(np.abs(rg)))


def test_training_lowers_the_loss_and_is_deterministic(idtx):
    x, t = _data(3000, 5)
    a = idtx.Screen(seed=7)
    b = idtx.Screen(seed=7)
    l0, _ = idtx.screen_loss_grad(a, x, t)
    la = idtx.screen_train(a, x, t, epochs=40, batch=128, lr=3e-3, seed=11)
    lb = idtx.screen_train(b, x, t, epochs=40, batch=128, lr=3e-3, seed=11)
    assert la < 0.2 * l0
    assert la == lb and np.array_equal(a.params, b.params)
    # the loss the trainer reports is the oracle's loss of the trained parameters
    rl, _ = oracle.mlp_loss_grad(a.params, 10, 64, a.feat_mean, a.feat_scale, x, t, bf16=True)
    assert abs(la - rl) <= 1e-5 * max(1.0, rl)


def _net():
    return synth.var_network(n_nodes=5, order=3, T=900, density=0.4, weight=0.6, seed=21)


def test_screened_step_keeping_everything_equals_exact(idtx):
    net = _net()
    ctx = idtx.Context(0)
    sc = idtx.Screen(delta=1e30, s0=4)
    idtx.screen_set(sc, ctx=ctx)
    args = (torch.from_numpy(net.series).cuda(), 0, 2, 1, 3, (), 0)
    ex, e_est = idtx.mte_step(*args, k=4, n_surr=30, seed=3, want_estimates=True, ctx=ctx)
    sr, s_est = idtx.mte_step(*args, k=4, n_surr=30, seed=3, want_estimates=True,
                              mode=idtx.MODE_SCREENED, ctx=ctx)
    assert tuple(sr) == tuple(ex)
    assert sr.n_full == sr.n_cand == ex.n_cand
    ok = ~np.isnan(e_est[:, 0])
    assert np.max(np.abs(e_est[ok] - s_est[ok])) < 1e-10


def test_screened_step_skipping_everything_uses_only_cheap_surrogates(idtx):
    net = _net()
    ctx = idtx.Context(0)
    idtx.screen_set(idtx.Screen(delta=-1e30, s0=5), ctx=ctx)
    args = (torch.from_numpy(net.series).cuda(), 0, 2, 1, 3, (), 0)
    ex, e_est = idtx.mte_step(*args, k=4, n_surr=30, seed=3, want_estimates=True, ctx=ctx)
    sr, s_est = idtx.mte_step(*args, k=4, n_surr=30, seed=3, want_estimates=True,
                              mode=idtx.MODE_SCREENED, ctx=ctx)
    assert sr.n_full == 0
    ok = ~np.isnan(e_est[:, 0])
    assert np.max(np.abs(e_est[ok][:, :6] - s_est[ok][:, :6])) < 1e-10
    assert np.all(np.isnan(s_est[ok][:, 6:]))
    # the count only sees the cheap surrogates, over all candidates
    t_obs = e_est[ok][:, 0].max()
    cnt = np.count_nonzero(e_est[ok][:, 1:6].max(axis=0) >= t_obs)
    assert sr[3] == cnt / 30 and sr[0] == ex[0] and abs(sr[2] - ex[2]) < 1e-12


def test_screened_step_with_a_sound_screen_agrees_with_exact(idtx):
    """A screen whose bound holds for every candidate it skips must reproduce the
    exact decision.  With an all-zero network the bound is cheap maximum + delta;
    delta just above the largest excess of a candidate's surrogate maximum over
    its cheap maximum makes it sound."""
    net = _net()
    ctx = idtx.Context(0)
    args = (torch.from_numpy(net.series).cuda(), 0, 2, 1, 3, (), 0)
    ex, e_est = idtx.mte_step(*args, k=4, n_surr=30, seed=3, want_estimates=True, ctx=ctx)
    ok = np.flatnonzero(~np.isnan(e_est[:, 0]))
    cheap = e_est[ok, 1:5].max(axis=1)
    excess = e_est[ok, 1:].max(axis=1) - cheap
    t_obs = e_est[ok, 0].max()
    delta = float(excess.max()) + 1e-6
    sc = idtx.Screen(params=np.zeros(idtx.SCREEN_NPARAMS, np.float32), s0=4, delta=delta)
    idtx.screen_set(sc, ctx=ctx)
    sr = idtx.mte_step(*args, k=4, n_surr=30, seed=3, mode=idtx.MODE_SCREENED, ctx=ctx)
    assert (sr[0], sr[1], sr[3]) == (ex[0], ex[1], ex[3])
    assert sr.n_full == int(np.count_nonzero(cheap + np.float32(delta) >= t_obs))


def test_screened_step_stops_early_on_a_non_significant_step(idtx):
    rng = np.random.default_rng(8)
    series = rng.standard_normal((4, 1200)).astype(np.float32)   # no coupling at all
    ctx = idtx.Context(0)
    idtx.screen_set(idtx.Screen(delta=1e30, s0=4), ctx=ctx)      # keep every candidate
    args = (torch.from_numpy(series).cuda(), 0, 1, 1, 3, (), 0)
    ex = idtx.mte_step(*args, k=4, n_surr=100, seed=5, ctx=ctx)
    sr, s_est = idtx.mte_step(*args, k=4, n_surr=100, seed=5, want_estimates=True,
                              mode=idtx.MODE_SCREENED, ctx=ctx)
    assert not ex[1] and not sr[1]                               # same decision
    assert sr[0] == ex[0] and abs(sr[2] - ex[2]) < 1e-12
    assert sr.surr_done < 100                                   # stopped early
    assert 0.05 <= sr[3] <= ex[3]                               # a deciding lower bound
    ok = ~np.isnan(s_est[:, 0])
    assert np.all(np.isnan(s_est[ok][:, 1 + sr.surr_done:]))
    assert ex.surr_done == 100


@pytest.mark.slow
def test_trained_screen_gains_over_the_network_free_rule(idtx):
    """The shipped screen against the method without it: exact mode (every
    candidate gets every surrogate) and the network-free bound (cheap maximum
    plus a constant margin, calibrated the same way).  On a 20-node VAR(3)
    network drawn with seeds unseen in training, all three give the same parent
    sets, and the trained screen sends fewer candidates to full surrogates
    than the network-free rule."""
    import os
    path = os.path.join(os.path.dirname(idtx.__file__), "screen_weights.npz")
    trained = idtx.Screen.load(path)
    free = idtx.Screen(params=np.zeros(idtx.SCREEN_NPARAMS, np.float32), s0=trained.s0,
                       delta=float(trained.meta["network_free_margin"]))
    net = synth.var_network_indegree(n_nodes=20, order=3, indegree=3, T=5000, seed=424242)
    s = torch.from_numpy(net.series).cuda()
    ctx_t, ctx_f = idtx.Context(0), idtx.Context(0)
    idtx.screen_set(trained, ctx=ctx_t)
    idtx.screen_set(free, ctx=ctx_f)
    kw = dict(k=4, n_surr=200, alpha=0.05, seed=77, max_parents=6)
    full_t = full_f = 0
    for t in range(0, 20, 2):
        ex = idtx.mte_select_target(s, t, 3, 1, 3, ctx=ctx_t, **kw)
        tr = idtx.mte_select_target(s, t, 3, 1, 3, mode=idtx.MODE_SCREENED, ctx=ctx_t, **kw)
        fr = idtx.mte_select_target(s, t, 3, 1, 3, mode=idtx.MODE_SCREENED, ctx=ctx_f, **kw)
        assert tr["parents"] == ex["parents"] == fr["parents"]
        full_t += sum(st.n_full for st in tr["steps"])
        full_f += sum(st.n_full for st in fr["steps"])
    assert full_t < full_f


def _shipped(idtx, ext):
    import os
    return os.path.join(os.path.dirname(idtx.__file__), "screen_weights" + ext)


def test_screen_loaded_from_file_through_the_c_abi(idtx):
    """idtx_screen_load of the shipped flat file installs the same screen as
    idtx_screen_set of the trained parameters: a screened step gives the same
    decision, statistic, p-value, kept candidates and estimates."""
    net = synth.var_network(n_nodes=6, order=3, T=3000, density=0.4, weight=0.5, seed=31)
    args = (torch.from_numpy(net.series).cuda(), 0, 3, 1, 3, (), 0)
    kw = dict(k=4, n_surr=200, seed=9, want_estimates=True, mode=idtx.MODE_SCREENED)
    c_file, c_set = idtx.Context(0), idtx.Context(0)
    idtx.screen_load(_shipped(idtx, ".bin"), ctx=c_file)
    idtx.screen_set(idtx.Screen.load(_shipped(idtx, ".npz")), ctx=c_set)
    a, ea = idtx.mte_step(*args, ctx=c_file, **kw)
    b, eb = idtx.mte_step(*args, ctx=c_set, **kw)
    assert tuple(a) == tuple(b) and a.n_full == b.n_full and a.surr_done == b.surr_done
    assert np.array_equal(np.isnan(ea), np.isnan(eb))
    ok = ~np.isnan(ea)
    assert np.array_equal(ea[ok], eb[ok])


def test_bad_screen_files_are_rejected_and_leave_the_screen(idtx, tmp_path):
    good = open(_shipped(idtx, ".bin"), "rb").read()
    ctx = idtx.Context(0)
    idtx.screen_load(_shipped(idtx, ".bin"), ctx=ctx)
    for name, data in (("short", good[:-4]), ("long", good + b"\0"),
                       ("magic", b"IDTXSCR2" + good[8:]), ("missing", None)):
        path = tmp_path / name
        if data is not None:
            path.write_bytes(data)
        with pytest.raises(idtx.IdtxError) as err:
            idtx.screen_load(str(path), ctx=ctx)
        assert err.value.code == idtx.IDTX_EINVAL
    # the installed screen still works (screened step runs)
    net = _net()
    idtx.mte_step(torch.from_numpy(net.series).cuda(), 0, 2, 1, 3, (), 0, k=4, n_surr=30,
                  seed=3, mode=idtx.MODE_SCREENED, ctx=ctx)


def test_screen_features_follow_the_header_definition(idtx):
    """The features the screened step computes (idtx_screen_features, also the
    training features) against the definition in idtx.h written out in numpy:
    (I_c, ln N, dx, dy, dz, k, mean, std (divisor s0), max of the first s0
    surrogate estimates, ln n_surr)."""
    net = _net()
    s0, n_surr, n = 8, 30, 900 - 3
    _, est = idtx.mte_step(torch.from_numpy(net.series).cuda(), 0, 2, 1, 3, (), 0, k=4,
                           n_surr=n_surr, seed=3, want_estimates=True)
    rows = est[~np.isnan(est[:, 0])]
    got = idtx.screen_features(rows, n, 2, 4, n_surr, s0)
    cheap = rows[:, 1:1 + s0]
    ref = np.stack([rows[:, 0], np.full(len(rows), np.log(n)), np.ones(len(rows)),
                    np.ones(len(rows)), np.full(len(rows), 2.0), np.full(len(rows), 4.0),
                    cheap.mean(axis=1), cheap.std(axis=1), cheap.max(axis=1),
                    np.full(len(rows), np.log(n_surr))], axis=1).astype(np.float32)
    exact_cols = [0, 1, 2, 3, 4, 5, 8, 9]
    assert np.array_equal(got[:, exact_cols], ref[:, exact_cols])
    assert np.allclose(got[:, 6:8], ref[:, 6:8], rtol=1e-6, atol=1e-9)

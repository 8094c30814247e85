"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bar (the estimator's definition fixes it): eps_i bit-exact, every neighbour
count exact, every estimate within 1e-10 nats (different fp64 summation order),
greedy decisions identical.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _oracle_all(x, y, z, k, S, seed):
    """eps/counts/cmi of the original and every surrogate, by the oracle."""
    n = x.shape[1]
    eps, cnt, cmi = [], [], []
    for s in range(S + 1):
        xs = x if s == 0 else x[:, oracle.perm(seed, s - 1, n)]
        e, a, b, c = oracle.ksg_counts(xs, y, z, k)
        eps.append(e)
        cnt.append(np.stack([a, b, c]))
        cmi.append(oracle.cmi_ksg(xs, y, z, k))
    return np.array(eps), np.array(cnt), np.array(cmi)


def _check_problem(idtx, x, y, z, k, S, seed, on_device=True):
    args = (_dev(x), _dev(y), None if z is None else _dev(z)) if on_device else (x, y, z)
    cmi, eps, cnt = idtx.cmi_ksg(*args, k=k, n_surr=S, seed=seed, want_eps=True,
                                 want_counts=True)
    if on_device:
        torch.cuda.synchronize()
        cmi, eps, cnt = cmi.cpu().numpy(), eps.cpu().numpy(), cnt.cpu().numpy()
    e_ref, c_ref, m_ref = _oracle_all(x, y, z, k, S, seed)
    assert np.array_equal(eps, e_ref), "eps differs"
    assert np.array_equal(cnt, c_ref), "counts differ"
    assert np.max(np.abs(cmi - m_ref)) < TOL
    return cmi


def test_config1_full(idtx):
    """Single problem N=1000, dims 1/1/2, k=4, 100 surrogates: every estimate."""
    g = synth.gaussian_problem(1000, 1, 1, 2)
    _check_problem(idtx, g.x, g.y, g.z, 4, 100, 20181028)


@pytest.mark.parametrize("n", [2, 5, 127, 128, 129, 300, 515])
def test_ragged_sizes(idtx, n):
    g = synth.gaussian_problem(n, 1, 1, 2, seed=n)
    _check_problem(idtx, g.x, g.y, g.z, min(4, n - 1), 3, 7)


@pytest.mark.parametrize("dims", [(1, 1, 0), (2, 1, 1), (1, 2, 3), (2, 2, 5), (1, 1, 7),
                                  (1, 1, 10), (2, 2, 16), (3, 1, 2), (1, 4, 4), (4, 4, 16)])
def test_dimension_buckets(idtx, dims):
    dx, dy, dz = dims
    g = synth.gaussian_problem(400, dx, dy, dz, seed=sum(dims))
    _check_problem(idtx, g.x, g.y, g.z if dz else None, 4, 17, 3)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 15])
def test_other_k(idtx, k):
    g = synth.gaussian_problem(333, 1, 1, 2, seed=k)
    _check_problem(idtx, g.x, g.y, g.z, k, 4, 11)


def test_ties_and_duplicates(idtx):
    rng = np.random.default_rng(5)
    x = rng.integers(0, 4, (1, 260)).astype(np.float32)
    y = rng.integers(0, 4, (1, 260)).astype(np.float32)
    z = rng.integers(0, 3, (2, 260)).astype(np.float32)
    for k in (1, 4, 8):
        _check_problem(idtx, x, y, z, k, 3, 1)


def test_host_pointers_match_device(idtx):
    g = synth.gaussian_problem(700, 1, 1, 2, seed=3)
    a = _check_problem(idtx, g.x, g.y, g.z, 4, 6, 5, on_device=False)
    b = idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=4, n_surr=6, seed=5).cpu().numpy()
    assert np.array_equal(a, b)


def test_deterministic(idtx):
    g = synth.gaussian_problem(2000, 1, 1, 3, seed=9)
    a = idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=4, n_surr=40, seed=1).cpu().numpy()
    b = idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=4, n_surr=40, seed=1).cpu().numpy()
    assert np.array_equal(a, b)


def test_nonfinite_input_is_rejected_and_context_survives(idtx):
    g = synth.gaussian_problem(200, 1, 1, 2, seed=4)
    bad = g.z.copy()
    bad[1, 17] = np.nan
    with pytest.raises(idtx.IdtxError) as ei:
        idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(bad), k=4, n_surr=2, seed=1)
    assert ei.value.code == idtx.IDTX_EINVAL
    with pytest.raises(idtx.IdtxError):
        idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=200, n_surr=2, seed=1)
    _check_problem(idtx, g.x, g.y, g.z, 4, 2, 1)


def test_plain_mode_matches_batched_and_oracle(idtx):
    g = synth.gaussian_problem(700, 1, 1, 3, seed=21)
    args = (_dev(g.x), _dev(g.y), _dev(g.z))
    plain = idtx.cmi_ksg(*args, k=4, n_surr=9, seed=3, mode=idtx.MODE_PLAIN).cpu().numpy()
    batched = idtx.cmi_ksg(*args, k=4, n_surr=9, seed=3).cpu().numpy()
    ref = oracle.cmi_surrogates(g.x, g.y, g.z, 4, 9, 3)
    assert np.max(np.abs(plain - ref)) < TOL
    assert np.max(np.abs(plain - batched)) < TOL
    g = synth.gaussian_problem(300, 2, 2, 0, seed=22)
    plain = idtx.cmi_ksg(_dev(g.x), _dev(g.y), None, k=7, n_surr=3, seed=4,
                         mode=idtx.MODE_PLAIN).cpu().numpy()
    assert np.max(np.abs(plain - oracle.cmi_surrogates(g.x, g.y, None, 7, 3, 4))) < TOL


@pytest.mark.parametrize("n,dims,k", [(129, (1, 1, 2), 4), (700, (2, 1, 4), 1),
                                      (333, (3, 2, 5), 6), (515, (1, 2, 16), 4)])
def test_plain_mode_buckets_match_oracle(idtx, n, dims, k):
    """The plain schedule (one launch per estimate) in the k = 4 buckets and the
    runtime-k one, ragged N: estimates against the oracle."""
    g = synth.gaussian_problem(n, *dims, seed=n + k)
    plain = idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=k, n_surr=5, seed=8,
                         mode=idtx.MODE_PLAIN).cpu().numpy()
    assert np.max(np.abs(plain - oracle.cmi_surrogates(g.x, g.y, g.z, k, 5, 8))) < TOL


def test_plain_greedy_step_matches_batched(idtx):
    net = synth.var_network(n_nodes=4, order=2, T=500, density=0.5, weight=0.6, seed=5)
    a, ea = idtx.mte_step(_dev(net.series), 1, 1, 1, 2, (), 0, k=4, n_surr=10, seed=2,
                          want_estimates=True)
    b, eb = idtx.mte_step(_dev(net.series), 1, 1, 1, 2, (), 0, k=4, n_surr=10, seed=2,
                          want_estimates=True, mode=idtx.MODE_PLAIN)
    ok = ~np.isnan(ea[:, 0])
    assert np.max(np.abs(ea[ok] - eb[ok])) < TOL
    assert a[0] == b[0] and a[1] == b[1] and a[3] == b[3]


def test_unknown_mode_is_rejected(idtx):
    g = synth.gaussian_problem(100, 1, 1, 1, seed=1)
    with pytest.raises(idtx.IdtxError):
        idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=4, n_surr=1, mode=7)


def test_batch_uneven(idtx):
    probs = synth.batch_problems(n_probs=6, n_min=150, n_max=900, n_surr=5, dz_max=8, seed=77)
    out = idtx.cmi_batch([dict(x=_dev(p.x), y=_dev(p.y), z=_dev(p.z), n_surr=p.n_surr,
                               seed=p.seed) for p in probs], k=4)
    for p, o in zip(probs, out):
        ref = oracle.cmi_surrogates(p.x, p.y, p.z, 4, p.n_surr, p.seed)
        assert np.max(np.abs(o.cpu().numpy() - ref)) < TOL


@pytest.mark.parametrize("k", [4, 3])
def test_batch_is_one_launch_per_variant_and_equals_separate_calls(idtx, k):
    """A batch runs as one persistent fused launch per kernel variant; every
    estimate equals the one a separate call gives, bit for bit (same per-CTA
    arithmetic, same fixed-order sums).  Sizes include query tiles made only
    of padding (N mod 128 < 64) and problems sharing a variant."""
    shapes = [(700, 1, 1, 2), (1030, 1, 1, 2), (385, 2, 1, 3), (260, 1, 2, 1), (129, 1, 1, 2)]
    probs = [synth.gaussian_problem(n, dx, dy, dz, seed=40 + i)
             for i, (n, dx, dy, dz) in enumerate(shapes)]
    ctx = idtx.Context(0)
    ctx.set_kernel(idtx.KERNEL_TILE)   # the persistent launches are the tile kernel's
    ctx.reset_stats()
    out = idtx.cmi_batch([dict(x=_dev(p.x), y=_dev(p.y), z=_dev(p.z), n_surr=9, seed=5 + i)
                          for i, p in enumerate(probs)], k=k, ctx=ctx)
    st = ctx.stats()
    n_variants = 3 if k == 4 else 1   # (1,1,2) x3, (2,1,3), (1,2,1); k=3: generic
    assert st["fused_launches"] == n_variants
    for i, (p, o) in enumerate(zip(probs, out)):
        sep = idtx.cmi_ksg(_dev(p.x), _dev(p.y), _dev(p.z), k=k, n_surr=9, seed=5 + i)
        assert np.array_equal(o.cpu().numpy(), sep.cpu().numpy())
    ref = oracle.cmi_surrogates(probs[2].x, probs[2].y, probs[2].z, k, 9, 7)
    assert np.max(np.abs(out[2].cpu().numpy() - ref)) < TOL


def test_greedy_step_matches_oracle(idtx):
    net = synth.var_network(n_nodes=5, order=3, T=700, density=0.4, weight=0.6, seed=21)
    S = 20
    ref = oracle.select_target(net.series, 0, n_past=2, min_lag=1, max_lag=3, k=4, n_surr=S,
                               alpha=0.05, seed=17, max_parents=1, want_first_step=True)
    (cand, sig, stat, pval), est = idtx.mte_step(_dev(net.series), 0, 2, 1, 3, (), 0, k=4,
                                                 n_surr=S, alpha=0.05, seed=17,
                                                 want_estimates=True)
    alive = ~np.isnan(ref["first_step"][:, 0])
    assert np.array_equal(alive, ~np.isnan(est[:, 0]))
    assert np.max(np.abs(est[alive] - ref["first_step"][alive])) < TOL
    rc, rsig, rstat, rp = ref["steps"][0]
    assert (cand, sig, pval) == (rc, rsig, rp)
    assert abs(stat - rstat) < TOL


def test_greedy_selection_matches_oracle(idtx):
    net = synth.var_network(n_nodes=4, order=2, T=600, density=0.5, weight=0.8, seed=8)
    for target in range(2):
        ref = oracle.select_target(net.series, target, n_past=1, min_lag=1, max_lag=2, k=4,
                                   n_surr=20, alpha=0.05, seed=5, max_parents=4)
        got = idtx.mte_select_target(net.series, target, 1, 1, 2, k=4, n_surr=20, alpha=0.05,
                                     seed=5, max_parents=4)
        assert got["parents"] == ref["parents"]
        assert [s[:2] for s in got["steps"]] == [s[:2] for s in ref["steps"]]
        assert [s[3] for s in got["steps"]] == [s[3] for s in ref["steps"]]
        for a, b in zip(got["steps"], ref["steps"]):
            assert abs(a[2] - b[2]) < TOL


@pytest.mark.slow
def test_config2_full_size_sampled(idtx):
    """The benchmarked greedy step at full size (10-node VAR(5), T=10000, lags 1..5,
    target history 3, k=4, 200 surrogates): gate and sampled estimates vs the oracle."""
    net = synth.var_network()
    S = 200
    (cand, sig, stat, pval), est = idtx.mte_step(_dev(net.series), 0, 3, 1, 5, (), 0, k=4,
                                                 n_surr=S, alpha=0.05, seed=20181029,
                                                 want_estimates=True)
    alive = np.flatnonzero(~np.isnan(est[:, 0]))
    assert len(alive) == 47
    L, T = 5, net.series.shape[1]
    y = net.series[0, L:]
    z = np.stack([net.series[0, L - lag:T - lag] for lag in (1, 2, 3)])
    rng = np.random.default_rng(0)
    for c in rng.choice(alive, 3, replace=False):
        p, lag = divmod(int(c), 5)
        lag += 1
        xc = net.series[p, L - lag:T - lag][None, :]
        for s in [0, int(rng.integers(1, S + 1))]:
            xs = xc if s == 0 else xc[:, oracle.perm(20181029, (int(c) << 24) | (s - 1), T - L)]
            assert abs(est[c, s] - oracle.cmi_ksg(xs, y, z, 4)) < TOL
    # the gate from the returned estimates (same decision rule)
    t_obs = est[alive, 0].max()
    assert cand == alive[np.argmax(est[alive, 0])] and stat == t_obs
    assert pval == np.count_nonzero(est[alive, 1:].max(axis=0) >= t_obs) / S


@pytest.mark.slow
def test_benchmark_size_sampled_eps_and_counts_both_kernels(idtx):
    """At the benchmarked size and the default list capacities -- N = 9995,
    joint dimension 5 (a candidate of the benchmarked greedy step: node 2 at
    lag 1 for target 0, whose lags 1..3 are Z), 200 surrogates -- eps and the
    three counts of 64 sampled queries in 4 estimates bit-exact against the
    oracle, under the list kernel and under the tile kernel; all 201
    estimates identical between the two, the original within 1e-10 of the
    oracle's."""
    net = synth.var_network()
    L, T = 5, net.series.shape[1]
    n = T - L
    y = net.series[0, L:][None, :]
    z = np.stack([net.series[0, L - lag:T - lag] for lag in (1, 2, 3)])
    x = net.series[2, L - 1:T - 1][None, :]
    S, seed = 200, 20181029
    out = {}
    for name, kern in (("list", idtx.KERNEL_LIST), ("tile", idtx.KERNEL_TILE)):
        ctx = idtx.Context(0)
        ctx.set_kernel(kern)
        cmi, eps, cnt = idtx.cmi_ksg(_dev(x), _dev(y), _dev(z), k=4, n_surr=S, seed=seed,
                                     want_eps=True, want_counts=True, ctx=ctx)
        out[name] = (cmi.cpu().numpy(), eps.cpu().numpy(), cnt.cpu().numpy())
        st = ctx.stats()
        assert st["list_launches"] == (1 if name == "list" else 0)
        if name == "list":
            assert (st["list_cap_a"], st["list_cap_b"]) == (2048, 4096)
    idx = np.random.default_rng(2).choice(n, 64, replace=False)
    for s in (0, 1, 117, 200):
        xs = x if s == 0 else x[:, oracle.perm(seed, s - 1, n)]
        e, a, b, c = oracle.ksg_counts_at(xs, y, z, 4, idx)
        for name, (_, eps, cnt) in out.items():
            assert np.array_equal(eps[s, idx], e), name
            assert np.array_equal(cnt[s, 0, idx], a), name
            assert np.array_equal(cnt[s, 1, idx], b), name
            assert np.array_equal(cnt[s, 2, idx], c), name
    assert np.array_equal(out["list"][0], out["tile"][0])
    assert abs(out["list"][0][0] - oracle.cmi_ksg(x, y, z, 4)) < TOL


@pytest.mark.slow
@pytest.mark.parametrize("kernel", ["list", "tile"])
def test_large_n_sampled_queries(idtx, kernel):
    """N = 99850 logistic-map problem, joint dim 12, 200 surrogates (the large
    single-problem configuration), with each kernel forced: sampled queries of
    the original and of two surrogates, eps and counts exact; estimates of
    those within 1e-10 through their per-sample terms."""
    x, y, z = synth.logistic_problem(1, 1, 10)
    n = x.shape[1]
    S, seed = 200, 4
    ctx = idtx.Context(0)
    ctx.set_kernel(idtx.KERNEL_LIST if kernel == "list" else idtx.KERNEL_TILE)
    cmi, eps, cnt = idtx.cmi_ksg(_dev(x), _dev(y), _dev(z), k=4, n_surr=S, seed=seed,
                                 want_eps=True, want_counts=True, ctx=ctx)
    assert ctx.stats()["list_launches"] == (1 if kernel == "list" else 0)
    cmi, eps, cnt = cmi.cpu().numpy(), eps.cpu().numpy(), cnt.cpu().numpy()
    idx = np.random.default_rng(1).choice(n, 48, replace=False)
    for s in (0, 1, 137):
        xs = x if s == 0 else x[:, oracle.perm(seed, s - 1, n)]
        e, a, b, c = oracle.ksg_counts_at(xs, y, z, 4, idx)
        assert np.array_equal(eps[s, idx], e)
        assert np.array_equal(cnt[s, 0, idx], a)
        assert np.array_equal(cnt[s, 1, idx], b)
        assert np.array_equal(cnt[s, 2, idx], c)
    # every estimate equals the digamma sum of its own returned counts
    psi = oracle.psi_table(n + 1)
    for s in (0, 5, 200):
        c = cnt[s]
        ref = psi[4] + np.mean(psi[c[2] + 1] - psi[c[0] + 1] - psi[c[1] + 1])
        assert abs(cmi[s] - ref) < 1e-10


@pytest.mark.slow
def test_batch_full_size_sampled(idtx):
    """The uneven batch at full size: 64 problems, N log-uniform in [2000, 50000],
    dx, dy in {1,2}, dz in 1..8, 500 surrogates each, in one call; sampled
    estimates of the five smallest problems against the oracle."""
    probs = synth.batch_problems()
    out = idtx.cmi_batch([dict(x=_dev(p.x), y=_dev(p.y), z=_dev(p.z), n_surr=p.n_surr,
                               seed=p.seed) for p in probs], k=4)
    out = [o.cpu().numpy() for o in out]
    assert all(np.all(np.isfinite(o)) and o.shape == (501,) for o in out)
    smallest = np.argsort([p.x.shape[1] for p in probs])[:5]
    rng = np.random.default_rng(3)
    for i in smallest:
        p = probs[i]
        for s in [0] + list(rng.choice(np.arange(1, 501), 2, replace=False)):
            xs = p.x if s == 0 else p.x[:, oracle.perm(p.seed, int(s) - 1, p.x.shape[1])]
            assert abs(out[i][s] - oracle.cmi_ksg(xs, p.y, p.z, 4)) < TOL


@pytest.mark.slow
@pytest.mark.parametrize("n", [16384, 16385, 32768, 32769, 65536, 65537, 102400, 102401])
def test_shuffle_length_classes_sampled(idtx, n):
    """Surrogate permutations of each row-length class: up to 32768 samples
    (shared-memory row, equal-draw flags in the entries' top bits),
    32769..65536 (shared-memory row, flag bitmap), 65537..102400 (entries'
    bit 16 in a shared bitmap), beyond (in place in global memory); the rows
    composed with the sample order (batched mode) and not (plain mode).
    Eps and counts of sampled queries of three surrogates exact against the
    oracle's permutations; the two modes' estimates within 1e-10."""
    g = synth.gaussian_problem(n, dx=1, dy=1, dz=1, seed=31 + n)
    S, seed = 3, 11
    idx = np.random.default_rng(n).choice(n, 24, replace=False)
    refs = {}
    for s in (1, 2, 3):
        xs = g.x[:, oracle.perm(seed, s - 1, n)]
        refs[s] = oracle.ksg_counts_at(xs, g.y, g.z, 4, idx)
    est = {}
    for mode in (idtx.MODE_BATCHED, idtx.MODE_PLAIN):
        cmi, eps, cnt = idtx.cmi_ksg(_dev(g.x), _dev(g.y), _dev(g.z), k=4, n_surr=S, seed=seed,
                                     want_eps=True, want_counts=True, mode=mode)
        est[mode] = cmi.cpu().numpy()
        eps, cnt = eps.cpu().numpy(), cnt.cpu().numpy()
        for s, (e, a, b, c) in refs.items():
            assert np.array_equal(eps[s, idx], e), (mode, s)
            assert np.array_equal(cnt[s, 0, idx], a), (mode, s)
            assert np.array_equal(cnt[s, 1, idx], b), (mode, s)
            assert np.array_equal(cnt[s, 2, idx], c), (mode, s)
    assert np.allclose(est[idtx.MODE_PLAIN], est[idtx.MODE_BATCHED], rtol=0, atol=TOL)

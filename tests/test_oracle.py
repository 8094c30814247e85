"""Pins for the CPU oracle: each test ties it to something other than itself.

The IDTxl paper (arXiv 1807.10459) prints no formula or worked example, so the
pins are a hand-worked example, closed forms (the linear-Gaussian estimator the
paper lists beside KSG, Summary paragraph on estimators), invariants of the
max-norm neighbour statistics, special cases that reduce to textbook formulas
and library routines, and the published output sequence of SplitMix64.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special
import scipy.stats

import oracle
from paper_1807_10459_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gaussian_closed_form(cov, dx, dy, dz):
    """I(X;Y|Z) = 1/2 ln[det S_xz det S_yz / (det S_z det S_xyz)] for a Gaussian law."""
    X = list(range(dx))
    Y = list(range(dx, dx + dy))
    Z = list(range(dx + dy, dx + dy + dz))

    def ld(idx):
        return np.linalg.slogdet(cov[np.ix_(idx, idx)])[1] if idx else 0.0

    return 0.5 * (ld(X + Z) + ld(Y + Z) - ld(Z) - ld(X + Y + Z))


def numpy_bruteforce(x, y, z, k):
    """Independent float32 brute force with numpy broadcasting and np.partition."""
    x = np.asarray(x, np.float32)
    y = np.asarray(y, np.float32)
    n = x.shape[1]

    def cheb(a):
        if a is None or a.shape[0] == 0:
            return np.zeros((n, n), np.float32)
        return np.max(np.abs(a[:, :, None] - a[:, None, :]), axis=0)

    dX, dY, dZ = cheb(x), cheb(y), cheb(None if z is None else np.asarray(z, np.float32))
    joint = np.maximum(np.maximum(dX, dY), dZ)
    np.fill_diagonal(joint, np.inf)
    eps = np.partition(joint, k - 1, axis=1)[:, k - 1]
    off = ~np.eye(n, dtype=bool)
    e = eps[:, None]
    nxz = ((np.maximum(dX, dZ) < e) & off).sum(1)
    nyz = ((np.maximum(dY, dZ) < e) & off).sum(1)
    nz = ((dZ < e) & off).sum(1)
    return eps.astype(np.float32), nxz, nyz, nz


# ---------------------------------------------------------------- hand example
def test_hand_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "hand_n6_k1.json")))
    x = np.array([g["x"]], np.float32)
    y = np.array([g["y"]], np.float32)
    z = np.array([g["z"]], np.float32)
    eps, nxz, nyz, nz = oracle.ksg_counts(x, y, z, g["k"])
    assert eps.tolist() == [float(v) for v in g["eps"]]
    assert nxz.tolist() == g["nxz"]
    assert nyz.tolist() == g["nyz"]
    assert nz.tolist() == g["nz"]
    cmi = oracle.cmi_ksg(x, y, z, g["k"])
    assert abs(cmi - g["cmi_numerator"] / g["cmi_denominator"]) < 1e-14


# ---------------------------------------------------------------- digamma
def test_psi_matches_library_digamma():
    n_max = 100000
    t = oracle.psi_table(n_max)
    assert math.isnan(t[0])
    assert abs(t[1] + np.euler_gamma) < 1e-16
    n = np.arange(1, n_max + 1, dtype=np.float64)
    assert np.max(np.abs(t[1:] - scipy.special.digamma(n))) < 1e-13


def test_psi_recurrence():
    t = oracle.psi_table(5000)
    n = np.arange(1, 5000)
    assert np.max(np.abs((t[2:] - t[1:-1]) - 1.0 / n)) < 1e-13


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("dims,k,n", [((1, 1, 2), 4, 300), ((2, 1, 0), 3, 257), ((1, 2, 3), 1, 200),
                                      ((2, 2, 5), 6, 180)])
def test_matches_independent_numpy_bruteforce(dims, k, n):
    dx, dy, dz = dims
    g = synth.gaussian_problem(n, dx, dy, dz, seed=77 + n)
    z = g.z if dz else None
    eps, nxz, nyz, nz = oracle.ksg_counts(g.x, g.y, z, k)
    e2, a2, b2, c2 = numpy_bruteforce(g.x, g.y, z, k)
    assert np.array_equal(eps, e2)
    assert np.array_equal(nxz, a2)
    assert np.array_equal(nyz, b2)
    assert np.array_equal(nz, c2)


def test_bruteforce_with_ties_and_duplicates():
    rng = np.random.default_rng(5)
    # values on a coarse grid: many equal distances and duplicate samples
    x = rng.integers(0, 4, (1, 150)).astype(np.float32)
    y = rng.integers(0, 4, (1, 150)).astype(np.float32)
    z = rng.integers(0, 3, (2, 150)).astype(np.float32)
    for k in (1, 2, 4, 8):
        got = oracle.ksg_counts(x, y, z, k)
        ref = numpy_bruteforce(x, y, z, k)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


# ---------------------------------------------------------------- special case dz = 0
def test_dz0_reduces_to_ksg_mutual_information():
    g = synth.gaussian_problem(2000, 1, 1, 0, seed=11)
    k = 4
    eps, nx, ny, nz = oracle.ksg_counts(g.x, g.y, None, k)
    n = g.x.shape[1]
    assert np.all(eps > 0)
    assert np.all(nz == n - 1)
    mi = scipy.special.digamma(k) + scipy.special.digamma(n) - np.mean(
        scipy.special.digamma(nx + 1.0) + scipy.special.digamma(ny + 1.0))
    assert abs(oracle.cmi_ksg(g.x, g.y, None, k) - mi) < 1e-12
    # bivariate Gaussian MI closed form -1/2 ln(1 - rho^2)
    c = g.cov
    rho = c[0, 1] / math.sqrt(c[0, 0] * c[1, 1])
    assert abs(mi - (-0.5 * math.log(1 - rho * rho))) < 0.06


# ---------------------------------------------------------------- closed forms
def test_gaussian_closed_form_n1e4_mean_of_10():
    cov = synth.gaussian_problem(1000, 1, 1, 2).cov
    truth = gaussian_closed_form(cov, 1, 1, 2)
    vals = [oracle.cmi_ksg(*(lambda g: (g.x, g.y, g.z))(
        synth.gaussian_problem(10000, 1, 1, 2, seed=1000 + s, cov=cov)), 4) for s in range(10)]
    assert abs(np.mean(vals) - truth) < 0.02


def test_gaussian_closed_form_n1e3_single():
    g = synth.gaussian_problem(1000, 1, 1, 2)
    truth = gaussian_closed_form(g.cov, 1, 1, 2)
    assert abs(oracle.cmi_ksg(g.x, g.y, g.z, 4) - truth) < 0.06


def test_independent_shuffle_is_near_zero():
    cov = synth.gaussian_problem(1000, 1, 1, 2).cov
    vals = []
    for s in range(10):
        g = synth.gaussian_problem(10000, 1, 1, 2, seed=3000 + s, cov=cov)
        xs = g.x[:, np.random.default_rng(s).permutation(10000)]
        vals.append(oracle.cmi_ksg(xs, g.y, g.z, 4))
    assert abs(np.mean(vals)) < 0.01


# ---------------------------------------------------------------- invariants
def test_xy_swap_is_bit_identical():
    g = synth.gaussian_problem(700, 1, 1, 2, seed=3)
    a = oracle.ksg_counts(g.x, g.y, g.z, 4)
    b = oracle.ksg_counts(g.y, g.x, g.z, 4)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[2]) and np.array_equal(a[2], b[1])
    assert np.array_equal(a[3], b[3])
    assert oracle.cmi_ksg(g.x, g.y, g.z, 4) == oracle.cmi_ksg(g.y, g.x, g.z, 4)


def test_sample_reordering_permutes_counts():
    g = synth.gaussian_problem(600, 2, 1, 2, seed=4)
    perm = np.random.default_rng(9).permutation(600)
    a = oracle.ksg_counts(g.x, g.y, g.z, 4)
    b = oracle.ksg_counts(g.x[:, perm], g.y[:, perm], g.z[:, perm], 4)
    for u, v in zip(a, b):
        assert np.array_equal(u[perm], v)


@pytest.mark.parametrize("m", [-3, 5])
def test_power_of_two_scaling_is_bit_identical(m):
    g = synth.gaussian_problem(500, 1, 1, 3, seed=6)
    s = np.float32(2.0 ** m)
    a = oracle.ksg_counts(g.x, g.y, g.z, 4)
    b = oracle.ksg_counts(g.x * s, g.y * s, g.z * s, 4)
    assert np.array_equal(a[0] * s, b[0])
    for u, v in zip(a[1:], b[1:]):
        assert np.array_equal(u, v)


def test_count_nesting_and_lower_bounds():
    g = synth.gaussian_problem(800, 1, 1, 2, seed=8)
    eps, nxz, nyz, nz = oracle.ksg_counts(g.x, g.y, g.z, 4)
    assert np.all(nz >= nxz) and np.all(nz >= nyz)
    # continuous data: no ties at eps, so at least k-1 neighbours lie strictly inside
    assert np.all(nxz >= 3) and np.all(nyz >= 3)


# ---------------------------------------------------------------- permutations
def test_splitmix64_published_sequence():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64_1234567.json")))
    out = oracle.splitmix64(g["state"], len(g["outputs"]))
    assert [int(v) for v in out] == [int(s) for s in g["outputs"]]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 16, 17, 255, 1000, 9995, 65537])
def test_permutation_is_a_bijection(n):
    for stream in (0, 1, 12345, (3 << 48) | (7 << 24) | 9):
        p = oracle.perm(20181027, stream, n)
        assert np.array_equal(np.sort(p), np.arange(n))


def test_permutation_positions_are_uniform():
    n, reps = 10, 20000
    hist = np.zeros((n, n))
    for s in range(reps):
        p = oracle.perm(99, s, n)
        hist[np.arange(n), p] += 1
    expected = reps / n
    chi2 = ((hist - expected) ** 2 / expected).sum(axis=1)
    # each row: chi-square with n-1 = 9 dof; 0.999 quantile is 27.9
    assert np.all(chi2 < 27.9 * 1.3)
    assert scipy.stats.chi2.sf(chi2.sum(), n * (n - 1)) > 1e-3


def test_permutations_differ_by_stream_and_seed():
    a = oracle.perm(1, 0, 1000)
    b = oracle.perm(1, 1, 1000)
    c = oracle.perm(2, 0, 1000)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


# ---------------------------------------------------------------- surrogates
def test_surrogates_permute_rows_of_x():
    g = synth.gaussian_problem(400, 2, 1, 1, seed=12)
    out = oracle.cmi_surrogates(g.x, g.y, g.z, 4, 5, 777)
    assert out[0] == oracle.cmi_ksg(g.x, g.y, g.z, 4)
    for s in range(5):
        p = oracle.perm(777, s, 400)
        assert out[1 + s] == oracle.cmi_ksg(g.x[:, p], g.y, g.z, 4)


def test_surrogate_distribution_is_centred_below_signal():
    g = synth.gaussian_problem(1000, 1, 1, 2)
    out = oracle.cmi_surrogates(g.x, g.y, g.z, 4, 40, 5)
    assert out[0] > np.max(out[1:])
    assert abs(np.mean(out[1:])) < 0.03


# ---------------------------------------------------------------- greedy selection
def test_greedy_recovers_strong_parents():
    net = synth.var_network(n_nodes=5, order=3, T=1500, density=0.35, weight=0.9, seed=31)
    target = 0
    edges = {(p, lag) for (p, q, lag) in net.edges if q == target}
    truth = {(p, lag) for (p, lag) in edges if abs(net.coef[lag - 1, target, p]) > 0.2}
    assert truth, "generator seed must give the target at least one strong parent"
    res = oracle.select_target(net.series, target, n_past=1, min_lag=1, max_lag=3, k=4,
                               n_surr=20, alpha=0.05, seed=123, max_parents=6)
    got = {(c // 3, 1 + c % 3) for c in res["parents"]}
    assert truth <= got
    assert len(got - edges) <= 1
    last = res["steps"][-1]
    assert not last[1] or len(res["parents"]) == 6


def test_greedy_first_step_gate_from_estimates():
    net = synth.var_network(n_nodes=4, order=2, T=600, density=0.5, weight=0.7, seed=8)
    S = 20
    res = oracle.select_target(net.series, 1, n_past=1, min_lag=1, max_lag=2, k=3, n_surr=S,
                               alpha=0.05, seed=9, max_parents=1, want_first_step=True)
    est = res["first_step"]
    alive = ~np.isnan(est[:, 0])
    assert alive.sum() == 4 * 2 - 1       # the target's own lag 1 is in Z
    c_best = int(np.flatnonzero(alive)[np.argmax(est[alive, 0])])
    t_obs = est[c_best, 0]
    t_s = np.max(est[alive, 1:], axis=0)
    cand, sig, stat, pval = res["steps"][0]
    assert cand == c_best and stat == t_obs
    assert pval == np.count_nonzero(t_s >= t_obs) / S
    assert sig == (pval < 0.05)


# ---------------------------------------------------------------- learned screen network
def _rand_net(f, h, seed):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(oracle.mlp_nparams(f, h)) * 0.4).astype(np.float32)
    x = rng.standard_normal((37, f)).astype(np.float32)
    t = rng.standard_normal(37).astype(np.float32)
    mean = rng.standard_normal(f).astype(np.float32) * 0.1
    scale = (1.0 + rng.random(f)).astype(np.float32)
    return p, x, t, mean, scale


def test_bf16_rounding_matches_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.standard_normal(5000).astype(np.float32) * 10.0 ** rng.integers(-5, 5, 5000),
                        # exact ties: a bf16 value plus half an ulp of bf16
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -3.0 - 2.0 ** -7], np.float32)])
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.bf16_round(float(a)) for a in v], np.float32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("quantile", [0.0, 0.9])
def test_mlp_gradient_matches_finite_differences(quantile):
    f, h = 3, 5
    p, x, t, mean, scale = _rand_net(f, h, 1)
    loss, g = oracle.mlp_loss_grad(p, f, h, mean, scale, x, t, bf16=False, quantile=quantile)

    def fd(idx, eps):
        hi, lo = p.copy(), p.copy()
        hi[idx] += np.float32(eps)
        lo[idx] -= np.float32(eps)
        step = float(hi[idx]) - float(lo[idx])
        lh, _ = oracle.mlp_loss_grad(hi, f, h, mean, scale, x, t, bf16=False, quantile=quantile)
        ll, _ = oracle.mlp_loss_grad(lo, f, h, mean, scale, x, t, bf16=False, quantile=quantile)
        return (lh - ll) / step

    checked = 0
    for idx in range(len(p)):
        a, b = fd(idx, 1e-3), fd(idx, 5e-4)
        if abs(a - b) > 1e-6:      # a ReLU kink inside the interval: not differentiable there
            continue
        assert abs(a - g[idx]) <= 1e-5 * max(1.0, abs(g[idx])), (idx, a, g[idx])
        checked += 1
    assert checked >= 0.8 * len(p)


def test_mlp_bf16_forward_equals_exact_forward_on_rounded_weights():
    f, h = 10, 64
    p, x, t, mean, scale = _rand_net(f, h, 4)
    pr = p.copy()
    nw = [(0, h * f), (h * f + h, h * f + h + h * h), (h * f + 2 * h + h * h, h * f + 3 * h + h * h)]
    for a, b in nw:
        pr[a:b] = [oracle.bf16_round(float(v)) for v in p[a:b]]
    y1 = oracle.mlp_forward(p, f, h, mean, scale, x, bf16=True)
    y2 = oracle.mlp_forward(pr, f, h, mean, scale, x, bf16=False)
    assert np.array_equal(y1, y2)
    l1, g1 = oracle.mlp_loss_grad(p, f, h, mean, scale, x, t, bf16=True)
    l2, g2 = oracle.mlp_loss_grad(pr, f, h, mean, scale, x, t, bf16=False)
    assert l1 == l2 and np.array_equal(g1, g2)


def test_mlp_forward_closed_form_linear_case():
    # with all hidden pre-activations positive the network is affine: check by hand
    f, h = 2, 2
    W1 = np.array([[1.0, 0.5], [0.25, 2.0]], np.float32)
    b1 = np.array([3.0, 3.0], np.float32)
    W2 = np.array([[1.0, 0.0], [0.5, 0.5]], np.float32)
    b2 = np.array([0.0, 1.0], np.float32)
    w3 = np.array([2.0, -1.0], np.float32)
    b3 = np.array([0.5], np.float32)
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, b3])
    x = np.array([[1.0, 0.0], [0.0, 1.0]], np.float32)
    y = oracle.mlp_forward(p, f, h, np.zeros(2, np.float32), np.ones(2, np.float32), x)
    for s in range(2):
        a1 = W1 @ x[s] + b1
        a2 = W2 @ a1 + b2
        assert abs(y[s] - (w3 @ a2 + b3[0])) < 1e-12


def test_pinball_loss_of_a_constant_is_minimised_at_the_quantile():
    # zero weights: the network is the constant b3; the pinball loss over a
    # sample is smallest when that constant is the sample's quantile
    f, h = 2, 3
    rng = np.random.default_rng(6)
    t = rng.standard_normal(2001).astype(np.float32)
    x = np.zeros((2001, f), np.float32)
    p = np.zeros(oracle.mlp_nparams(f, h), np.float32)
    q = 0.9
    best = np.quantile(t, q, method="inverted_cdf")
    losses = []
    for c in (best - 0.05, best, best + 0.05):
        p[-1] = c
        losses.append(oracle.mlp_loss_grad(p, f, h, np.zeros(f, np.float32),
                                           np.ones(f, np.float32), x, t, quantile=q)[0])
    assert losses[1] < losses[0] and losses[1] < losses[2]
    p[-1] = best
    _, g = oracle.mlp_loss_grad(p, f, h, np.zeros(f, np.float32), np.ones(f, np.float32), x, t,
                                quantile=q)
    assert abs(g[-1] - (np.count_nonzero(t < best) / 2001 - q)) < 1e-12


# ---------------------------------------------------------------- tests after selection
def _driven_system(T=1500, seed=3):
    """Node 0 is driven at lag 1 by nodes 1 and 2 (AR(1) each); nodes 3, 4, 5
    are independent noise.  Candidates use lag 1 only: candidate id = node."""
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


def test_pruning_keeps_drivers_and_empties_a_noise_list():
    """The minimum statistic compares the weakest parent with the minima of
    all parents' surrogates; true drivers pass in the first round, a list of
    independent sources is pruned away one round at a time."""
    s = _driven_system()
    r = oracle.prune(s, parents=[2, 1], **POST)
    assert r["kept"] == [2, 1] and len(r["rounds"]) == 1 and r["rounds"][0][1]
    r = oracle.prune(s, parents=[3, 4, 5], **POST)
    assert r["kept"] == [] and len(r["rounds"]) == 3
    assert all(not sig for (_, sig, _, _) in r["rounds"])
    # each round removes the parent at the minimum of the remaining ones
    removed = [c for (c, _, _, _) in r["rounds"]]
    assert sorted(removed) == [3, 4, 5]


def test_omnibus_separates_drivers_from_noise():
    s = _driven_system()
    stat, p, sig = oracle.omnibus(s, parents=[1, 2], **POST)
    assert sig and p == 0.0 and stat > 0.2
    stat_n, p_n, sig_n = oracle.omnibus(s, parents=[3, 4], **POST)
    assert not sig_n and abs(stat_n) < 0.05


def test_sequential_max_statistic_orders_and_stops():
    s = _driven_system()
    stats, pvals, sig = oracle.seqmax(s, parents=[1, 3, 2], **POST)
    assert list(sig) == [True, False, True]
    assert stats[1] < min(stats[0], stats[2])
    assert pvals[0] == 0.0 and pvals[2] == 0.0 and pvals[1] >= POST["alpha"]
    # leave-one-out statistics are those of the first pruning round (same conditioning)
    r = oracle.prune(s, parents=[1, 3, 2], **POST)
    assert r["rounds"][0][0] == 3 and r["rounds"][0][2] == stats[1]


def test_single_parent_statistics_equal_the_greedy_estimate():
    """With one parent, the leave-one-out statistic, the omnibus statistic and
    the greedy step's estimate of that candidate are the same CMI."""
    s = _driven_system(T=700, seed=5)
    sel = oracle.select_target(s, 0, 1, 1, 1, 4, 5, 0.05, 11, 1, want_first_step=True)
    for c in (1, 2, 3):
        greedy = sel["first_step"][c, 0]
        stat, _, _ = oracle.omnibus(s, parents=[c], **POST)
        stats, _, _ = oracle.seqmax(s, parents=[c], **POST)
        r = oracle.prune(s, parents=[c], **POST)
        assert stat == greedy and stats[0] == greedy and r["rounds"][0][2] == greedy


def test_post_selection_rejects_bad_arguments():
    s = _driven_system(T=300)
    for bad in (dict(parents=[]), dict(parents=[9]), dict(parents=[1], n_surr=0)):
        args = dict(POST, **bad)
        with pytest.raises(ValueError):
            oracle.prune(s, **args)


def test_bivariate_te_finds_drivers_and_matches_the_greedy_estimates():
    s = _driven_system()
    est, p = oracle.bivariate_te(s, 0, 1, 1, 1, 4, 40, 11)
    assert np.isnan(p[0])                         # the target's own variable is not a source
    assert p[1] == 0.0 and p[2] == 0.0            # the two drivers
    assert all(p[c] >= 0.05 for c in (3, 4, 5))  # independent sources
    sel = oracle.select_target(s, 0, 1, 1, 1, 4, 3, 0.05, 11, 1, want_first_step=True)
    for c in range(1, 6):
        assert est[c, 0] == sel["first_step"][c, 0]


# ---------------------------------------------------------------- non-uniform target past
def test_source_selection_from_a_uniform_past_equals_select_target():
    """Two implementations of the greedy loop: starting the source selection
    from the past (target, lags 1..n_past) reproduces select_target(n_past)."""
    net = synth.var_network(n_nodes=4, order=3, T=900, density=0.5, weight=0.6, seed=17)
    for target, n_past in ((0, 2), (2, 1), (3, 3)):
        ref = oracle.select_target(net.series, target, n_past, 1, 3, 4, 15, 0.05, 8, 4)
        past = [target * 3 + lag - 1 for lag in range(1, n_past + 1)]
        got = oracle.select_sources(net.series, target, past, 1, 3, 4, 15, 0.05, 8, 4)
        assert got["parents"] == ref["parents"]
        assert got["steps"] == ref["steps"]


def test_past_of_an_ar2_target_is_its_first_two_lags():
    rng = np.random.default_rng(2)
    T = 1500
    x = np.zeros((2, T + 100))
    e = rng.standard_normal((2, T + 100))
    for t in range(2, T + 100):
        x[0, t] = 0.6 * x[0, t - 1] - 0.4 * x[0, t - 2] + e[0, t]
        x[1, t] = e[1, t]
    s = x[:, 100:].astype(np.float32)
    r = oracle.select_past(s, 0, 1, 4, 4, 30, 0.05, 5, 4)
    assert sorted(r["past"]) == [0, 1]            # ids of (target, lag 1) and (target, lag 2)
    assert r["steps"][-1][1] is False             # stopped by a non-significant step
    assert all(c < 4 for (c, _, _, _) in r["steps"])   # only the target's own variables


# ---------------------------------------------------------------- replication-level surrogates
def test_replication_surrogates_with_single_sample_replications_are_sample_surrogates():
    g = synth.gaussian_problem(240, 1, 1, 2, seed=6)
    a = oracle.cmi_surrogates_reps(g.x, g.y, g.z, 4, 6, 13, n_reps=240)
    b = oracle.cmi_surrogates(g.x, g.y, g.z, 4, 6, 13)
    assert np.array_equal(a, b)


def test_replication_surrogates_move_whole_replications():
    """A surrogate equals the estimate with X's replications reordered by the
    permutation of the replication indices."""
    g = synth.gaussian_problem(300, 2, 1, 1, seed=7)
    reps, length = 12, 25
    out = oracle.cmi_surrogates_reps(g.x, g.y, g.z, 4, 3, 21, n_reps=reps)
    for s in range(3):
        pr = oracle.perm(21, s, reps)
        idx = (pr[:, None] * length + np.arange(length)[None, :]).ravel()
        assert out[1 + s] == oracle.cmi_ksg(g.x[:, idx], g.y, g.z, 4)
    with pytest.raises(ValueError):
        oracle.cmi_surrogates_reps(g.x, g.y, g.z, 4, 3, 21, n_reps=7)   # 300 % 7 != 0


# ---------------------------------------------------------------- multivariate MI inference
def test_mi_inference_steps_are_ksg_mi_then_cmi_of_the_embedded_columns():
    """With no target past the first greedy step estimates, per candidate, the
    plain KSG MI (algorithm 1) of the lagged source column with the target's
    present; the second step's statistic conditions on the first parent's
    column only.  Both are recomputed here from an embedding built by hand
    (samples t = max_lag .. T-1) with the independent numpy brute force."""
    net = synth.var_network(n_nodes=3, order=2, T=400, density=0.6, weight=0.7, seed=23)
    s = net.series
    target, lo, hi, k = 1, 1, 2, 4
    sel = oracle.select_target(s, target, 0, lo, hi, k, 20, 0.05, 5, 2, want_first_step=True)
    T = s.shape[1]
    n = T - hi
    y = s[target, hi:][None, :]

    def col(c):
        p, lag = divmod(c, hi - lo + 1)
        lag += lo
        return s[p, hi - lag:T - lag][None, :]

    psi = scipy.special.digamma
    for c in range(3 * (hi - lo + 1)):
        _, nx, ny, _ = numpy_bruteforce(col(c), y, None, k)
        mi = psi(k) + psi(n) - np.mean(psi(nx + 1.0) + psi(ny + 1.0))
        assert abs(sel["first_step"][c, 0] - mi) < 1e-12
    assert len(sel["steps"]) >= 2 and sel["steps"][0][1]
    first, second = sel["steps"][0][0], sel["steps"][1][0]
    assert sel["steps"][0][2] == np.max(sel["first_step"][:, 0])
    _, nxz, nyz, nz = numpy_bruteforce(col(second), y, col(first), k)
    cmi = psi(k) + np.mean(psi(nz + 1.0) - psi(nxz + 1.0) - psi(nyz + 1.0))
    assert abs(sel["steps"][1][2] - cmi) < 1e-12


# ------------------------------------------ tests after selection, recomputed
def _loo_table(s, parents, tag, n_past, seed, k, n_surr):
    """Leave-one-out statistics and their surrogates, assembled here from the
    pinned estimator and permutations (lag-1 candidates: candidate id =
    node): row i = [T_i, T_i,0 .. T_i,S-1]."""
    T = s.shape[1]
    L = max(1, n_past)
    y = s[0, L:]
    past = [s[0, L - lag:T - lag] for lag in range(1, n_past + 1)]
    col = lambda c: s[c, L - 1:T - 1][None, :]
    out = np.zeros((len(parents), 1 + n_surr))
    for i, c in enumerate(parents):
        z = np.stack(past + [col(d)[0] for j, d in enumerate(parents) if j != i])
        out[i, 0] = oracle.cmi_ksg(col(c), y, z, k)
        for t in range(n_surr):
            pi = oracle.perm(seed, (tag << 48) | (c << 24) | t, T - L)
            out[i, 1 + t] = oracle.cmi_ksg(col(c)[:, pi], y, z, k)
    return out


def test_pruning_omnibus_and_seqmax_recomputed_from_the_estimator():
    """The three tests' decisions and statistics follow from the estimates by
    the stated rules: pruning by the minimum statistic (round r tagged
    0x9000 + r), the omnibus test of the parents jointly, the step-down
    maximum statistic (tag 0xB000)."""
    s = _driven_system(T=400, seed=9)
    kw = dict(POST, n_surr=12, seed=4)
    S, alpha, seed, k = kw["n_surr"], kw["alpha"], kw["seed"], kw["k"]
    parents = [1, 3, 4, 2]

    # pruning, round by round
    ref = oracle.prune(s, parents=parents, **kw)
    cur, rounds = list(parents), []
    while cur:
        e = _loo_table(s, cur, 0x9000 + len(rounds), 1, seed, k, S)
        at = int(np.argmin(e[:, 0]))                   # first index among ties
        p = np.count_nonzero(e[:, 1:].min(axis=0) >= e[at, 0]) / S
        rounds.append((cur[at], p < alpha, e[at, 0], p))
        if p < alpha:
            break
        cur.pop(at)
    assert ref["kept"] == cur
    assert ref["rounds"] == rounds

    # omnibus: the parents' columns permuted together
    T = s.shape[1]
    x = np.stack([s[c, 0:T - 1] for c in parents])
    y, z = s[0, 1:], s[0, 0:T - 1][None, :]
    t_obs = oracle.cmi_ksg(x, y, z, k)
    surr = [oracle.cmi_ksg(x[:, oracle.perm(seed, (0xA000 << 48) | (0xFFFFFF << 24) | t, T - 1)],
                           y, z, k) for t in range(S)]
    p = np.count_nonzero(np.array(surr) >= t_obs) / S
    assert oracle.omnibus(s, parents=parents, **kw) == (t_obs, p, p < alpha)

    # sequential maximum statistic
    e = _loo_table(s, parents, 0xB000, 1, seed, k, S)
    order = sorted(range(len(parents)), key=lambda i: (-e[i, 0], i))
    pv, sig, still = np.zeros(len(parents)), np.zeros(len(parents), bool), True
    for r, i in enumerate(order):
        mx = e[order[r:], 1:].max(axis=0)
        pv[i] = np.count_nonzero(mx >= e[i, 0]) / S
        still = still and pv[i] < alpha
        sig[i] = still
    stats, pvals, sigs = oracle.seqmax(s, parents=parents, **kw)
    assert np.array_equal(stats, e[:, 0])
    assert np.array_equal(pvals, pv) and np.array_equal(np.asarray(sigs, bool), sig)


def test_bivariate_te_surrogates_and_pvalues_recomputed():
    """Each source's surrogates are its column permuted with stream
    0xC000 << 48 | c << 24 | s, and p(c) counts the surrogates at or above
    the estimate."""
    s = _driven_system(T=300, seed=13)
    S, seed, k = 9, 6, 4
    est, p = oracle.bivariate_te(s, 0, 1, 1, 1, k, S, seed)
    T = s.shape[1]
    y, z = s[0, 1:], s[0, 0:T - 1][None, :]
    for c in (1, 4):
        x = s[c, 0:T - 1][None, :]
        assert est[c, 0] == oracle.cmi_ksg(x, y, z, k)
        for t in (0, S - 1):
            pi = oracle.perm(seed, (0xC000 << 48) | (c << 24) | t, T - 1)
            assert est[c, 1 + t] == oracle.cmi_ksg(x[:, pi], y, z, k)
    for c in range(1, 6):
        assert p[c] == np.count_nonzero(est[c, 1:] >= est[c, 0]) / S


def test_target_past_selection_recomputed():
    """The greedy loop over the target's own lags, rebuilt here step by step
    from the pinned estimator and shuffle: step s tags its streams 0xD000 + s,
    the first maximum wins, p counts surrogate maxima at or above it."""
    rng = np.random.default_rng(8)
    T, lo, hi, k, S, seed, alpha = 350, 1, 3, 4, 10, 3, 0.05
    x = np.zeros((2, T + 100))
    e = rng.standard_normal((2, T + 100))
    for t in range(2, T + 100):
        x[0, t] = 0.5 * x[0, t - 1] - 0.4 * x[0, t - 2] + e[0, t]
        x[1, t] = e[1, t]
    s = x[:, 100:].astype(np.float32)
    ref = oracle.select_past(s, 0, lo, hi, k, S, alpha, seed, hi - lo + 1)
    n = T - hi
    y = s[0, hi:][None, :]
    col = lambda c: s[0, hi - (lo + c):T - (lo + c)][None, :]   # c = lag - lo (target 0)
    open_c, zcols, steps = list(range(hi - lo + 1)), [], []
    while open_c:
        z = np.stack(zcols) if zcols else None
        tab = {}
        for c in open_c:
            row = [oracle.cmi_ksg(col(c), y, z, k)]
            for i in range(S):
                pi = oracle.perm(seed, ((0xD000 + len(steps)) << 48) | (c << 24) | i, n)
                row.append(oracle.cmi_ksg(col(c)[:, pi], y, z, k))
            tab[c] = row
        best = max(open_c, key=lambda c: (tab[c][0], -c))
        t_obs = tab[best][0]
        p = sum(max(tab[c][1 + i] for c in open_c) >= t_obs for i in range(S)) / S
        steps.append((best, p < alpha, t_obs, p))
        if p >= alpha:
            break
        open_c.remove(best)
        zcols.append(col(best)[0])
    assert ref["steps"] == steps
    assert ref["past"] == [c for (c, sig, _, _) in steps if sig]
    assert len(steps) >= 2


@pytest.mark.parametrize("n", [2, 3, 4, 7, 33])
def test_smallest_problems_every_k(n):
    """Edge sizes: N from 2 (a single neighbour) upward, every k up to N-1
    (eps = the largest joint distance), against the numpy brute force, and
    the estimate against the digamma sum of those counts."""
    g = synth.gaussian_problem(n, 1, 2, 2, seed=40 + n)
    for k in range(1, n):
        got = oracle.ksg_counts(g.x, g.y, g.z, k)
        ref = numpy_bruteforce(g.x, g.y, g.z, k)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        psi = scipy.special.digamma
        eps, nxz, nyz, nz = got
        want = psi(k) + np.mean(psi(nz + 1.0) - psi(nxz + 1.0) - psi(nyz + 1.0))
        assert abs(oracle.cmi_ksg(g.x, g.y, g.z, k) - want) < 1e-12

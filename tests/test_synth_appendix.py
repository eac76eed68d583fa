"""The appendix generator (App. A) against what its construction fixes:
Poisson resource counts (law checked against the Poisson pmf and moments),
distinct requests per resource, the item-major and user-major forms holding
the same edge set, a_ij / c_ij constant per resource, the value cap, and the
greedy load recomputed by a brute-force loop.  CPU only."""
import math

import numpy as np
import pytest

import synth


def small(seed=11, I=3000, J=120, **kw):
    return synth.AppRecipe(I=I, J=J, seed=seed, **kw)


def test_same_instance_for_any_thread_count():
    r = small(I=40_000, J=300)
    one = synth.generate_appendix(r, nthreads=1)
    many = synth.generate_appendix(r, nthreads=4)
    for f in ("row_ptr", "col", "c", "a", "b"):
        assert np.array_equal(getattr(one, f), getattr(many, f)), f


@pytest.mark.parametrize("mu", [0.4, 3.0, 17.0])
def test_poisson_sampler_matches_the_pmf(mu):
    scipy_stats = pytest.importorskip("scipy.stats")
    n = 40_000
    x = synth.poisson(5, 2, 9, mu, n)
    kmax = int(mu + 6 * math.sqrt(mu) + 6)
    obs = np.bincount(np.minimum(x, kmax), minlength=kmax + 1).astype(np.float64)
    pmf = scipy_stats.poisson.pmf(np.arange(kmax + 1), mu)
    pmf[-1] = scipy_stats.poisson.sf(kmax - 1, mu)
    exp = n * pmf
    keep = exp >= 5
    stat = (((obs - exp) ** 2 / exp)[keep]).sum() + (
        (obs[~keep].sum() - exp[~keep].sum()) ** 2 / max(exp[~keep].sum(), 1e-300) if (~keep).any() else 0.0)
    dof = int(keep.sum()) + (1 if (~keep).any() else 0) - 1
    assert stat < scipy_stats.chi2.ppf(1 - 1e-4, dof), (stat, dof)


@pytest.mark.parametrize("mu", [150.0, 1234.5, 50_000.0])
def test_poisson_sampler_moments_for_large_means(mu):
    # large means are sums of pieces of at most 200: mean and variance mu
    n = 20_000
    x = synth.poisson(6, 3, 9, mu, n).astype(np.float64)
    se_mean = math.sqrt(mu / n)
    assert abs(x.mean() - mu) <= 5 * se_mean
    # the sample variance of a Poisson has standard error ~ mu sqrt(2 / n)
    assert abs(x.var() - mu) <= 5 * mu * math.sqrt(2.0 / n) + 1.0


def test_resource_lists_are_distinct_sorted_and_sum_to_poisson_total():
    r = small(I=200_000, J=400)
    im = synth.appendix_item_major(r)
    K = np.diff(im.col_ptr)
    assert (K >= 0).all() and (K <= r.I).all()
    for j in range(r.J):
        u = im.users[im.col_ptr[j]:im.col_ptr[j + 1]]
        assert ((u >= 0) & (u < r.I)).all()
        assert (np.diff(u) > 0).all()
    # no truncation here (the broadest resource is far below I), so sum K_j
    # is Poisson(I nu)
    assert K.max() < r.I // 4
    tot = r.I * r.nu
    assert abs(K.sum() - tot) <= 5 * math.sqrt(tot)


def test_truncation_at_the_number_of_requests_and_the_complement_draw():
    # few requests and a large nu: the broad resources ask for more than I
    r = small(I=500, J=30, nu=40.0)
    im = synth.appendix_item_major(r)
    K = np.diff(im.col_ptr)
    assert (K <= r.I).all()
    assert (K == r.I).any()  # truncated
    assert ((K > r.I // 2) & (K < r.I)).any()  # drawn by leaving requests out
    for j in range(r.J):
        u = im.users[im.col_ptr[j]:im.col_ptr[j + 1]]
        assert len(np.unique(u)) == len(u) and ((u >= 0) & (u < r.I)).all()


def test_picks_are_uniform_over_requests():
    # every request is equally likely to be picked by a resource: the
    # user-side degrees are sums of independent Bernoulli(K_j / I)
    r = small(I=2000, J=400, nu=8.0)
    im = synth.appendix_item_major(r)
    deg = np.bincount(im.users, minlength=r.I).astype(np.float64)
    K = np.diff(im.col_ptr).astype(np.float64)
    p = K / r.I
    mean, var = p.sum(), (p * (1 - p)).sum()
    assert abs(deg.mean() - mean) <= 5 * math.sqrt(var / r.I)
    # first and second halves of the request range are hit equally often
    half = deg[: r.I // 2].sum() - deg[r.I // 2:].sum()
    assert abs(half) <= 5 * math.sqrt(deg.sum())


def test_user_major_form_holds_the_item_major_edges():
    r = small()
    im = synth.appendix_item_major(r)
    inst = synth.generate_appendix(r)
    assert inst.nnz == len(im.users)
    item_of = np.repeat(np.arange(r.J), np.diff(im.col_ptr))
    a = np.sort(im.users * r.J + item_of)
    users = np.repeat(np.arange(r.I), np.diff(inst.row_ptr))
    b = users * r.J + inst.col.astype(np.int64)
    assert np.array_equal(np.sort(b), a)
    # rows list their resources in ascending order
    for i in range(r.I):
        row = inst.col[inst.row_ptr[i]:inst.row_ptr[i + 1]]
        assert (np.diff(row) > 0).all()


def test_values_capped_and_constraint_rows_are_scaled_values():
    r = small(I=20_000, J=200)
    inst = synth.generate_appendix(r)
    v = -inst.c.astype(np.float64)
    assert (v > 0).all() and v.max() <= r.c_max
    assert (v == r.c_max).any()  # the cap binds somewhere
    ratio = inst.a.astype(np.float64) / v
    for j in range(r.J):
        rj = ratio[inst.col == j]
        if len(rj):
            # a and c are float32 roundings of s_j * value and value
            assert np.abs(rj / rj[0] - 1).max() <= 2.5e-7
    # log s_j ~ N(0, 1.5): sample moments over the resources
    s = np.array([ratio[inst.col == j][0] for j in range(r.J) if (inst.col == j).any()])
    ls = np.log(s)
    assert abs(ls.mean() - r.s_mu) <= 5 * r.s_sigma / math.sqrt(len(ls))
    assert abs(ls.std() / r.s_sigma - 1) <= 0.2
    # log value = log v_j + log u_i + log eps_ij below the cap: std about 0.75
    lv = np.log(v[v < r.c_max])
    assert abs(lv.std() - math.sqrt(r.v_sigma ** 2 + r.u_sigma ** 2 + r.eps_sigma ** 2)) <= 0.1


def test_greedy_load_by_brute_force():
    r = small(I=5000, J=80)
    inst, load = synth.generate_appendix(r, want_load=True)
    ref = np.zeros(r.J)
    for i in range(r.I):
        lo, hi = inst.row_ptr[i], inst.row_ptr[i + 1]
        if hi == lo:
            continue
        best = lo
        for e in range(lo + 1, hi):
            if inst.a[e] > inst.a[best]:
                best = e
        ref[inst.col[best]] += float(inst.a[best])
    np.testing.assert_allclose(load, ref, rtol=1e-12, atol=0)
    rho = inst.b / (load + r.b_eps)
    assert (rho >= r.rho_lo).all() and (rho <= r.rho_hi).all()
    # rho_j ~ U[0.5, 1]: its mean over the resources
    assert abs(rho.mean() - 0.75) <= 5 * (0.5 / math.sqrt(12)) / math.sqrt(r.J)
    # some resources receive no greedy load and keep only rho_j eps_b
    assert (load == 0).any() and (load > 0).any()

"""Pins of the oracle's index-set enumerator, Philox generator, uniforms,
normals and sampling densities against values fixed outside the oracle:
the paper's printed cardinalities and counting formula (Sec. 2.4.2), closed
forms, published Philox4x32-10 known-answer vectors, and scipy's
distributions."""
import os
from math import comb

import numpy as np
import pytest
from scipy import integrate, stats

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KIND = {"TOTAL": 4, "HYP": 5}  # ORA_G_TOTAL_N, ORA_G_HYP_N


def _paper_counts():
    rows = []
    for line in open(os.path.join(GOLD, "gamma_counts_paper.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        kind, d, deg, cnt = line.split()[:4]
        rows.append((KIND[kind], int(d), int(deg), int(cnt)))
    return rows


@pytest.mark.parametrize("kind,d,deg,cnt", _paper_counts())
def test_gamma_counts_printed_in_paper(ora, kind, d, deg, cnt):
    assert ora.gamma_count(kind, d, deg) == cnt


def _factor(g):
    out, p = {}, 2
    while p * p <= g:
        while g % p == 0:
            out[p] = out.get(p, 0) + 1
            g //= p
        p += 1
    if g > 1:
        out[g] = out.get(g, 0) + 1
    return out


def _hyp_count_paper_formula(d, deg):
    """#Gamma_H(DEG) by the prime-factorisation recurrence of Sec. 2.4.2."""

    def n_upsilon(dd, g):
        r = 1
        for v in _factor(g).values():
            r *= comb(v + dd - 1, dd - 1)
        return r

    def n_gamma1(dd):
        return sum(n_upsilon(dd, g) for g in range(2, deg + 1)) + 1

    return n_gamma1(d) + sum(comb(d, c) * n_gamma1(d - c) for c in range(1, d)) + 1


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("deg", [1, 2, 5, 7, 12, 30])
def test_gamma_matches_paper_counting_formulas(ora, d, deg):
    assert ora.gamma_count(5, d, deg) == _hyp_count_paper_formula(d, deg)
    assert ora.gamma_count(4, d, deg) == comb(deg + d, d)  # #Gamma_T = C(DEG+d, d)
    assert ora.gamma_count(3, d, deg) == (deg + 1) ** d


@pytest.mark.parametrize("d,n", [(1, 3), (2, 4), (3, 3), (4, 4), (5, 2), (6, 5), (8, 3)])
def test_gamma_z_closed_forms(ora, d, n):
    assert ora.gamma_count(0, d, n) == (2 * n + 1) ** d
    assert ora.gamma_count(1, d, n) == sum(2 ** i * comb(d, i) * comb(n, i) for i in range(d + 1))


@pytest.mark.parametrize("kind,d,n", [(0, 2, 4), (1, 4, 4), (1, 6, 5), (2, 3, 6), (4, 3, 5), (5, 4, 6)])
def test_gamma_canonical_order(ora, kind, d, n):
    K = ora.gamma_list(kind, d, n)
    # strictly increasing in lexicographic order, k_1 most significant
    keys = [tuple(r) for r in K]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    # membership, brute force over the bounding box
    lo = -n if kind in (0, 1, 2) else 0
    grid = np.array(np.meshgrid(*[np.arange(lo, n + 1)] * d, indexing="ij")).reshape(d, -1).T
    a = np.abs(grid)
    member = {
        0: a.max(1) <= n, 1: a.sum(1) <= n, 2: np.maximum(a, 1).prod(1) <= n,
        3: a.max(1) <= n, 4: a.sum(1) <= n, 5: np.maximum(a, 1).prod(1) <= n,
    }[kind]
    assert sorted(map(tuple, grid[member])) == keys
    if kind in (0, 1, 2):
        # Z^d sets are symmetric: lexicographic order reverses under negation,
        # so index(-k) = |Gamma|-1-index(k) and k = 0 sits in the middle.
        idx = {k: e for e, k in enumerate(keys)}
        G = len(keys)
        assert all(idx[tuple(-np.array(k))] == G - 1 - e for e, k in enumerate(keys))
        assert keys[G // 2] == (0,) * d


def test_philox_known_answers(ora):
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        assert list(ora.philox(w[0:4], w[4:6])) == w[6:10]


def test_u01_bit_layout(ora):
    assert ora.u01(0, 0) == 2.0 ** -53
    assert ora.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    # n = (a << 20) ^ (b >> 12): a = 1, b = 0x1000 -> n = 2^20 + 1
    assert ora.u01(1, 0x1000) == (2 * (2 ** 20 + 1) + 1) * 2.0 ** -53
    # the low 12 bits of b never matter
    assert ora.u01(7, 0xFFF) == ora.u01(7, 0)


def test_start_uniforms_use_the_counter_layout(ora):
    seed, inst, i, m = 0x0123456789ABCDEF, 5, 7, 99
    u = ora.start_uniforms(seed, inst, i, m, 3)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    w0 = ora.philox([m, 0, 0xFFFFFFFF, (inst << 20) | (0 << 16) | i], key)
    w1 = ora.philox([m, 1, 0xFFFFFFFF, (inst << 20) | (0 << 16) | i], key)
    assert u[0] == ora.u01(w0[0], w0[1]) and u[1] == ora.u01(w0[2], w0[3])
    assert u[2] == ora.u01(w1[0], w1[1])


def test_uniforms_and_normals_distribution(ora):
    n = 20000
    u = np.array([ora.start_uniforms(11, 0, 3, m, 2) for m in range(n)]).ravel()
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    z = np.array([ora.normals(11, 0, 3, m, 2, 4) for m in range(n)]).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    # pairs of one Box-Muller call are uncorrelated
    zz = np.array([ora.normals(11, 0, 3, m, 2, 2) for m in range(n)])
    assert abs(np.corrcoef(zz.T)[0, 1]) < 5 / np.sqrt(n)
    # streams of different time steps are uncorrelated
    z5 = np.array([ora.normals(11, 0, 3, m, 5, 1)[0] for m in range(n)])
    assert abs(np.corrcoef(zz[:, 0], z5)[0, 1]) < 5 / np.sqrt(n)


@pytest.mark.parametrize("mu", [1.0, 3.0, 4.5])
def test_lomax_density_against_scipy(ora, mu):
    # |X| is Lomax(mu) and the sign is symmetric: F(x) = 1/2 + sign(x)/2 * lomax.cdf(|x|)
    for x in [0.0, 0.3, 1.0, 7.5, 1e3]:
        ref = 0.5 + 0.5 * stats.lomax(c=mu).cdf(x)
        assert ora.nu_cdf(0, mu, x) == pytest.approx(ref, rel=1e-13, abs=1e-15)
        assert ora.nu_cdf(0, mu, -x) == pytest.approx(1 - ref, rel=1e-12, abs=1e-15)
        assert ora.nu_pdf(0, mu, x) == pytest.approx(0.5 * stats.lomax(c=mu).pdf(x), rel=1e-13)
    tot = integrate.quad(lambda x: ora.nu_pdf(0, mu, x), -np.inf, 0)[0] + integrate.quad(
        lambda x: ora.nu_pdf(0, mu, x), 0, np.inf)[0]
    assert tot == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("kind,mu", [(0, 3.0), (1, 2.0), (2, 1.0)])
def test_inverse_cdf_round_trip(ora, kind, mu):
    us = np.concatenate([[2.0 ** -53, 2.0 ** -52, 1e-12, 1e-7, 0.25, 0.5, 0.75],
                         np.linspace(0.001, 0.999, 997), [1 - 1e-7, 1 - 2.0 ** -40]])
    for u in us:
        x = ora.nu_icdf(kind, mu, u)
        back = ora.nu_cdf(kind, mu, x)
        if kind == 0:
            # the double-Lomax forms are free of cancellation in both tails:
            # F(F^{-1}(u)) = u to a few ulp of u itself, even for u ~ 1e-16
            assert abs(back - u) <= 16 * np.spacing(u) + 4 * np.spacing(0.5 if u >= 0.5 else 0.0)
        else:
            # the closed forms of Sec. 5 add to 1/2 and, for mu = 2, form
            # -(u-1/2)^2 by cancellation: absolute accuracy of tens of ulp
            assert abs(back - u) <= 64 * np.spacing(1.0)


def test_student2_and_cauchy_against_scipy(ora):
    for x in [-30.0, -2.0, -0.1, 0.0, 0.4, 3.0, 100.0]:
        # nu is the density of X/sqrt(mu), X ~ Student t with mu = 2 dof (Example 1)
        assert ora.nu_cdf(1, 2.0, x) == pytest.approx(stats.t(df=2).cdf(np.sqrt(2) * x), rel=1e-12)
        assert ora.nu_pdf(1, 2.0, x) == pytest.approx(np.sqrt(2) * stats.t(df=2).pdf(np.sqrt(2) * x), rel=1e-12)
        assert ora.nu_cdf(2, 1.0, x) == pytest.approx(stats.cauchy.cdf(x), rel=1e-12)


def test_sampled_start_points_follow_nu(ora):
    n = 20000
    x = np.array([ora.nu_icdf(0, 3.0, ora.start_uniforms(4, 0, 0, m, 1)[0]) for m in range(n)])
    assert stats.kstest(x, lambda t: 0.5 + 0.5 * np.sign(t) * stats.lomax(c=3.0).cdf(np.abs(t))).pvalue > 1e-4

"""Pins of the oracle's QRMC iteration (Sec. 2.3, Algorithm 1) against results
fixed by the mathematics rather than by the oracle itself:

* exact recovery of a planted trigonometric polynomial on a lattice (basis,
  conjugation, 1/M normalisation, Gamma order, all at once);
* the linear driver f = lambda*y, whose discrete solution is (1+lambda dt)^{N-i}
  times the terminal polynomial (pins "f at t_j, y at j+1, dt-weighted");
* Feynman-Kac with f = 0 and a drift, against exact coefficients computed by
  1-D quadrature (Euler scheme, Brownian scaling, drift sign, conj convention);
* sampled orthonormality of phi_k under nu (Lemma eqInnerNorms);
* Picard iterate N == backward sweep, bit for bit (same clouds);
* linearity of the estimator in the path range;
* the manufactured cubic PDE: its driver solves the PDE (finite differences)
  and the estimate approaches the exact projection of the solution.
"""
import numpy as np
import pytest
from scipy import integrate

from paper_2407_21084_b300 import workloads as W


def _planted_coefs(rng, K):
    """Random conjugate-symmetric coefficients on a symmetric Z^d set."""
    idx = {tuple(k): e for e, k in enumerate(K)}
    c = rng.normal(size=len(K)) + 1j * rng.normal(size=len(K))
    for e, k in enumerate(K):
        e2 = idx[tuple(-k)]
        if e2 == e:
            c[e] = c[e].real
        elif e2 < e:
            c[e] = np.conj(c[e2])
    return c


def _lattice_problem(ora, d, kind, n, lat, N, f_kind, f_par, c):
    K = ora.gamma_list(kind, d, n)
    return ora.Problem(d=d, N=N, T=1.0, k=K, b=np.zeros(d), sigma=np.zeros((d, d)),
                       f_kind=f_kind, f_par=f_par, g_kind=ora.GT_TRIGPOLY,
                       g_par=c.view(np.float64), M=lat ** d, seed=1, lattice_n=lat)


@pytest.mark.parametrize("d,kind,n", [(1, 0, 3), (2, 0, 2), (3, 1, 2), (4, 1, 2)])
def test_planted_polynomial_exact_recovery(ora, d, kind, n):
    rng = np.random.default_rng(100 + d)
    K = ora.gamma_list(kind, d, n)
    c = _planted_coefs(rng, K)
    lat = 2 * n + 1  # lattice sums are exact for |k_l - k'_l| < lat
    p = _lattice_problem(ora, d, kind, n, lat, 3, ora.F_ZERO, [0.0], c)
    a, _ = ora.picard(p, 1)
    assert np.abs(a - c[None, :]).max() < 1e-12 * max(1.0, np.abs(c).max())
    # and the series reproduces g at arbitrary points
    x = rng.normal(size=(5, d))
    assert np.allclose(ora.series(p, a[0], x), ora.g(p, x), atol=1e-11)


def test_linear_driver_closed_form(ora):
    d, n, lat, N, lam = 2, 2, 5, 4, 0.7
    rng = np.random.default_rng(7)
    K = ora.gamma_list(0, d, n)
    c = _planted_coefs(rng, K)
    p = _lattice_problem(ora, d, 0, n, lat, N, ora.F_LINEAR, [lam], c)
    dt = 1.0 / N
    a1, _ = ora.picard(p, 1)
    # first iterate from y == 0: only the terminal step sees g, so (1 + lam dt) c
    assert np.abs(a1 - (1 + lam * dt) * c[None, :]).max() < 1e-12
    aN, _ = ora.picard(p, N)
    for i in range(N):
        assert np.abs(aN[i] - (1 + lam * dt) ** (N - i) * c).max() < 1e-11


def _fk_exact(s, k, nu_pdf, nu_cdf, X=200.0):
    """int e^{i s x} e^{-2 pi i k F(x)} nu(x) dx on [-X, X] by panel quadrature."""
    def re(x):
        return np.cos(s * x - 2 * np.pi * k * nu_cdf(x)) * nu_pdf(x)

    def im(x):
        return np.sin(s * x - 2 * np.pi * k * nu_cdf(x)) * nu_pdf(x)

    edges = np.concatenate([-np.geomspace(X, 1, 30), [0.0], np.geomspace(1, X, 30)])
    tot = 0j
    for lo, hi in zip(edges[:-1], edges[1:]):
        tot += integrate.quad(re, lo, hi, limit=200, epsabs=1e-13)[0]
        tot += 1j * integrate.quad(im, lo, hi, limit=200, epsabs=1e-13)[0]
    return tot


def _lomax(mu):
    def pdf(x):
        return 0.5 * mu * (1 + np.abs(x)) ** (-mu - 1)

    def cdf(x):
        return np.where(x < 0, 0.5 * (1 + np.abs(x)) ** (-mu), 1 - 0.5 * (1 + np.abs(x)) ** (-mu))

    return pdf, cdf


def test_feynman_kac_zero_driver(ora):
    d, N, T, sig0, M = 2, 4, 1.0, 0.5, 2 ** 18
    s = np.array([1.0, 0.5])
    bvec = np.array([0.3, -0.2])
    K = ora.gamma_list(0, d, 2)
    p = ora.Problem(d=d, N=N, T=T, k=K, b=bvec, sigma=sig0 * np.eye(d), f_kind=ora.F_ZERO,
                    f_par=[0.0], g_kind=ora.GT_COS, g_par=s, M=M, seed=21)
    a, _ = ora.picard(p, 1)
    pdf, cdf = _lomax(3.0)
    I = {}
    for l in range(d):
        for kk in range(-2, 3):
            I[(l, kk, 1)] = _fk_exact(s[l], kk, pdf, cdf)
            I[(l, kk, -1)] = _fk_exact(-s[l], kk, pdf, cdf)
    tol = 5.0 / np.sqrt(M)  # |S conj(phi)| <= 1, so 5 standard errors
    worst, max_im = 0.0, 0.0
    for i in range(N):
        tau = T - i * T / N
        # y_i(x) = E cos(s.(x + b tau + sig0 W_tau)) = cos(s.x + s.b tau) e^{-sig0^2 |s|^2 tau / 2}
        ph = s @ bvec * tau
        decay = np.exp(-0.5 * sig0 ** 2 * (s @ s) * tau)
        for e, k in enumerate(K):
            plus = np.prod([I[(l, k[l], 1)] for l in range(d)])
            minus = np.prod([I[(l, k[l], -1)] for l in range(d)])
            ex = decay * 0.5 * (np.exp(1j * ph) * plus + np.exp(-1j * ph) * minus)
            worst = max(worst, abs(a[i, e] - ex))
            max_im = max(max_im, abs(ex.imag))
    assert worst < tol
    # the drift makes the exact coefficients complex: projecting on phi_k instead
    # of conj(phi_k) would conjugate them, an error of 2|Im| > 3 tol
    assert 2 * max_im > 3 * tol


def test_sampled_orthonormality(ora):
    d, M = 2, 4096
    K = ora.gamma_list(0, d, 2)
    nG = len(K)
    p = ora.Problem(d=d, N=1, T=1.0, k=K, b=np.zeros(d), sigma=np.eye(d), f_kind=0, f_par=[0.0],
                    g_kind=0, g_par=np.zeros(d), M=M, seed=3)
    X = np.array([[ora.nu_icdf(0, 3.0, u) for u in ora.start_uniforms(3, 0, 0, m, d)]
                  for m in range(M)])
    Phi = np.zeros((M, nG), dtype=complex)
    for e in range(nG):
        a = np.zeros(nG, dtype=complex)
        a[e] = 1.0
        re = ora.series(p, a, X)
        a[e] = 1j
        im = -ora.series(p, a, X)  # Re(i phi) = -Im(phi)
        Phi[:, e] = re + 1j * im
    G = Phi.T @ Phi.conj() / M
    bound = 5 * np.sqrt(2 * np.log(nG ** 2) / M)
    assert np.abs(G - np.eye(nG)).max() < bound
    assert np.allclose(np.abs(Phi), 1.0, atol=1e-13)


def _c1_small(ora, M=2 ** 10, N=4):
    w = W.c1()
    K = ora.gamma_list(w.gamma_kind, w.d, w.gamma_n)
    return ora.Problem(d=w.d, N=N, T=w.T, k=K, b=w.b, sigma=w.sigma, f_kind=ora.F_CUBIC_MANUF,
                       f_par=w.f_par, g_kind=ora.GT_COS, g_par=w.g_par, M=M, seed=w.seed,
                       clamp_L=w.clamp_L)


def test_picard_N_equals_backward_sweep_bitwise(ora):
    p = _c1_small(ora)
    aq, _ = ora.picard(p, p.N)
    ab, _ = ora.backward_sweep(p)
    assert np.array_equal(aq.view(np.float64), ab.view(np.float64))
    # and fewer iterations have not converged yet on the earliest rows
    a1, _ = ora.picard(p, 1)
    assert np.abs(a1[0] - ab[0]).max() > 1e-6
    assert np.array_equal(a1[p.N - 1].view(np.float64), ab[p.N - 1].view(np.float64))


def test_linearity_in_path_range(ora):
    p = _c1_small(ora, M=3000)
    a0 = ora.picard(p, 1)[0]
    Mp = 1234
    a_lo = ora.picard_iter(p, p.zeros(), m_range=(0, Mp))[0]
    a_hi = ora.picard_iter(p, p.zeros(), m_range=(Mp, p.M))[0]
    comb = (Mp * a_lo + (p.M - Mp) * a_hi) / p.M
    assert np.abs(a0 - comb).max() < 1e-13


def test_manufactured_driver_solves_the_pde(ora):
    for w in (W.c1(), W.c2()):
        K = ora.gamma_list(0, w.d, 1)
        p = ora.Problem(d=w.d, N=w.N, T=w.T, k=K, b=w.b, sigma=w.sigma, f_kind=ora.F_CUBIC_MANUF,
                        f_par=w.f_par, g_kind=ora.GT_COS, g_par=w.g_par, M=1, seed=0)
        rng = np.random.default_rng(5)
        h = 1e-4
        for _ in range(5):
            t = rng.uniform(0, 1)
            x = rng.normal(size=w.d)

            def u(tt, xx):
                return w.exact_u(tt, xx)[0]

            dtu = (u(t + h, x) - u(t - h, x)) / (2 * h)
            lap = sum((u(t, x + h * np.eye(w.d)[l]) - 2 * u(t, x) + u(t, x - h * np.eye(w.d)[l])) / h ** 2
                      for l in range(w.d))
            res = dtu + 0.5 * w.sigma0 ** 2 * lap + ora.f(p, t, x, u(t, x))
            assert abs(res) < 1e-5
        # terminal condition
        assert ora.g(p, np.ones((1, w.d)))[0] == pytest.approx(w.exact_u(w.T, np.ones(w.d))[0])


def test_manufactured_cubic_approaches_projection_of_exact_solution(ora):
    """C1 problem. By Parseval, ||ybar_i - P_Gamma u(t_i)||_nu = |alpha_i - c_i|_2
    where c_i = e^{a(T-t_i)} <cos(s.x), phi_k>_nu are exact projection coefficients
    (1-D quadrature, as in the Feynman-Kac pin). Theorem th:main bounds this by
    the variance term ~ Lambda_Gamma/M plus propagated truncation: it must shrink
    with M, like M^-1/2 on the last row (y_N = g is exact there)."""
    w = W.c1()
    K = ora.gamma_list(w.gamma_kind, w.d, w.gamma_n)
    pdf, cdf = _lomax(w.mu)
    kmax = w.gamma_n
    Ip = {(l, k): _fk_exact(w.s[l], k, pdf, cdf) for l in range(w.d) for k in range(-kmax, kmax + 1)}
    Im = {(l, k): _fk_exact(-w.s[l], k, pdf, cdf) for l in range(w.d) for k in range(-kmax, kmax + 1)}
    c = np.array([0.5 * (np.prod([Ip[(l, k[l])] for l in range(w.d)])
                         + np.prod([Im[(l, k[l])] for l in range(w.d)])) for k in K])

    def excess(M):
        p = ora.Problem(d=w.d, N=w.N, T=w.T, k=K, b=w.b, sigma=w.sigma, f_kind=ora.F_CUBIC_MANUF,
                        f_par=w.f_par, g_kind=ora.GT_COS, g_par=w.g_par, M=M, seed=w.seed,
                        clamp_L=w.clamp_L)
        a, _ = ora.backward_sweep(p)
        return np.array([np.sqrt(np.sum(np.abs(a[i] - np.exp(w.a * (w.T - i * w.T / w.N)) * c) ** 2))
                         for i in range(w.N)])

    e_small, e_big = excess(2 ** 12), excess(2 ** 16)
    assert np.all(e_big < e_small)
    assert e_big[-1] < 0.05
    assert e_small[-1] / e_big[-1] > 2.5  # sqrt(16) = 4 in the pure-variance regime
    assert e_big.max() < 0.12


def _lattice_recursion(Phi, gvals, N, lam, L, n_iter, where="y_next"):
    """The Jacobi-Picard iteration of Algorithm 1 written out in numpy for
    paths that stand still (sigma = 0, b = 0, start points on the centred
    lattice), f = lam*y: S_i = g + lam dt sum_{j=i}^{N-1} y_{j+1} with
    y_N = g and, for j+1 < N, y_{j+1} = T_L(ybar_{j+1}) (eq. Sqi:bar:M with
    the truncation of eq. TL:2); alpha_i = Phi^H S_i / M (eq. Aqi:bar:M);
    ybar_i = Re Phi alpha_i. `where` moves the truncation elsewhere (to
    show that the pin tells the placements apart): "none", "g" (also on
    y_N), "f" (on lam*y instead of y), "S" (on the response)."""
    M = Phi.shape[0]
    dt = 1.0 / N
    alpha = np.zeros((N, Phi.shape[1]), dtype=complex)
    hits = 0

    def clamp(v):
        return np.clip(v, -L, L)

    for _ in range(n_iter):
        ybar = (Phi @ alpha.T).real  # M x N: ybar_j at the lattice points
        new = np.empty_like(alpha)
        for i in range(N):
            S = gvals.copy() if where != "g" else clamp(gvals)
            for j in range(i, N):
                if j + 1 == N:
                    y1 = clamp(gvals) if where == "g" else gvals
                else:
                    y1 = ybar[:, j + 1]
                    if where == "y_next":
                        hits += int(np.count_nonzero(np.abs(y1) > L))
                        y1 = clamp(y1)
                term = lam * y1
                if where == "f" and j + 1 < N:
                    term = clamp(term)
                S = S + term * dt
            if where == "S":
                S = clamp(S)
            new[i] = Phi.conj().T @ S / M
        alpha = new
    return alpha, hits


def _clamp_case(ora):
    d, kind, n, lat, N, lam = 2, 0, 2, 5, 4, 0.7
    K = ora.gamma_list(kind, d, n)
    c = _planted_coefs(np.random.default_rng(31), K)
    c *= 0.25
    p = _lattice_problem(ora, d, kind, n, lat, N, ora.F_LINEAR, [lam], c)
    # lattice points in the oracle's order (dimension 0 = least significant digit)
    m = np.arange(lat ** d)
    U = np.stack([((m // lat ** l) % lat + 0.5) / lat for l in range(d)], axis=1)
    Phi = np.exp(2j * np.pi * (U @ K.T))
    gvals = (Phi @ c).real
    L = 0.6 * np.abs(gvals).max()  # below max|y|: the truncation binds
    p.clamp_L = L
    return p, Phi, gvals, N, lam, L


def test_truncation_TL_placement_on_lattice(ora):
    """T_L of eq. (TL:2) applied where eq. (Sqi:bar:M) puts it: to the
    previous iterate's series ybar_{j+1}(X_{j+1}) before the driver, not to
    g = y_N, not to f's output, not to the response. With standing paths on
    a lattice the whole scheme is a few numpy products, so the oracle's
    clamped Picard iterates are fixed independently, and the clamp count is
    the number of series values beyond L."""
    p, Phi, gvals, N, lam, L = _clamp_case(ora)
    for q in (1, 2, N):
        ref, hits_ref = _lattice_recursion(Phi, gvals, N, lam, L, q)
        a, hits = ora.picard(p, q)
        scale = np.abs(ref).max()
        assert np.abs(a - ref).max() < 1e-12 * scale
        assert hits == hits_ref
    assert hits_ref > 0
    # every other placement gives a visibly different fixed point
    for where in ("none", "g", "f", "S"):
        alt, _ = _lattice_recursion(Phi, gvals, N, lam, L, N, where=where)
        assert np.abs(alt - ref).max() > 1e-3 * scale, where

"""Pins of the damping exponent q of eq. (yqi) in the oracle: the series
represents ybar^q = y / (1 + |x|^2)^{q/2}; the response of eq. (Sqi:bar:M)
multiplies the series at X_{j+1} by the weight and divides the whole
response by the weight at the start point X_i^i.

* sigma = 0 on a midpoint lattice with the linear driver f = lambda y: every
  path stays at its start point, so the backward sweep gives exactly
  ybar^q_i = (1 + lambda dt)^{N-i} P[g / w], P the lattice projection,
  computed here independently with numpy (a missing weight at X_{j+1} or at
  X_i^i breaks the power law);
* Feynman-Kac with f = 0, Brownian motion and g = cos(s x): the damped
  coefficients against y_i(x) / (1 + x^2)^{q/2}, y_i = cos(s x)
  e^{-s^2 (T - t_i)/2}, projected by quadrature;
* q = 0 leaves the scheme bit for bit unchanged.
"""
import numpy as np
import pytest


def _student2_icdf(u):
    return (u - 0.5) / np.sqrt(u * (1.0 - u))


@pytest.mark.parametrize("q", [2.1, 5.1])
def test_damped_linear_driver_on_lattice(ora, q):
    d, n, lat, N, lam = 2, 2, 7, 4, 0.7
    rng = np.random.default_rng(31)
    K = ora.gamma_list(ora.G_LINF_Z, d, n)
    idx = {tuple(k): e for e, k in enumerate(K)}
    c = rng.normal(size=len(K)) + 1j * rng.normal(size=len(K))
    for e, k in enumerate(K):  # conjugate symmetry: g real
        e2 = idx[tuple(-k)]
        if e2 == e:
            c[e] = c[e].real
        elif e2 < e:
            c[e] = np.conj(c[e2])
    p = ora.Problem(d=d, N=N, T=1.0, k=K, b=np.zeros(d), sigma=np.zeros((d, d)), f_kind=ora.F_LINEAR,
                    f_par=[lam], g_kind=ora.GT_TRIGPOLY, g_par=c.view(np.float64), M=lat ** d, seed=1,
                    lattice_n=lat, nu_kind=ora.NU_STUDENT2, mu=2.0, q_damp=q)
    a, _ = ora.backward_sweep(p)
    # independent lattice projection of g / w (digit l of m is coordinate l)
    g1 = (np.arange(lat) + 0.5) / lat
    U = np.array([[g1[(m // lat ** l) % lat] for l in range(d)] for m in range(lat ** d)])
    X = _student2_icdf(U)
    phase = np.exp(2j * np.pi * U @ K.T)  # (M, |Gamma|)
    gx = (phase @ c).real
    w = (1.0 + (X * X).sum(1)) ** (q / 2)
    h = (gx / w) @ np.conj(phase) / len(U)
    dt = 1.0 / N
    for i in range(N):
        assert np.allclose(a[i], (1 + lam * dt) ** (N - i) * h, rtol=1e-11, atol=1e-12), i


def test_damped_feynman_kac(ora):
    s, q, N, M, n = 0.7, 2.1, 4, 2 ** 16, 4
    K = ora.gamma_list(ora.G_LINF_Z, 1, n)
    p = ora.Problem(d=1, N=N, T=1.0, k=K, b=np.zeros(1), sigma=np.eye(1), f_kind=ora.F_ZERO, f_par=[0.0],
                    g_kind=ora.GT_COS, g_par=[s], M=M, seed=5, nu_kind=ora.NU_STUDENT2, mu=2.0, q_damp=q)
    a, _ = ora.backward_sweep(p)
    # exact damped coefficients: int y_i(x) (1 + x^2)^{-q/2} e^{-2 pi i k F(x)} nu(x) dx on a fine grid
    x = np.linspace(-400.0, 400.0, 1_600_001)
    nu = 0.5 * (1 + x * x) ** -1.5
    F = 0.5 * (x / np.sqrt(x * x + 1) + 1)
    for i in range(N):
        y = np.cos(s * x) * np.exp(-s * s * (1.0 - i / N) / 2) * (1 + x * x) ** (-q / 2)
        ex = np.array([np.trapezoid(y * np.exp(-2j * np.pi * k[0] * F) * nu, x) for k in K])
        assert np.abs(a[i] - ex).max() < 5.0 / np.sqrt(M), i


def test_zero_damping_is_bitwise_the_undamped_scheme(ora):
    K = ora.gamma_list(ora.G_L1_Z, 2, 3)
    kw = dict(d=2, N=3, T=1.0, k=K, b=np.zeros(2), sigma=0.4 * np.eye(2), f_kind=ora.F_CUBIC_MANUF,
              f_par=[0.2, 1.0, 0.5], g_kind=ora.GT_COS, g_par=[1.0, 0.5], M=4096, seed=2, clamp_L=2.0)
    a0, _ = ora.picard(ora.Problem(**kw), 2)
    a1, _ = ora.picard(ora.Problem(**kw, q_damp=0.0), 2)
    assert np.array_equal(a0.view(np.float64), a1.view(np.float64))

"""Seeded synthetic workloads of the QRMC Picard benchmark.

This module holds no arithmetic of the method: it only fixes the problem
parameters (dimension, grid, index set, PDE coefficients, path counts, seeds)
that both the CUDA path and the CPU oracle are run on. Random problem
parameters (the wave vector ``s``) are drawn here with numpy's PCG64 from a
stated seed; the random numbers the method itself draws (start points and
Brownian increments) come from Philox inside each implementation.

The manufactured PDE is  d_t u + (1/2) sigma0^2 Lap u + f(t,x,u) = 0,
u(t,x) = e^{a(T-t)} cos(s.x),  f = -y^3 + r(t,x),  g = cos(s.x).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import comb, exp

import numpy as np

# index-set kinds (same numbering in the C-ABI and the oracle)
G_LINF_Z, G_L1_Z, G_HYP_Z, G_FULL_N, G_TOTAL_N, G_HYP_N = range(6)
NU_LOMAX, NU_STUDENT2, NU_CAUCHY = range(3)
F_ZERO, F_LINEAR, F_CUBIC_MANUF, F_PAPER_MIN = range(4)
GT_COS, GT_TRIGPOLY, GT_PAPER_SIN = range(3)


@dataclass
class Workload:
    name: str
    d: int
    N: int
    T: float
    sigma0: float
    gamma_kind: int
    gamma_n: int
    M: int
    n_iter: int
    a: float
    s: np.ndarray
    seed: int
    nu_kind: int = NU_LOMAX
    mu: float = 3.0
    n_test: int = 4096
    b: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.b is None:
            self.b = np.zeros(self.d)
        self.b = np.asarray(self.b, dtype=np.float64)
        self.s = np.asarray(self.s, dtype=np.float64)
        if self.b.shape != (self.d,) or self.s.shape != (self.d,):
            raise ValueError("b and s must have d = %d entries" % self.d)

    @property
    def sigma(self) -> np.ndarray:
        return self.sigma0 * np.eye(self.d)

    @property
    def clamp_L(self) -> float:
        """Constant truncation level 2 e^{aT} max|g| (max|cos| = 1)."""
        return 2.0 * exp(self.a * self.T)

    @property
    def f_par(self) -> np.ndarray:
        return np.concatenate([[self.a], self.s])

    @property
    def g_par(self) -> np.ndarray:
        return self.s.copy()

    def n_gamma(self) -> int:
        return gamma_size(self.gamma_kind, self.d, self.gamma_n)

    def evals_per_iter(self) -> float:
        """path.coef evaluations per Picard iteration: M |Gamma| N(N+1)/2."""
        return float(self.M) * self.n_gamma() * self.N * (self.N + 1) / 2.0

    def exact_u(self, t: float, x: np.ndarray) -> np.ndarray:
        return np.exp(self.a * (self.T - t)) * np.cos(np.atleast_2d(x) @ self.s)

    def with_(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        if "d" in kw and "b" not in kw:
            d["b"] = None  # the drift follows the dimension (zero)
        d.update(kw)
        return Workload(**d)


def gamma_size(kind: int, d: int, n: int) -> int:
    """Closed-form |Gamma| for the Z^d sets used by the workloads."""
    if kind == G_LINF_Z:
        return (2 * n + 1) ** d
    if kind == G_L1_Z:
        return sum(2 ** i * comb(d, i) * comb(n, i) for i in range(min(d, n) + 1))
    raise ValueError("closed form only for |k|_inf and |k|_1 sets")


def _s(seed: int, d: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=d)


def c1() -> Workload:
    """d=2, N=8, M=2^14, |k|_inf<=4 (81 coefs), sigma0=0.5, 3 iterations, seed 1."""
    return Workload("c1_d2_N8_M16384_linf4", d=2, N=8, T=1.0, sigma0=0.5, gamma_kind=G_LINF_Z,
                    gamma_n=4, M=2 ** 14, n_iter=3, a=0.2, s=[1.0, 0.5], seed=1)


def c2() -> Workload:
    """d=4, N=16, M=2^20, |k|_1<=4 (321 coefs), sigma0=0.4, 5 iterations, s~U[-1,1]^4 (seed 2)."""
    return Workload("c2_d4_N16_M1048576_l1_4", d=4, N=16, T=1.0, sigma0=0.4, gamma_kind=G_L1_Z,
                    gamma_n=4, M=2 ** 20, n_iter=5, a=0.2, s=_s(2, 4), seed=2)


def c3() -> Workload:
    """d=6, N=32, M=2^22, |k|_1<=5 (3653 coefs), sigma0=0.3, s~U[-1,1]^6 (seed 3)."""
    return Workload("c3_d6_N32_M4194304_l1_5", d=6, N=32, T=1.0, sigma0=0.3, gamma_kind=G_L1_Z,
                    gamma_n=5, M=2 ** 22, n_iter=1, a=0.2, s=_s(3, 6), seed=3)


# index-set class per dimension for the multi-instance workload (the engine
# compiles these classes): |Gamma| from 81 to 1289
C4_CLASSES = {2: [(G_LINF_Z, 4)], 3: [(G_L1_Z, 5)], 4: [(G_L1_Z, 4)], 5: [(G_L1_Z, 4)],
              6: [(G_L1_Z, 3), (G_L1_Z, 4)], 7: [(G_L1_Z, 3)], 8: [(G_L1_Z, 3)]}


def c4(n_instances: int = 256, n_shared: int = 64, M: int = 2 ** 18, seed: int = 4) -> list:
    """Many independent problems of uneven size: d ~ U{2..8} with the index
    set of C4_CLASSES (|Gamma| 81..1289), N ~ U{8,16,32}, sigma0 ~ U[0.2,0.6],
    a ~ U[0,0.5], s ~ U[-1,1]^d, M paths each. The last n_shared instances
    share their sample points (same d, N, sigma0, index set, seed and Philox
    instance; only a and s differ)."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n_instances - n_shared):
        d = int(rng.integers(2, 9))
        kind, n = C4_CLASSES[d][int(rng.integers(len(C4_CLASSES[d])))]
        out.append(Workload("c4_inst%03d_d%d" % (q, d), d=d, N=int(rng.choice([8, 16, 32])), T=1.0,
                            sigma0=float(rng.uniform(0.2, 0.6)), gamma_kind=kind, gamma_n=n, M=M, n_iter=1,
                            a=float(rng.uniform(0.0, 0.5)), s=rng.uniform(-1.0, 1.0, size=d), seed=4000 + q))
    if n_shared:
        d, sig = 6, float(rng.uniform(0.2, 0.6))
        for q in range(n_shared):
            out.append(Workload("c4_shared%02d_d6" % q, d=d, N=16, T=1.0, sigma0=sig, gamma_kind=G_L1_Z, gamma_n=3,
                                M=M, n_iter=1, a=float(rng.uniform(0.0, 0.5)), s=rng.uniform(-1.0, 1.0, size=d),
                                seed=4999))
    return out


@dataclass
class Sec5Problem:
    """The test problem of Sec. 5 of the paper: dX = dW (sigma = I, b = 0),
    g = 1 + kappa + sin(lam sum x), f = min(1, [y - kappa - 1 - sin(lam sum x)
    e^{lam^2 d (t-T)/2}]^2), exact solution u = 1 + kappa + sin(lam sum x)
    e^{lam^2 d (t-T)/2}; kappa = 0.6, lam = 1/sqrt(d), T = 1; Student nu with
    mu = 2 (nu_kind NU_CAUCHY: mu = 1, the choice of the paper's tables with
    mixed-derivative damping exponents); cosine basis on an N^d set
    (Gamma_F, Gamma_T or Gamma_H); damping exponent q of eq. (yqi)."""

    d: int
    N: int
    gamma_kind: int
    gamma_n: int
    M: int
    seed: int
    T: float = 1.0
    kappa: float = 0.6
    q: float = 0.0  # damping exponent of eq. (yqi)
    nu_kind: int = NU_STUDENT2  # or NU_CAUCHY

    @property
    def mu(self) -> float:
        return 1.0 if self.nu_kind == NU_CAUCHY else 2.0

    @property
    def lam(self) -> float:
        return 1.0 / np.sqrt(self.d)

    @property
    def sigma(self) -> np.ndarray:
        return np.eye(self.d)

    @property
    def b(self) -> np.ndarray:
        return np.zeros(self.d)

    @property
    def f_par(self) -> np.ndarray:
        return np.array([self.kappa, self.lam])

    @property
    def g_par(self) -> np.ndarray:
        return np.array([self.kappa, self.lam])

    def exact_u(self, t: float, x: np.ndarray) -> np.ndarray:
        sx = np.atleast_2d(x).sum(axis=1)
        return 1.0 + self.kappa + np.sin(self.lam * sx) * np.exp(self.lam ** 2 * self.d * (t - self.T) / 2.0)


def sec5_d1(K: int, N: int, M: int, seed: int, q: float = 0.0) -> Sec5Problem:
    """d = 1 rows of the paper's Sec. 5 (Delta = 1/N, K + 1 cosines, M paths)."""
    return Sec5Problem(d=1, N=N, gamma_kind=G_FULL_N, gamma_n=K, M=M, seed=seed, q=q)


CONFIGS = {"c1": c1, "c2": c2, "c3": c3}

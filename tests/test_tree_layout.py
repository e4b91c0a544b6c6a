"""Host pin of the coefficient layout of the compile-time tree kernels
(qr_tree_layout, no device): the series evaluated slot by slot in the order
the kernels' traversal reads them (root, chain trees in Horner form, +-1 leaf
pairs and mirrored last-dimension chains as coefficient pairs, the mirrored
chains of the dimensions before it as sum and difference subtrees against
their powers) must equal the plain definition y(z) = Re sum_{k in Gamma}
alpha_k prod_l z_l^{k_l} (alpha_{-k} = conj alpha_k) at random phases, for
every compiled set shape; a sign or an index wrong anywhere in the layout
fails it. The traversal below is transcribed from the rules the kernels
follow, in FP64 complex arithmetic."""
import itertools

import numpy as np
import pytest

LINF, L1 = 0, 1


@pytest.fixture(scope="module")
def layout():
    from paper_2407_21084_b300 import build, solver

    build.build()
    return solver.tree_layout


def gamma(kind, d, n):
    out = []
    for k in itertools.product(range(-n, n + 1), repeat=d):
        a = np.abs(k)
        if (kind == LINF and a.max() <= n) or (kind == L1 and a.sum() <= n):
            out.append(k)
    return np.array(out)  # lexicographic = canonical order


def series_by_layout(slots, z, D, NN, kind, levels):
    l1 = kind == L1

    def ext_ok(S):
        return S >= 1 if l1 else S < NN

    def ext_S(S):
        return S - 1 if l1 else S + 1

    def new_ok(S):
        return S >= 1 if l1 else True

    def new_S(S):
        return S - 1 if l1 else 1

    def leaf(L, S):
        return S == 0 if l1 else (S == NN and L == D - 1)

    def chain_len(S):
        return 1 + ((1 if leaf(D - 1, ext_S(S)) else chain_len(ext_S(S))) if ext_ok(S) else 0)

    npow = max(1, NN - 1 if l1 else NN)
    nlv = min(levels, D - 2) if D > 2 else 0
    zl = [z[D - 1] ** (m + 1) for m in range(npow)]
    zk = [[z[D - 2 - v] ** (m + 1) for m in range(npow)] for v in range(nlv)]
    off = [1]

    def take():
        s = slots[off[0]]
        off[0] += 1
        return s

    def pair_acc(T, ac, be, w):
        # T += c+ w + c- conj(w) from the pre-combined slots (A, C), (B, E)
        return T + complex(ac[0] * w.real + be[0] * w.imag, ac[1] * w.imag + be[1] * w.real)

    def newdims(L2, S, T):
        for l2 in range(L2, D):
            S2 = new_S(S)
            if leaf(l2, S2):
                ac, be = take(), take()
                T = pair_acc(T, ac, be, z[l2])
            elif l2 == D - 1:
                for mm in range(chain_len(S2)):
                    ac, be = take(), take()
                    T = pair_acc(T, ac, be, zl[mm])
            elif l2 <= D - 2 and l2 >= D - 1 - nlv:
                T = pairchain(l2, S2, 0, T)
            else:
                for w in (z[l2], np.conj(z[l2])):
                    T = T + w * node(l2, S2, w)
        return T

    def pairchain(L, S2, MM, T):
        A, B = complex(*take()), complex(*take())
        if not leaf(L, S2) and new_ok(S2):
            A = newdims(L + 1, S2, A)
            B = newdims(L + 1, S2, B)
        w = zk[D - 2 - L][MM]
        T = T + A * w.real + B * w.imag
        if not leaf(L, S2) and ext_ok(S2):
            T = pairchain(L, ext_S(S2), MM + 1, T)
        return T

    def node(L, S, wl):
        T = complex(*take())
        if ext_ok(S):
            S2 = ext_S(S)
            if leaf(L, S2):
                T = T + complex(*take()) * wl
            else:
                T = T + wl * node(L, S2, wl)
        if new_ok(S):
            T = newdims(L + 1, S, T)
        return T

    T = complex(*slots[0])
    S0 = NN - 1 if l1 else 1
    for L in range(D):
        if leaf(L, S0):
            T = T + complex(*take()) * z[L]
        else:
            T = T + z[L] * node(L, S0, z[L])
    assert off[0] == len(slots)
    return T.real


@pytest.mark.parametrize("kind,d,n", [(LINF, 1, 3), (LINF, 2, 2), (LINF, 2, 4), (LINF, 3, 2), (L1, 3, 2),
                                      (L1, 3, 5), (L1, 4, 4), (L1, 5, 4), (L1, 6, 3), (L1, 6, 5), (L1, 7, 3),
                                      (L1, 8, 3)])
def test_layout_reproduces_the_series(layout, kind, d, n):
    idx, coef = layout(kind, d, n)
    K = gamma(kind, d, n)
    assert idx.shape[0] == (len(K) + 1) // 2
    levels = int(np.log2(idx.shape[2])) - 1
    rng = np.random.default_rng(d * 31 + n)
    z0 = len(K) // 2
    alpha = np.zeros(len(K), dtype=complex)
    alpha[z0] = rng.normal()
    alpha[z0 + 1:] = rng.normal(size=z0) + 1j * rng.normal(size=z0)
    alpha[:z0] = np.conj(alpha[z0 + 1:][::-1])  # the canonical order is symmetric: -k at the mirrored index
    assert np.array_equal(K[:z0], -K[z0 + 1:][::-1])
    a = alpha.view(np.float64)
    used = np.where(idx >= 0, idx, 0)
    slots = [tuple(v) for v in (coef * a[used] * (idx >= 0)).sum(axis=2)]
    for _ in range(4):
        z = np.exp(2j * np.pi * rng.random(d))
        want = (alpha * np.prod(z[None, :] ** K, axis=1)).sum().real
        got = series_by_layout(slots, z, d, n, kind, levels)
        assert abs(got - want) < 1e-12 * (1 + np.abs(alpha).sum())

"""Pins on the paper's polyphase matrices, schemes and Table 1.

* Proposed Schemes: T_P = T_P^V T_P^H and S_U = S_U^V S_U^H (the non-separable
  lifting merges the separable steps), N_{P,U} = S_U T_P with V = PU + 1, and
  N_{P,U} equals the tensor square of the 1-D pair [[V, U], [P, 1]];
* Optimization Approach: T_{P0}^V T_{P0}^H T_{P1} = T_P (and for S_U);
* Table 1: steps and operation counts of the lifting schemes;
* Eq. 2 with the CDF 9/7 constants reproduces the closed-form filter bank;
* scheme equivalence ("they all compute the same values"): the separable,
  non-separable and reduced schemes, applied as printed to quads, agree with
  each other and with the oracle away from the image boundary.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import polyphase as pp

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(7)


def _rand_poly(rng, nterms=3, span=2):
    t = {}
    for _ in range(nterms):
        k = (int(rng.integers(-span, span + 1)), int(rng.integers(-span, span + 1)))
        t[k] = Fraction(int(rng.integers(-9, 10)), int(rng.integers(1, 7)))
    return pp.LPoly(t)


def _rand_hpoly(rng, nterms=3, span=2):
    return pp.LPoly.h({int(rng.integers(-span, span + 1)): Fraction(int(rng.integers(-9, 10)), int(rng.integers(1, 7)))
                       for _ in range(nterms)})


@pytest.mark.parametrize("seed", range(5))
def test_nonseparable_steps_are_products_of_separable_steps(seed):
    rng = np.random.default_rng(seed)
    P, U = _rand_hpoly(rng), _rand_hpoly(rng)
    assert pp.mat_eq(pp.T(P), pp.chain(pp.T_V(P), pp.T_H(P)))
    assert pp.mat_eq(pp.S(U), pp.chain(pp.S_V(U), pp.S_H(U)))
    # horizontal and vertical steps commute (Background: they may be interleaved)
    assert pp.mat_eq(pp.chain(pp.T_V(P), pp.T_H(P)), pp.chain(pp.T_H(P), pp.T_V(P)))


@pytest.mark.parametrize("seed", range(5))
def test_polyconvolution_identity(seed):
    rng = np.random.default_rng(100 + seed)
    P, U = _rand_hpoly(rng), _rand_hpoly(rng)
    N = pp.N_poly(P, U)
    assert pp.mat_eq(N, pp.chain(pp.S(U), pp.T(P)))
    # tensor square of the 1-D pair [[V, U], [P, 1]]: entry (2a+b, 2c+d) = A*[a][c] A[b][d]
    V = P * U + pp.ONE
    A = [[V, U], [P, pp.ONE]]
    for r in range(4):
        for c in range(4):
            a, b = divmod(r, 2)
            cc, d = divmod(c, 2)
            assert N[r][c] == A[a][cc].star() * A[b][d]


@pytest.mark.parametrize("seed", range(4))
def test_reduced_split_reproduces_the_step(seed):
    rng = np.random.default_rng(200 + seed)
    P = _rand_hpoly(rng, 4) + pp.LPoly.const(Fraction(3, 7))
    U = _rand_hpoly(rng, 4) + pp.LPoly.const(Fraction(-2, 5))
    P0, P1 = P.split0()
    U0, U1 = U.split0()
    assert P0 == pp.LPoly.const(P.t[(0, 0)]) and (0, 0) not in P1.t
    assert pp.mat_eq(pp.chain(pp.T_V(P0), pp.T_H(P0), pp.T(P1)), pp.T(P))
    assert pp.mat_eq(pp.chain(pp.S_V(U0), pp.S_H(U0), pp.S(U1)), pp.S(U))


def test_table1_lifting_rows():
    with open(os.path.join(GOLD, "table1_lifting.json")) as f:
        t1 = json.load(f)["lifting"]
    wav = {"cdf53": pp.pairs_cdf53(), "cdf97": pp.pairs_cdf97(exact=True), "dd137": pp.pairs_dd137()}
    for name, pairs in wav.items():
        for rule in ("terms", "distinct"):
            st, ops = pp.table1_row(pp.scheme_separable(pairs), rule)
            assert (st, ops) == (t1[name]["separable"]["steps"], t1[name]["separable"]["ops"]), (name, rule)
            st, ops = pp.table1_row(pp.scheme_nonsep_reduced(pairs), rule)
            assert (st, ops) == (t1[name]["nonseparable"]["steps"], t1[name]["nonseparable"]["ops"]), (name, rule)
    # without the split the non-separable lifting costs more (12 terms per step)
    assert pp.table1_row(pp.scheme_nonsep(pp.pairs_cdf97(exact=True)), "terms") == (4, 48)


def test_lifting_product_is_the_closed_form_filter_bank():
    """Eq. 2: the product of the lifting pairs (times the scaling) is the
    polyphase matrix of Eq. 1, i.e. the CDF 9/7 analysis filters."""
    from tests.test_oracle import L9, H7
    z = pp.CDF97_COEFS["zeta"]
    # 1-D 2x2 polyphase matrix over horizontal polynomials, components (even, odd)
    M = [[pp.ONE, pp.ZERO], [pp.ZERO, pp.ONE]]

    def mul(A, B):
        return [[A[i][0] * B[0][j] + A[i][1] * B[1][j] for j in range(2)] for i in range(2)]
    for P, U in pp.pairs_cdf97():
        M = mul([[pp.ONE, pp.ZERO], [P, pp.ONE]], M)   # predict: odd += P even
        M = mul([[pp.ONE, U], [pp.ZERO, pp.ONE]], M)   # update: even += U odd
    M = mul([[pp.LPoly.const(z), pp.ZERO], [pp.ZERO, pp.LPoly.const(1 / z)]], M)
    # low-pass output n: sum over even inputs 2(n+e) and odd inputs 2(n+e)+1
    low = np.zeros(9)
    for (e, _), v in M[0][0].t.items():
        low[2 * e + 4] += v
    for (e, _), v in M[0][1].t.items():
        low[2 * e + 1 + 4] += v
    high = np.zeros(7)  # centred on the odd sample 2n+1
    for (e, _), v in M[1][0].t.items():
        high[2 * e - 1 + 3] += v
    for (e, _), v in M[1][1].t.items():
        high[2 * e + 3] += v
    assert np.abs(low - L9).max() < 1e-8
    assert np.abs(high - H7).max() < 1e-8


def test_dd137_lifting_product_is_the_published_filter_bank():
    """The DD 13/7 pair multiplied out (Eq. 2, no scaling) is the published
    13-tap / 7-tap analysis bank."""
    from tests.test_oracle import L13, H7DD
    (P, U), = pp.pairs_dd137()
    # even output n: s = e + U(odd after predict); odd output: d = o + P e
    low = np.zeros(13)
    high = np.zeros(7)
    for (k, _), p in P.t.items():          # d[n] = x[2n+1] + sum_k p_k x[2(n+k)]
        high[2 * k - 1 + 3] += float(p)
    high[3] += 1.0
    low[6] += 1.0                            # s[n] = x[2n] + sum_j u_j d[n+j]
    for (j, _), u in U.t.items():
        low[2 * j + 1 + 6] += float(u)
        for (k, _), p in P.t.items():
            low[2 * (j + k) + 6] += float(u * p)
    assert np.array_equal(low, L13)
    assert np.array_equal(high, H7DD)


def test_dd137_schemes_compute_the_same_values_as_the_oracle():
    hq, wq = 16, 20
    x = RNG.uniform(0, 255, size=(2 * hq, 2 * wq))
    pairs = pp.pairs_dd137()
    q = pp.to_quads(x)
    outs = [pp.apply_steps(s(pairs), q) for s in (pp.scheme_separable, pp.scheme_nonsep)]
    assert np.abs(outs[0] - outs[1]).max() < 1e-10
    ref = oracle.forward137(x, 1)
    bands = np.stack([ref[:hq, :wq], ref[:hq, wq:], ref[hq:, :wq], ref[hq:, wq:]])
    m = 4  # the periodic and the symmetric extension differ only near the edges
    assert np.abs(outs[1][:, m:-m, m:-m] - bands[:, m:-m, m:-m]).max() < 1e-9


@pytest.mark.parametrize("hq,wq", [(16, 16), (12, 20)])
def test_schemes_compute_the_same_values_as_the_oracle(hq, wq):
    h, w = 2 * hq, 2 * wq
    x = RNG.uniform(0, 255, size=(h, w))
    pairs = pp.pairs_cdf97()
    q = pp.to_quads(x)
    outs = [pp.apply_steps(s(pairs), q) for s in (pp.scheme_separable, pp.scheme_nonsep, pp.scheme_nonsep_reduced)]
    assert np.abs(outs[0] - outs[1]).max() < 1e-10
    assert np.abs(outs[0] - outs[2]).max() < 1e-10
    z = pp.CDF97_COEFS["zeta"]
    scale = np.array([z * z, 1.0, 1.0, 1.0 / (z * z)])[:, None, None]
    y = outs[1] * scale
    ref = oracle.forward97(x, 1)
    bands = np.stack([ref[:hq, :wq], ref[:hq, wq:], ref[hq:, :wq], ref[hq:, wq:]])
    m = 3  # the periodic and the symmetric extension differ only near the edges
    assert np.abs(bands[:, m:-m, m:-m] - y[:, m:-m, m:-m]).max() < 1e-9

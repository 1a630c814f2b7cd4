"""The paper's 4x4 polyphase matrices over bivariate Laurent polynomials.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Barina et al., arXiv:1704.08657:
  * a filter (g_k) has transfer function G(z) = sum_k g_k z^-k; in 2-D the
    variable z_m is the horizontal axis and z_n the vertical one, and
    G*(z_m, z_n) = G(z_n, z_m) is the transposed polynomial (Background);
  * the separable lifting steps T_P^H, T_P^V, S_U^H, S_U^V (Background);
  * the non-separable convolution N = N^V N^H, the polyconvolution N_{P,U}
    with V = PU + 1, and the spatial predict / update T_P, S_U of the
    non-separable lifting (Proposed Schemes);
  * the split P = P0 + P1, U = U0 + U1 into constant and remaining terms and
    the resulting step sequence (Optimization Approach);
  * the operation count rule: the number of terms of all polynomials in all
    matrices, units on the diagonal excluded (Background), and the per-scheme
    steps and operations of Table 1.

Polynomials are dicts {(e_m, e_n): coefficient} of the monomial z_m^e_m z_n^e_n.
Quads are arrays q[k, i, j], k = 0..3 for the components (c1, c2, c3, c4) of
quad row i, quad column j.  Applying z_m^a z_n^b to a component reads the
component at (i + b, j + a), since z^-k delays by k samples.
"""
from __future__ import annotations

from fractions import Fraction
from typing import Dict, List, Sequence, Tuple

import numpy as np

Mono = Tuple[int, int]


class LPoly:
    """Bivariate Laurent polynomial with exact or float coefficients."""

    __slots__ = ("t",)

    def __init__(self, terms: Dict[Mono, object] | None = None):
        self.t: Dict[Mono, object] = {}
        for k, v in (terms or {}).items():
            if v != 0:
                self.t[k] = v

    @staticmethod
    def const(c) -> "LPoly":
        return LPoly({(0, 0): c})

    @staticmethod
    def h(taps: Dict[int, object]) -> "LPoly":
        """Horizontal 1-D polynomial sum_e c_e z_m^e."""
        return LPoly({(e, 0): c for e, c in taps.items()})

    def __add__(self, o: "LPoly") -> "LPoly":
        r = dict(self.t)
        for k, v in o.t.items():
            r[k] = r.get(k, 0) + v
        return LPoly(r)

    def __neg__(self) -> "LPoly":
        return LPoly({k: -v for k, v in self.t.items()})

    def __sub__(self, o: "LPoly") -> "LPoly":
        return self + (-o)

    def __mul__(self, o) -> "LPoly":
        if not isinstance(o, LPoly):
            return LPoly({k: v * o for k, v in self.t.items()})
        r: Dict[Mono, object] = {}
        for (a, b), v in self.t.items():
            for (c, d), w in o.t.items():
                k = (a + c, b + d)
                r[k] = r.get(k, 0) + v * w
        return LPoly(r)

    __rmul__ = __mul__

    def star(self) -> "LPoly":
        """G*(z_m, z_n) = G(z_n, z_m)."""
        return LPoly({(b, a): v for (a, b), v in self.t.items()})

    def split0(self) -> Tuple["LPoly", "LPoly"]:
        """(P0, P1): the constant term and the remaining terms."""
        p0 = LPoly({k: v for k, v in self.t.items() if k == (0, 0)})
        p1 = LPoly({k: v for k, v in self.t.items() if k != (0, 0)})
        return p0, p1

    def nterms(self) -> int:
        return len(self.t)

    def is_zero(self) -> bool:
        return not self.t

    def is_one(self) -> bool:
        return self.t == {(0, 0): 1}

    def __eq__(self, o) -> bool:  # exact comparison
        return isinstance(o, LPoly) and (self - o).is_zero()

    def close(self, o: "LPoly", tol: float = 1e-12) -> bool:
        d = self - o
        return all(abs(float(v)) <= tol for v in d.t.values())

    def __repr__(self) -> str:
        return "LPoly(" + ", ".join(f"{v}*zm^{a}zn^{b}" for (a, b), v in sorted(self.t.items())) + ")"


ZERO = LPoly()
ONE = LPoly.const(1)
Mat = List[List[LPoly]]


def eye() -> Mat:
    return [[ONE if i == j else ZERO for j in range(4)] for i in range(4)]


def matmul(A: Mat, B: Mat) -> Mat:
    n = len(A)
    return [[sum((A[i][k] * B[k][j] for k in range(n)), ZERO) for j in range(n)] for i in range(n)]


def chain(*ms: Mat) -> Mat:
    """Product M1 M2 ... Mk (the rightmost acts first on column vectors)."""
    r = eye()
    for m in ms:
        r = matmul(r, m)
    return r


def mat_eq(A: Mat, B: Mat) -> bool:
    return all(A[i][j] == B[i][j] for i in range(4) for j in range(4))


# ---- the separable lifting steps (Background) ------------------------------

def T_H(P: LPoly) -> Mat:
    M = eye()
    M[1][0] = P
    M[3][2] = P
    return M


def T_V(P: LPoly) -> Mat:
    M = eye()
    M[2][0] = P.star()
    M[3][1] = P.star()
    return M


def S_H(U: LPoly) -> Mat:
    M = eye()
    M[0][1] = U
    M[2][3] = U
    return M


def S_V(U: LPoly) -> Mat:
    M = eye()
    M[0][2] = U.star()
    M[1][3] = U.star()
    return M


# ---- the non-separable schemes (Proposed Schemes) --------------------------

def T(P: LPoly) -> Mat:
    """Spatial predict T_P."""
    Ps = P.star()
    return [[ONE, ZERO, ZERO, ZERO],
            [P, ONE, ZERO, ZERO],
            [Ps, ZERO, ONE, ZERO],
            [P * Ps, Ps, P, ONE]]


def S(U: LPoly) -> Mat:
    """Spatial update S_U."""
    Us = U.star()
    return [[ONE, U, Us, U * Us],
            [ZERO, ONE, ZERO, Us],
            [ZERO, ZERO, ONE, U],
            [ZERO, ZERO, ZERO, ONE]]


def N_poly(P: LPoly, U: LPoly) -> Mat:
    """Non-separable polyconvolution N_{P,U} with V = PU + 1."""
    V = P * U + ONE
    Vs, Us, Ps = V.star(), U.star(), P.star()
    return [[Vs * V, Vs * U, Us * V, Us * U],
            [Vs * P, Vs, Us * P, Us],
            [Ps * V, Ps * U, V, U],
            [Ps * P, Ps, P, ONE]]


# ---- wavelets as lifting pairs ---------------------------------------------
# Alignment reading: predict reads the even samples n and n+1 (P = a(1 + z)),
# update reads the odd samples n-1 and n (U = b(1 + z^-1)).

CDF97_COEFS = dict(alpha=-1.586134342, beta=-0.052980119, gamma=0.882911076,
                   delta=0.443506852, zeta=1.149604398)


def pairs_cdf97(exact: bool = False) -> List[Tuple[LPoly, LPoly]]:
    c = CDF97_COEFS
    f = (lambda v: Fraction(str(v))) if exact else float
    return [(LPoly.h({0: f(c["alpha"]), 1: f(c["alpha"])}), LPoly.h({0: f(c["beta"]), -1: f(c["beta"])})),
            (LPoly.h({0: f(c["gamma"]), 1: f(c["gamma"])}), LPoly.h({0: f(c["delta"]), -1: f(c["delta"])}))]


def pairs_cdf53() -> List[Tuple[LPoly, LPoly]]:
    h = Fraction(1, 2)
    q = Fraction(1, 4)
    return [(LPoly.h({0: -h, 1: -h}), LPoly.h({0: q, -1: q}))]


def pairs_dd137() -> List[Tuple[LPoly, LPoly]]:
    """Deslauriers-Dubuc 13/7: four-tap predict (odd += P even, the negated
    cubic interpolation -(9/16)(1 + z) + (1/16)(z^-1 + z^2)) and four-tap
    update (even += U odd, (9/32)(1 + z^-1) - (1/32)(z + z^-2)).  The paper
    prints no coefficients (Table 1 only counts its terms); these are the
    published filter bank's, as in dwt2ref.c."""
    pn, pf = Fraction(-9, 16), Fraction(1, 16)
    un, uf = Fraction(9, 32), Fraction(-1, 32)
    return [(LPoly.h({-1: pf, 0: pn, 1: pn, 2: pf}), LPoly.h({-2: uf, -1: un, 0: un, 1: uf}))]


# ---- schemes as step sequences (lists of barrier-separated steps) -----------
# Each step is a list of matrices applied without a barrier between them
# (rightmost first).  The full scheme is the product of the steps in order.

def scheme_separable(pairs) -> List[List[Mat]]:
    steps = []
    for P, U in pairs:
        steps += [[T_H(P)], [T_V(P)], [S_H(U)], [S_V(U)]]
    return steps


def scheme_nonsep(pairs) -> List[List[Mat]]:
    steps = []
    for P, U in pairs:
        steps += [[T(P)], [S(U)]]
    return steps


def scheme_nonsep_reduced(pairs) -> List[List[Mat]]:
    """Optimization Approach: per step, the non-separable part with P1 (or U1)
    reads pre-step neighbours, then the constant parts P0 (U0) follow as
    separable lifting inside the unit, without a barrier."""
    steps = []
    for P, U in pairs:
        P0, P1 = P.split0()
        U0, U1 = U.split0()
        steps.append([T_V(P0), T_H(P0), T(P1)])  # T(P1) first, then T^H, T^V
        steps.append([S_V(U0), S_H(U0), S(U1)])
    return steps


def scheme_matrix(steps: List[List[Mat]]) -> Mat:
    """The whole scheme as one matrix: later steps multiply on the left."""
    r = eye()
    for st in steps:
        r = matmul(chain(*st), r)
    return r


# ---- Table 1 counting rule --------------------------------------------------

def count_ops(mats: Sequence[Mat], rule: str = "terms") -> int:
    """Operations of a list of matrices (Background, counting rule).

    rule='terms': number of terms of every polynomial entry, the units on the
    diagonal excluded.  rule='distinct': per column, the number of distinct
    (monomial, coefficient) terms over that column's off-diagonal entries.
    """
    n = 0
    for M in mats:
        for j in range(4):
            seen = set()
            for i in range(4):
                p = M[i][j]
                if i == j and p.is_one():
                    continue
                if rule == "terms":
                    n += p.nterms()
                else:
                    seen.update((k, v) for k, v in p.t.items())
            if rule == "distinct":
                n += len(seen)
    return n


def table1_row(steps: List[List[Mat]], rule: str = "terms") -> Tuple[int, int]:
    """(number of steps, number of operations) of a scheme."""
    return len(steps), count_ops([m for st in steps for m in st], rule)


# ---- applying matrices to quads (periodic extension) ------------------------

def apply_poly(p: LPoly, x: np.ndarray) -> np.ndarray:
    """p applied to one component array x[i, j] with periodic extension."""
    out = np.zeros_like(x, dtype=np.float64)
    for (a, b), v in p.t.items():
        out += float(v) * np.roll(np.roll(x, -b, axis=0), -a, axis=1)
    return out


def apply_mat(M: Mat, q: np.ndarray) -> np.ndarray:
    """y = M q for quads q[4, Hq, Wq]; every entry reads pre-step values."""
    y = np.zeros_like(q, dtype=np.float64)
    for i in range(4):
        for j in range(4):
            if not M[i][j].is_zero():
                y[i] += apply_poly(M[i][j], q[j])
    return y


def apply_steps(steps: List[List[Mat]], q: np.ndarray) -> np.ndarray:
    for st in steps:
        for M in reversed(st):  # rightmost first
            q = apply_mat(M, q)
    return q


def to_quads(x: np.ndarray) -> np.ndarray:
    """Image (even sides) -> quads (c1, c2, c3, c4)."""
    return np.stack([x[0::2, 0::2], x[0::2, 1::2], x[1::2, 0::2], x[1::2, 1::2]]).astype(np.float64)


def from_quads(q: np.ndarray) -> np.ndarray:
    h, w = q.shape[1] * 2, q.shape[2] * 2
    x = np.empty((h, w), dtype=np.float64)
    x[0::2, 0::2], x[0::2, 1::2], x[1::2, 0::2], x[1::2, 1::2] = q
    return x

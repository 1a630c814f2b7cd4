"""Pins for the oracle: checks against things other than the oracle itself.

* closed-form CDF 9/7 filter bank (built from the roots of the Daubechies
  polynomial 20y^3 + 10y^2 + 4y + 1, y = (2 - z - 1/z)/4), applied as a direct
  convolution with whole-sample symmetric extension;
* the dense 64x64 operator on 8x8 inputs vs the Kronecker square of the 1-D
  closed-form filter-bank matrix;
* perfect reconstruction, vanishing moments (constant and ramp images);
* adjoint: dot test and transpose of the dense operator;
* integer 5/3: hand-worked examples, exact reconstruction, exact zero details
  on constants and integer ramps, closeness to the linear 5/3 filter bank.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


# ---------------------------------------------------------------- closed form

def _closed_form_97():
    """(L9, H7): analysis low-pass (9 taps, centre index 4) and high-pass
    (7 taps, centre index 3) of CDF 9/7, normalised to DC / Nyquist gain sqrt 2."""
    roots = np.roots([20.0, 10.0, 4.0, 1.0])
    real = [r.real for r in roots if abs(r.imag) < 1e-12][0]
    cplx = [r for r in roots if r.imag > 1e-12][0]

    def lin(root):  # 1 - y/root as taps on z^-1, z^0, z^1
        c = 1.0 / (4.0 * root)
        return np.array([c, 1.0 - 2.0 * c, c])

    one_minus_y = np.array([0.25, 0.5, 0.25])
    base = np.convolve(one_minus_y, one_minus_y)
    l9 = np.convolve(base, np.convolve(lin(cplx), lin(np.conj(cplx)))).real
    l7 = np.convolve(base, lin(real)).real
    l9 *= np.sqrt(2) / l9.sum()
    l7 *= np.sqrt(2) / l7.sum()
    h7 = l7 * np.array([(-1) ** k for k in range(-3, 4)])
    return l9, h7


L9, H7 = _closed_form_97()


def _fold(k, n):
    """Whole-sample symmetric extension index (repeated reflection)."""
    if n == 1:
        return 0
    p = 2 * (n - 1)
    k %= p
    return k if k < n else p - k


def _conv_matrix_1d(n, lo=L9, hi=H7):
    """n x n analysis matrix: rows 0..ceil(n/2)-1 low-pass, then high-pass
    (odd-length symmetric filters, centred on the even / odd sample)."""
    nl = (n + 1) // 2
    cl, ch = len(lo) // 2, len(hi) // 2
    A = np.zeros((n, n))
    for i in range(nl):
        for k in range(-cl, cl + 1):
            A[i, _fold(2 * i + k, n)] += lo[k + cl]
    for i in range(n // 2):
        for k in range(-ch, ch + 1):
            A[nl + i, _fold(2 * i + 1 + k, n)] += hi[k + ch]
    return A


def _conv_dwt2(x, levels, lo=L9, hi=H7):
    """Direct-convolution 2-D pyramid (rows, then columns), Mallat layout."""
    y = np.array(x, dtype=np.float64)
    h, w = y.shape
    for _ in range(levels):
        Ah, Av = _conv_matrix_1d(w, lo, hi), _conv_matrix_1d(h, lo, hi)
        y[:h, :w] = Av @ y[:h, :w] @ Ah.T
        h, w = (h + 1) // 2, (w + 1) // 2
    return y


def _dense(fn, h, w):
    n = h * w
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        M[:, k] = fn(e.reshape(h, w)).ravel()
    return M


# ------------------------------------------------------------------ CDF 9/7

def test_closed_form_taps_sane():
    # symmetric, unit-gain sqrt 2, 4 vanishing moments of the high-pass
    assert np.allclose(L9, L9[::-1]) and np.allclose(H7, H7[::-1])
    assert abs(L9.sum() - np.sqrt(2)) < 1e-14
    k = np.arange(-3, 4)
    for p in range(4):
        assert abs((H7 * k ** p).sum()) < 1e-12


@pytest.mark.parametrize("h,w", [(16, 16), (17, 23), (8, 9), (2, 2), (3, 5), (2, 7), (5, 2), (33, 64)])
def test_forward97_equals_closed_form_convolution(h, w):
    x = RNG.uniform(0, 255, size=(h, w))
    ref = _conv_dwt2(x, 1)
    got = oracle.forward97(x, 1)
    assert np.abs(got - ref).max() <= 1e-7 * np.abs(x).max()


@pytest.mark.parametrize("h,w,levels", [(64, 64, 5), (40, 27, 3), (9, 13, 2), (8, 8, 3)])
def test_forward97_pyramid_equals_closed_form(h, w, levels):
    x = RNG.uniform(0, 255, size=(h, w))
    ref = _conv_dwt2(x, levels)
    got = oracle.forward97(x, levels)
    # level-k low-pass grows by 2 per level; constants carry ~1e-9 error
    assert np.abs(got - ref).max() <= 1e-7 * np.abs(x).max() * 2 ** levels


@pytest.mark.parametrize("h,w", [(8, 8), (7, 9)])
def test_dense_operator_is_kron_of_1d_filter_banks(h, w):
    M = _dense(lambda e: oracle.forward97(e, 1), h, w)
    Ah, Av = _conv_matrix_1d(w), _conv_matrix_1d(h)
    # row-major vec: vec(Av X Ah^T) = kron(Av, Ah) vec(X)
    K = np.kron(Av, Ah)
    assert np.abs(M - K).max() < 1e-8


def test_dense_three_levels_on_8x8():
    M = _dense(lambda e: oracle.forward97(e, 3), 8, 8)
    R = _dense(lambda e: _conv_dwt2(e, 3), 8, 8)
    assert np.abs(M - R).max() < 1e-7


@pytest.mark.parametrize("h,w,levels", [(32, 32, 1), (45, 38, 4), (2, 3, 1), (128, 96, 5)])
def test_perfect_reconstruction97(h, w, levels):
    x = RNG.uniform(-100, 300, size=(h, w))
    y = oracle.inverse97(oracle.forward97(x, levels), levels)
    assert np.abs(y - x).max() <= 1e-10 * np.abs(x).max()


def test_constant_image_has_no_detail():
    for (h, w, lv) in [(32, 32, 4), (13, 21, 3)]:
        c = 117.0
        y = oracle.forward97(np.full((h, w), c), lv)
        for lev, name, rs, cs in oracle.band_slices(h, w, lv):
            band = y[rs, cs]
            if name == "LL":
                assert np.allclose(band, c * 2 ** lev, rtol=1e-7)
            else:  # the 9-10 digit constants leave ~1e-9 relative residue
                assert np.abs(band).max() <= 1e-7 * c


def test_linear_ramp_interior_detail_vanishes():
    h, w = 40, 48
    i, j = np.mgrid[0:h, 0:w]
    x = 3.0 * i - 2.0 * j + 50.0
    y = oracle.forward97(x, 1)
    m = 4  # coefficients within m of an edge see the mirror kink
    for lev, name, rs, cs in oracle.band_slices(h, w, 1):
        if name == "LL":
            continue
        band = y[rs, cs]
        inner = band[m:band.shape[0] - m, m:band.shape[1] - m] if name == "HH" else None
        if name == "HL":
            inner = band[:, m:band.shape[1] - m]
        if name == "LH":
            inner = band[m:band.shape[0] - m, :]
        assert np.abs(inner).max() <= 1e-7 * np.abs(x).max()


@pytest.mark.parametrize("h,w,levels", [(16, 16, 2), (7, 9, 1), (33, 20, 3)])
def test_adjoint_dot(h, w, levels):
    x = RNG.standard_normal((h, w))
    g = RNG.standard_normal((h, w))
    lhs = float((oracle.forward97(x, levels) * g).sum())
    rhs = float((x * oracle.adjoint97(g, levels)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("h,w,levels", [(8, 8, 1), (7, 9, 1), (8, 8, 3), (6, 5, 2)])
def test_adjoint_is_dense_transpose(h, w, levels):
    M = _dense(lambda e: oracle.forward97(e, levels), h, w)
    MT = _dense(lambda e: oracle.adjoint97(e, levels), h, w)
    assert np.abs(MT - M.T).max() < 1e-13
    # and it is not the inverse (the 9/7 bank is biorthogonal)
    Mi = _dense(lambda e: oracle.inverse97(e, levels), h, w)
    assert np.abs(MT - Mi).max() > 1e-3


def test_levels_too_deep_rejected():
    with pytest.raises(ValueError):
        oracle.forward97(np.zeros((4, 4)), 3)  # 4 -> 2 -> 1: third level has side 1
    oracle.forward97(np.zeros((4, 4)), 2)


# ------------------------------------------------------------ integer 5/3

def test_int53_hand_worked_examples():
    with open(os.path.join(GOLD, "int53_hand.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        got = oracle.forward53i(np.array(case["x"], dtype=np.int64), case["levels"])
        assert got.tolist() == case["mallat"], case["name"]


@pytest.mark.parametrize("h,w,levels", [(32, 32, 3), (17, 30, 2), (2, 2, 1), (3, 2, 1), (128, 77, 5)])
def test_int53_exact_reconstruction(h, w, levels):
    x = RNG.integers(-300, 300, size=(h, w)).astype(np.int64)
    y = oracle.forward53i(x, levels)
    assert np.array_equal(oracle.inverse53i(y, levels), x)


def test_int53_constant_and_integer_ramp():
    h, w = 24, 30
    y = oracle.forward53i(np.full((h, w), 77, dtype=np.int64), 3)
    for lev, name, rs, cs in oracle.band_slices(h, w, 3):
        band = y[rs, cs]
        assert np.all(band == (77 if name == "LL" else 0))
    i, j = np.mgrid[0:h, 0:w]
    x = (4 * i + 6 * j + 10).astype(np.int64)  # integer slopes
    y = oracle.forward53i(x, 1)
    for lev, name, rs, cs in oracle.band_slices(h, w, 1):
        if name == "LL":
            continue
        band = y[rs, cs]
        m = 2
        if name == "HL":
            assert np.all(band[:, m:band.shape[1] - m] == 0)
        elif name == "LH":
            assert np.all(band[m:band.shape[0] - m, :] == 0)
        else:
            assert np.all(band[m:-m, m:-m] == 0)


def _linear53_matrix(n):
    """Linear (unrounded) 5/3 analysis matrix: low (-1,2,6,2,-1)/8, high (-1,2,-1)/2."""
    lo = np.array([-1, 2, 6, 2, -1]) / 8.0
    hi = np.array([-1, 2, -1]) / 2.0
    nl = (n + 1) // 2
    A = np.zeros((n, n))
    for i in range(nl):
        for k in range(-2, 3):
            A[i, _fold(2 * i + k, n)] += lo[k + 2]
    for i in range(n // 2):
        for k in range(-1, 2):
            A[nl + i, _fold(2 * i + 1 + k, n)] += hi[k + 1]
    return A


@pytest.mark.parametrize("h,w", [(32, 32), (19, 26), (2, 5)])
def test_int53_close_to_linear_filter_bank(h, w):
    x = RNG.integers(0, 256, size=(h, w)).astype(np.int64)
    y = oracle.forward53i(x, 1).astype(np.float64)
    ref = _linear53_matrix(h) @ x @ _linear53_matrix(w).T
    d = y - ref
    # rounding: each predict adds [0, 1/2], each update (-1/2, 3/4]; two axes
    assert np.abs(d).max() <= 2.5
    assert abs(d.mean()) < 0.5


def test_oracle_adjoint_is_the_gradient_fp64():
    """gradcheck (FP64, 32x32, three levels): the oracle's adjoint is the
    Jacobian transpose of its forward transform."""
    import torch

    class F(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x):
            return torch.from_numpy(oracle.forward97(x.detach().numpy(), 3))

        @staticmethod
        def backward(ctx, g):
            return torch.from_numpy(oracle.adjoint97(g.detach().numpy(), 3))

    x = torch.from_numpy(RNG.standard_normal((32, 32))).requires_grad_(True)
    assert torch.autograd.gradcheck(F.apply, (x,), eps=1e-6, atol=1e-8, rtol=1e-6, fast_mode=True)


# ------------------------------------------------------------------ DD 13/7
# The interpolating Deslauriers-Dubuc 13/7 filter bank as published (13-tap
# analysis low-pass / 512 and 7-tap high-pass / 16): an independent statement
# of what the oracle's two 4-tap lifting steps must multiply out to.
L13 = np.array([-1, 0, 18, -16, -63, 144, 348, 144, -63, -16, 18, 0, -1], dtype=np.float64) / 512.0
H7DD = np.array([1, 0, -9, 16, -9, 0, 1], dtype=np.float64) / 16.0


def test_dd137_closed_form_taps_sane():
    # symmetric, low-pass DC gain 1, high-pass kills cubics (4 vanishing moments)
    assert np.array_equal(L13, L13[::-1]) and np.array_equal(H7DD, H7DD[::-1])
    assert L13.sum() == 1.0
    k = np.arange(-3, 4)
    for p in range(4):
        assert (H7DD * k ** p).sum() == 0.0


@pytest.mark.parametrize("h,w", [(16, 16), (17, 23), (8, 9), (2, 2), (3, 5), (2, 7), (5, 2), (33, 64), (4, 6)])
def test_forward137_equals_closed_form_convolution(h, w):
    x = RNG.uniform(0, 255, size=(h, w))
    ref = _conv_dwt2(x, 1, L13, H7DD)
    got = oracle.forward137(x, 1)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(x).max()


@pytest.mark.parametrize("h,w,levels", [(64, 64, 5), (40, 27, 3), (9, 13, 2), (8, 8, 3)])
def test_forward137_pyramid_equals_closed_form(h, w, levels):
    x = RNG.uniform(0, 255, size=(h, w))
    ref = _conv_dwt2(x, levels, L13, H7DD)
    assert np.abs(oracle.forward137(x, levels) - ref).max() <= 1e-11 * np.abs(x).max()


def test_dd137_dense_operator_is_kron_of_1d_filter_banks():
    for (h, w) in [(8, 8), (7, 9)]:
        M = _dense(lambda e: oracle.forward137(e, 1), h, w)
        K = np.kron(_conv_matrix_1d(h, L13, H7DD), _conv_matrix_1d(w, L13, H7DD))
        assert np.abs(M - K).max() < 1e-13


@pytest.mark.parametrize("h,w,levels", [(32, 32, 1), (45, 38, 4), (2, 3, 1), (128, 96, 5)])
def test_perfect_reconstruction137(h, w, levels):
    x = RNG.uniform(-100, 300, size=(h, w))
    y = oracle.inverse137(oracle.forward137(x, levels), levels)
    assert np.abs(y - x).max() <= 1e-11 * np.abs(x).max()


def test_dd137_constant_and_cubic():
    # a constant keeps every detail exactly 0 and the low-low value (DC gain 1)
    y = oracle.forward137(np.full((21, 30), 117.0), 3)
    for lev, name, rs, cs in oracle.band_slices(21, 30, 3):
        assert np.all(y[rs, cs] == (117.0 if name == "LL" else 0.0))
    # a cubic along the rows has no horizontal detail away from the mirror kinks
    h, w = 24, 64
    j = np.arange(w, dtype=np.float64)
    x = np.tile(0.002 * j ** 3 - 0.1 * j ** 2 + 3.0 * j + 7.0, (h, 1))
    y = oracle.forward137(x, 1)
    hl = y[:(h + 1) // 2, (w + 1) // 2:]
    m = 3
    assert np.abs(hl[:, m:hl.shape[1] - m]).max() <= 1e-12 * np.abs(x).max()

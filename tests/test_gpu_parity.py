"""GPU kernels vs the oracle, element by element, through the C ABI.

Sizes span several strips (120 pixels) and segments plus ragged tails, odd
sides and the smallest legal images; every output buffer carries a guard band
(padding columns and rows) that must stay untouched.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1704_08657_gb300 import synth
from paper_1704_08657_gb300.dwt import Plan, round_up
from tests.util import assert_dd_close, assert_fp32_close, assert_lowp_close

pytestmark = pytest.mark.gpu

SENT = -12345.0
SCHEMES97 = ["nonsep", "reduced", "sep", "polyconv", "conv", "nsconv"]


def _levels_max(h, w, cap):
    lv = 0
    while lv < cap and h >= 2 and w >= 2:
        lv += 1
        h, w = (h + 1) // 2, (w + 1) // 2
    return lv


def _padded(x: np.ndarray, dtype, guard_rows=3):
    """Device buffer with pitch rounded to 4 and guard rows, filled with SENT."""
    h, w = x.shape
    pitch = round_up(w + 1, 4)  # at least one padding column
    buf = torch.full((h + guard_rows, pitch), SENT, dtype=dtype, device="cuda")
    buf[:h, :w] = torch.from_numpy(np.ascontiguousarray(x)).to(dtype)
    return buf, pitch


def _guard_ok(buf: torch.Tensor, h, w):
    b = buf.float().cpu().numpy()
    sent = float(torch.tensor(SENT, dtype=buf.dtype))  # the sentinel as stored in this dtype
    return bool(np.all(b[:h, w:] == sent) and np.all(b[h:, :] == sent))


def gpu_forward(x, levels, scheme="nonsep", coef_dtype=torch.float32, wavelet="cdf97"):
    h, w = x.shape
    in_dt = torch.int32 if wavelet == "cdf53" else torch.float32
    xin, pitch = _padded(x, in_dt)
    out = torch.full_like(xin, SENT, dtype=coef_dtype)
    plan = Plan.single(h, w, levels, pitch=pitch, wavelet=wavelet, scheme=scheme, coef_dtype=coef_dtype)
    plan.forward(xin, out)
    assert plan.status() == 0
    torch.cuda.synchronize()
    assert _guard_ok(out, h, w), "forward wrote outside the coefficient region"
    return out[:h, :w].float().cpu().numpy() if coef_dtype != torch.int32 else out[:h, :w].cpu().numpy()


def gpu_inverse(c, levels, scheme="nonsep", coef_dtype=torch.float32, wavelet="cdf97"):
    h, w = c.shape
    out_dt = torch.int32 if wavelet == "cdf53" else torch.float32
    cin, pitch = _padded(c, coef_dtype)
    out = torch.full_like(cin, SENT, dtype=out_dt)
    plan = Plan.single(h, w, levels, pitch=pitch, wavelet=wavelet, scheme=scheme, coef_dtype=coef_dtype)
    plan.inverse(cin, out)
    assert plan.status() == 0
    torch.cuda.synchronize()
    assert _guard_ok(out, h, w), "inverse wrote outside the image"
    return out[:h, :w].cpu().numpy()


def gpu_adjoint(g, levels):
    h, w = g.shape
    gin, pitch = _padded(g, torch.float32)
    out = torch.full_like(gin, SENT)
    plan = Plan.single(h, w, levels, pitch=pitch)
    plan.adjoint(gin, out)
    assert plan.status() == 0
    torch.cuda.synchronize()
    assert _guard_ok(out, h, w), "adjoint wrote outside the image"
    return out[:h, :w].cpu().numpy()


SHAPES = [(512, 512), (33, 65), (7, 5), (2, 2), (3, 3), (2, 9), (9, 2), (130, 250), (257, 129),
          (64, 1000), (1000, 64), (121, 241), (244, 124)]


@pytest.mark.parametrize("scheme", SCHEMES97)
@pytest.mark.parametrize("h,w", SHAPES)
def test_forward97_fp32(h, w, scheme):
    x = synth.uniform(h, w, seed=1 + h * 7 + w)
    for levels in sorted({1, _levels_max(h, w, 5)}):
        if levels == 0:
            continue
        ref = oracle.forward97(x.astype(np.float64), levels)
        got = gpu_forward(x, levels, scheme)
        assert_fp32_close(got, ref, levels, 255.0, f"{scheme} {h}x{w} L{levels}")


# (100, 1028) and (66, 3000): widths a multiple of 4, whose first and last
# strips of each row stream through the staged row loop with mirrored columns
@pytest.mark.parametrize("scheme", SCHEMES97)
@pytest.mark.parametrize("h,w", [(512, 512), (33, 65), (7, 5), (2, 2), (130, 250), (257, 129), (100, 1028),
                                 (66, 3000)])
def test_inverse97_fp32(h, w, scheme):
    levels = _levels_max(h, w, 4)
    x = synth.uniform(h, w, seed=11)
    c = oracle.forward97(x.astype(np.float64), levels)
    got = gpu_inverse(c.astype(np.float32), levels, scheme)
    ref = oracle.inverse97(c.astype(np.float32).astype(np.float64), levels)
    assert np.abs(got - ref).max() <= 1e-3 * 255.0 / 255.0 * 2, f"max err {np.abs(got - ref).max()}"
    # and forward then inverse on the GPU reconstructs the image
    rec = gpu_inverse(gpu_forward(x, levels, scheme), levels, scheme)
    assert np.abs(rec - x).max() <= 2e-3


@pytest.mark.parametrize("scheme", ["nonsep", "sep"])
@pytest.mark.parametrize("h,w", [(512, 512), (33, 65), (7, 5), (2, 2), (3, 2), (130, 250), (257, 129), (64, 1000)])
def test_int53_bit_exact(h, w, scheme):
    levels = _levels_max(h, w, 5)
    x = synth.to_int(synth.gradient(h, w, seed=2)) - 128
    ref = oracle.forward53i(x.astype(np.int64), levels)
    got = gpu_forward(x, levels, scheme, torch.int32, "cdf53")
    assert np.array_equal(got.astype(np.int64), ref), f"{int((got != ref).sum())} coefficients differ"
    back = gpu_inverse(ref.astype(np.int32), levels, scheme, torch.int32, "cdf53")
    assert np.array_equal(back.astype(np.int64), x.astype(np.int64))


@pytest.mark.parametrize("dtype,rel", [(torch.float16, 1e-3), (torch.bfloat16, 8e-3)])
@pytest.mark.parametrize("h,w", [(512, 512), (130, 250), (96, 1028)])
def test_lowp_storage(h, w, dtype, rel):
    levels = _levels_max(h, w, 5)
    x = synth.noisy(h, w, seed=3)
    ref = oracle.forward97(x.astype(np.float64), levels)
    for scheme in SCHEMES97:
        got = gpu_forward(x, levels, scheme, dtype)
        assert_lowp_close(got, ref, levels, rel, f"{dtype} {scheme}")
    # the inverse reads the low-precision coefficients
    c = ref.astype(np.float32)
    got = gpu_inverse(torch.from_numpy(c).to(dtype).float().numpy(), levels, "nonsep", dtype)
    ref_i = oracle.inverse97(torch.from_numpy(c).to(dtype).double().numpy(), levels)
    assert np.abs(got - ref_i).max() <= 2e-3 * np.abs(ref_i).max() / 255.0 * 2


@pytest.mark.parametrize("h,w", [(512, 512), (33, 65), (7, 5), (2, 2), (3, 3), (130, 250), (257, 129), (100, 1028),
                                 (70, 1000)])
def test_adjoint_matches_oracle(h, w):
    levels = _levels_max(h, w, 4)
    rng = np.random.default_rng(h * 1000 + w)
    g = rng.standard_normal((h, w)).astype(np.float32)
    ref = oracle.adjoint97(g.astype(np.float64), levels)
    got = gpu_adjoint(g, levels)
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max()) * 2 ** levels


@pytest.mark.parametrize("env", [{"DWT2_EDGE_SPLIT": "1"}, {"DWT2_EDGE_SPLIT": "3"}, {"DWT2_EDGE_SPLIT": "7"},
                                 {"DWT2_SEG_ROWS": "9", "DWT2_EDGE_SPLIT": "2"}])
def test_inverse_adjoint_unit_pieces_bit_identical(monkeypatch, env):
    """The edge units of the inverse and the adjoint run in pieces of a
    segment (each with its own warm-up rows) beside the inner units; a quad's
    arithmetic does not depend on which unit computes it, so every piece
    count and segment height gives the same bits, for single-image and
    grouped plans, and the pieces stay within the oracle's bound."""
    cases = [(512, 512), (257, 129), (130, 250), (100, 1028), (33, 65), (70, 1000)]
    base = []
    for h, w in cases:
        levels = _levels_max(h, w, 4)
        rng = np.random.default_rng(h * 7 + w)
        g = rng.standard_normal((h, w)).astype(np.float32)
        c = oracle.forward97(synth.uniform(h, w, seed=5).astype(np.float64), levels).astype(np.float32)
        base.append((gpu_adjoint(g, levels), gpu_inverse(c, levels, "reduced"), g, c, levels))
    shapes = synth.batch_shapes(12, seed=4)
    buf, descs = synth.batch_pack(shapes, seed=9)
    gd = torch.from_numpy(buf).cuda()
    plan = Plan(descs, 3, scheme="reduced")
    b_adj, b_inv = plan.adjoint(gd).cpu(), plan.inverse(gd).cpu()
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    for (a0, i0, g, c, levels), (h, w) in zip(base, cases):
        a1 = gpu_adjoint(g, levels)
        assert np.array_equal(a1, a0), f"adjoint {h}x{w} {env}"
        assert np.array_equal(gpu_inverse(c, levels, "reduced"), i0), f"inverse {h}x{w} {env}"
        ref = oracle.adjoint97(g.astype(np.float64), levels)
        assert np.abs(a1 - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max()) * 2 ** levels
    plan2 = Plan(descs, 3, scheme="reduced")
    assert torch.equal(plan2.adjoint(gd).cpu(), b_adj), f"grouped adjoint {env}"
    assert torch.equal(plan2.inverse(gd).cpu(), b_inv), f"grouped inverse {env}"
    assert plan2.status() == 0


def test_schemes_agree_with_each_other():
    # every scheme is within the FP32 bound of the oracle, so two schemes are
    # within twice that of each other, band by band
    x = synth.gradient(300, 260, seed=2)
    outs = [gpu_forward(x, 3, s) for s in SCHEMES97]
    for s, o in zip(SCHEMES97[1:], outs[1:]):
        assert_fp32_close(o, outs[0].astype(np.float64), 3, 2 * 255.0, f"{s} vs {SCHEMES97[0]}")


def test_plan_errors_on_gpu():
    from paper_1704_08657_gb300 import abi
    with pytest.raises(abi.Dwt2Error) as e:
        Plan.single(64, 64, 1, pitch=66)
    assert e.value.code == abi.DWT2_ERR_MISALIGNED
    with pytest.raises(abi.Dwt2Error) as e:
        Plan.single(64, 64, 7)
    assert e.value.code == abi.DWT2_ERR_LEVELS_TOO_DEEP
    with pytest.raises(abi.Dwt2Error) as e:
        Plan.single(64, 64, 1, wavelet="cdf53", scheme="reduced", coef_dtype=torch.int32)
    assert e.value.code == abi.DWT2_ERR_UNSUPPORTED
    # misaligned input pointer is rejected before any launch
    p = Plan.single(64, 64, 1)
    x = torch.zeros(64 * 64 + 1, device="cuda")
    rc = abi.raw_call("dwt2_forward", p.handle, x.data_ptr() + 4, torch.empty(64 * 64, device="cuda").data_ptr(),
                      p.workspace.data_ptr(), 0)
    assert rc == abi.DWT2_ERR_MISALIGNED


@pytest.mark.parametrize("n,levels", [(128, 1), (256, 1), (384, 1), (512, 1), (2048, 4), (2048, 5)])
@pytest.mark.parametrize("cfg", ["0", "1", "2", "3", "4"])
def test_unpadded_pitch_every_configuration(n, levels, cfg, monkeypatch):
    """pitch == width, every compiled kernel configuration: every coefficient
    is written (the output starts as NaN) and matches the oracle."""
    monkeypatch.setenv("DWT2_FWD_CFG", cfg)
    x = synth.gradient(n, n, seed=3)
    xd = torch.from_numpy(x).cuda()
    plan = Plan.single(n, n, levels, scheme="reduced")
    out = torch.full_like(xd, float("nan"))
    plan.forward(xd, out)
    torch.cuda.synchronize()
    assert plan.status() == 0
    got = out.cpu().numpy()
    assert not np.isnan(got).any(), f"{int(np.isnan(got).sum())} coefficients left unwritten"
    assert_fp32_close(got, oracle.forward97(x.astype(np.float64), levels), levels, 255.0, f"{n} L{levels} cfg {cfg}")


# ------------------------------------------------------------------ DD 13/7
# one lifting pair with 4-tap steps: strips with a 4-quad halo, 3 warm-up rows
DD_SCHEMES = ["nonsep", "reduced", "sep"]


@pytest.mark.parametrize("scheme", DD_SCHEMES)
@pytest.mark.parametrize("h,w", SHAPES + [(100, 1028), (66, 3000), (5, 7)])
def test_forward137_fp32(h, w, scheme):
    x = synth.uniform(h, w, seed=3 + h * 5 + w)
    for levels in sorted({1, _levels_max(h, w, 5)}):
        if levels == 0:
            continue
        ref = oracle.forward137(x.astype(np.float64), levels)
        got = gpu_forward(x, levels, scheme, wavelet="dd137")
        assert_dd_close(got, ref, levels, 255.0, f"dd137 {scheme} {h}x{w} L{levels}")


@pytest.mark.parametrize("scheme", DD_SCHEMES)
@pytest.mark.parametrize("h,w", [(512, 512), (33, 65), (7, 5), (2, 2), (130, 250), (257, 129), (100, 1028),
                                 (66, 3000)])
def test_inverse137_fp32(h, w, scheme):
    levels = _levels_max(h, w, 4)
    x = synth.uniform(h, w, seed=11)
    c = oracle.forward137(x.astype(np.float64), levels)
    got = gpu_inverse(c.astype(np.float32), levels, scheme, wavelet="dd137")
    ref = oracle.inverse137(c.astype(np.float32).astype(np.float64), levels)
    assert np.abs(got - ref).max() <= 1e-3, f"max err {np.abs(got - ref).max()}"
    rec = gpu_inverse(gpu_forward(x, levels, scheme, wavelet="dd137"), levels, scheme, wavelet="dd137")
    assert np.abs(rec - x).max() <= 2e-3


@pytest.mark.parametrize("dtype,rel", [(torch.float16, 1e-3), (torch.bfloat16, 8e-3)])
@pytest.mark.parametrize("h,w", [(512, 512), (130, 250), (96, 1028)])
def test_dd137_lowp_storage(h, w, dtype, rel):
    levels = _levels_max(h, w, 5)
    x = synth.noisy(h, w, seed=3)
    ref = oracle.forward137(x.astype(np.float64), levels)
    for scheme in DD_SCHEMES:
        got = gpu_forward(x, levels, scheme, dtype, "dd137")
        assert_lowp_close(got, ref, levels, rel, f"dd137 {dtype} {scheme}")
    c = ref.astype(np.float32)
    got = gpu_inverse(torch.from_numpy(c).to(dtype).float().numpy(), levels, "nonsep", dtype, "dd137")
    ref_i = oracle.inverse137(torch.from_numpy(c).to(dtype).double().numpy(), levels)
    assert np.abs(got - ref_i).max() <= 2e-3 * np.abs(ref_i).max() / 255.0 * 2


def test_dd137_has_no_adjoint_or_filter_bank_form():
    from paper_1704_08657_gb300 import abi
    with pytest.raises(abi.Dwt2Error) as e:
        Plan.single(64, 64, 2, wavelet="dd137", scheme="conv")
    assert e.value.code == abi.DWT2_ERR_UNSUPPORTED
    p = Plan.single(64, 64, 2, wavelet="dd137")
    g = torch.zeros(64, 64, device="cuda")
    rc = abi.raw_call("dwt2_adjoint", p.handle, g.data_ptr(), torch.empty_like(g).data_ptr(), p.workspace.data_ptr(), 0)
    assert rc == abi.DWT2_ERR_UNSUPPORTED


def test_dd137_schemes_agree():
    # the reduced split (Table 1: 2 steps, 50 operations) computes the same
    # transform as the plain non-separable and the separable lifting
    x = synth.gradient(300, 260, seed=8)
    outs = {s: gpu_forward(x, 4, s, wavelet="dd137") for s in DD_SCHEMES}
    for s in ("reduced", "sep"):
        assert_dd_close(outs[s], outs["nonsep"].astype(np.float64), 4, 2 * 255.0, f"dd137 {s} vs nonsep")

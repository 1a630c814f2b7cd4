"""Persistent forward (DWT2_FLAG_PERSISTENT): every level of every image in one
launch with a device work queue and bounded inter-level waits.

Checked against the oracle per image, against the per-level launches (same
arithmetic, so identical bits), under CUDA-graph capture, and with a dropped
completion signal, which must surface as DWT2_ERR_TIMEOUT from dwt2_status
without hanging, after which the context stays usable.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1704_08657_gb300 import abi, synth
from paper_1704_08657_gb300.dwt import Plan
from tests.util import assert_fp32_close, assert_lowp_close

pytestmark = pytest.mark.gpu


def _batch(shapes, seed=5, dtype=np.float32):
    buf, descs = synth.batch_pack(shapes, seed=seed)
    return buf.astype(dtype), descs


def _unpack(flat: np.ndarray, descs):
    return [flat[o:o + h * p].reshape(h, p)[:, :w] for (o, h, w, p) in descs]


@pytest.mark.parametrize("h,w,levels", [(512, 512, 5), (1000, 764, 4), (130, 250, 3), (7, 5, 2), (2, 2, 1),
                                        (2048, 96, 5), (33, 4100, 3)])
@pytest.mark.parametrize("scheme", ["reduced", "nonsep", "sep"])
@pytest.mark.parametrize("loader", ["tma", "cpasync"])
def test_persistent_single_image(h, w, levels, scheme, loader, monkeypatch):
    # the persistent launch loads with TMA (a device table of tensor maps);
    # the cp.async loader is forced here to cover it as well
    monkeypatch.setenv("DWT2_PML_CPASYNC", "1" if loader == "cpasync" else "0")
    x = synth.gradient(h, w, seed=2)
    pitch = (w + 3) // 4 * 4
    xd = torch.zeros((h, pitch), device="cuda")
    xd[:, :w] = torch.from_numpy(x).cuda()
    pp = Plan.single(h, w, levels, pitch=pitch, scheme=scheme, flags=abi.DWT2_FLAG_PERSISTENT)
    pl = Plan.single(h, w, levels, pitch=pitch, scheme=scheme)
    cp = pp.forward(xd)
    cl = pl.forward(xd)
    torch.cuda.synchronize()
    assert pp.status() == 0
    assert torch.equal(cp[:, :w], cl[:, :w]), "persistent and per-level launches differ"
    ref = oracle.forward97(x.astype(np.float64), levels)
    assert_fp32_close(cp[:, :w].cpu().numpy(), ref, levels, 255.0, f"persistent {scheme} {h}x{w}")


@pytest.mark.parametrize("n,seed", [(40, 4), (512, 4)])
def test_persistent_batch_uneven_images(n, seed):
    shapes = synth.batch_shapes(n, seed=seed)
    if n == 512:  # the full batch: sizes 64..2048, three levels
        assert min(min(s) for s in shapes) >= 64 and max(max(s) for s in shapes) <= 2048
    buf, descs = _batch(shapes)
    xd = torch.from_numpy(buf).cuda()
    plan = Plan(descs, 3, flags=abi.DWT2_FLAG_PERSISTENT)
    c = plan.forward(xd)
    torch.cuda.synchronize()
    assert plan.status() == 0
    got = _unpack(c.cpu().numpy(), descs)
    imgs = _unpack(buf, descs)
    for i, (g, x) in enumerate(zip(got, imgs)):
        if n == 512 and i % 16 != 0:
            continue  # the oracle checks every 16th image of the full batch
        ref = oracle.forward97(x.astype(np.float64), 3)
        assert_fp32_close(g, ref, 3, 255.0, f"image {i} {x.shape}")
    # every image also equals the one-launch-per-image path, bit for bit
    per = _unpack(Plan(descs, 3).forward(xd).cpu().numpy(), descs)
    for i, (a, b) in enumerate(zip(per, got)):
        assert np.array_equal(a, b), f"image {i}"  # padding between images is never written


def test_persistent_batch_lowp_and_int():
    shapes = synth.batch_shapes(24, seed=9)
    buf, descs = _batch(shapes)
    xd = torch.from_numpy(buf).cuda()
    imgs = _unpack(buf, descs)
    c = Plan(descs, 3, coef_dtype=torch.float16, flags=abi.DWT2_FLAG_PERSISTENT).forward(xd)
    got = _unpack(c.float().cpu().numpy(), descs)
    for g, x in zip(got, imgs):
        assert_lowp_close(g, oracle.forward97(x.astype(np.float64), 3), 3, 1e-3, "fp16 batch")
    bi = np.rint(buf).astype(np.int32)
    ci = Plan(descs, 3, wavelet="cdf53", coef_dtype=torch.int32, flags=abi.DWT2_FLAG_PERSISTENT).forward(
        torch.from_numpy(bi).cuda())
    goti = _unpack(ci.cpu().numpy(), descs)
    for g, x in zip(goti, _unpack(bi, descs)):
        assert np.array_equal(g.astype(np.int64), oracle.forward53i(x.astype(np.int64), 3))


def test_persistent_under_cuda_graph():
    shapes = synth.batch_shapes(64, seed=4)
    buf, descs = _batch(shapes)
    xd = torch.from_numpy(buf).cuda()
    plan = Plan(descs, 3, flags=abi.DWT2_FLAG_PERSISTENT)
    ws = plan.workspace  # allocated before capture
    out = torch.zeros_like(xd)  # pitch padding and gaps between images are never written
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.forward(xd, out, stream=s)  # warm-up outside the capture
    torch.cuda.synchronize()
    ref = out.clone()
    g = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(g, stream=s):
        plan.forward(xd, out, stream=s)
    for _ in range(3):
        out.zero_()
        g.replay()
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.equal(out, ref)
    del ws


def test_persistent_first_call_for_new_buffers_outside_capture():
    """The first call for a set of buffers writes the plan's tensor-map table
    (a synchronous copy): made during a stream capture it is refused before
    anything is recorded; after one call outside the capture the same buffers
    capture and replay."""
    shapes = synth.batch_shapes(20, seed=12)
    buf, descs = _batch(shapes)
    xd = torch.from_numpy(buf).cuda()
    plan = Plan(descs, 3, flags=abi.DWT2_FLAG_PERSISTENT)
    ws = plan.workspace
    out = torch.zeros_like(xd)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(abi.Dwt2Error) as e:
        with torch.cuda.graph(g, stream=s):
            plan.forward(xd, out, stream=s)
    assert e.value.code == abi.DWT2_ERR_INVALID_ARG
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        plan.forward(xd, out, stream=s)
    torch.cuda.synchronize()
    ref = out.clone()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s):
        plan.forward(xd, out, stream=s)
    out.zero_()
    g2.replay()
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.equal(out, ref)
    del ws


def test_dropped_signal_times_out_without_hanging(monkeypatch):
    monkeypatch.setenv("DWT2_TIMEOUT_MS", "30")
    h = w = 512
    x = torch.from_numpy(synth.uniform(h, w, seed=1)).cuda()
    plan = Plan.single(h, w, 3, flags=abi.DWT2_FLAG_PERSISTENT | abi.DWT2_TESTONLY_DROP_SIGNAL)
    plan.forward(x)
    assert plan.status() == abi.DWT2_ERR_TIMEOUT
    assert plan.status() == 0  # the status word was cleared
    # the context is still usable
    ok = Plan.single(h, w, 3, flags=abi.DWT2_FLAG_PERSISTENT)
    c = ok.forward(x)
    assert ok.status() == 0
    ref = oracle.forward97(x.cpu().numpy().astype(np.float64), 3)
    assert_fp32_close(c.cpu().numpy(), ref, 3, 255.0, "after timeout")


def test_batch_inverse_adjoint_and_l1():
    """Multi-image plans run the inverse and adjoint as grouped launches per
    level (up to 160 images a launch)."""
    shapes = synth.batch_shapes(30, seed=11)
    buf, descs = _batch(shapes)
    xd = torch.from_numpy(buf).cuda()
    plan = Plan(descs, 3, scheme="reduced")
    c = plan.forward(xd)
    rec = plan.inverse(c)
    g = torch.randn_like(xd)
    gin = plan.adjoint(g)
    gl1 = plan.adjoint_l1(c, 0.5)
    torch.cuda.synchronize()
    assert plan.status() == 0
    imgs = _unpack(buf, descs)
    cs = _unpack(c.cpu().numpy(), descs)
    for x, r, ci, gi, gref, gl in zip(imgs, _unpack(rec.cpu().numpy(), descs), cs, _unpack(g.cpu().numpy(), descs),
                                     _unpack(gin.cpu().numpy(), descs), _unpack(gl1.cpu().numpy(), descs)):
        assert np.abs(r - x).max() <= 2e-3
        ref = oracle.inverse97(ci.astype(np.float64), 3)
        assert np.abs(r - ref).max() <= 2e-3
        aref = oracle.adjoint97(gi.astype(np.float64), 3)
        assert np.abs(gref - aref).max() <= 1e-4 * max(1.0, np.abs(aref).max())
        sg = 0.5 * np.sign(ci.astype(np.float64))
        hl, wl = ci.shape
        for _ in range(3):
            hl, wl = (hl + 1) // 2, (wl + 1) // 2
        sg[:hl, :wl] = 0.0
        lref = oracle.adjoint97(sg, 3)
        assert np.abs(gl - lref).max() <= 1e-4 * max(1.0, np.abs(lref).max())
    # integer 5/3: the batched inverse is exact
    bi = np.rint(buf).astype(np.int32)
    pi = Plan(descs, 3, wavelet="cdf53", coef_dtype=torch.int32)
    ci = pi.forward(torch.from_numpy(bi).cuda())
    back = pi.inverse(ci)
    for x, r in zip(_unpack(bi, descs), _unpack(back.cpu().numpy(), descs)):
        assert np.array_equal(x, r)


@pytest.mark.parametrize("scheme,coef_dtype", [("reduced", torch.float32), ("sep", torch.float16),
                                               ("polyconv", torch.float32)])
def test_grouped_batch_equals_single_image_plans(scheme, coef_dtype):
    """A plan of several images runs each level as grouped launches (up to 76
    images per launch, every scheme); every image equals its own single-image
    plan bit for bit, for the default and for tuned configurations."""
    shapes = synth.batch_shapes(40, seed=7)
    buf, descs = _batch(shapes, seed=8)
    xd = torch.from_numpy(buf).cuda()
    plan = Plan(descs, 3, scheme=scheme, coef_dtype=coef_dtype)
    for choice in (-1, 0, 3 | (30 << 6) | (17 << 12)):  # the default, then per-level tuned configurations
        if choice >= 0:
            assert abi.dwt2_autotune(plan.handle, xd.data_ptr(), torch.empty_like(xd, dtype=coef_dtype).data_ptr(),
                                     plan.workspace.data_ptr(), 0, choice) == choice
        c = plan.forward(xd, torch.zeros_like(xd, dtype=coef_dtype))
        torch.cuda.synchronize()
        assert plan.status() == 0
        got = _unpack(c.float().cpu().numpy(), descs)
        for i, (o, h, w, p) in enumerate(descs):
            if i % 5:
                continue
            xi = xd[o:o + h * p].view(h, p).contiguous()
            single = Plan.single(h, w, 3, pitch=p, scheme=scheme, coef_dtype=coef_dtype).forward(xi)
            assert np.array_equal(single[:, :w].float().cpu().numpy(), got[i]), f"image {i} {h}x{w} choice {choice}"
    imgs = _unpack(buf, descs)
    for i in (0, 17, 39):
        ref = oracle.forward97(imgs[i].astype(np.float64), 3)
        if coef_dtype == torch.float32:
            assert_fp32_close(got[i], ref, 3, 255.0, f"image {i}")
        else:
            assert_lowp_close(got[i], ref, 3, 1e-3, f"image {i}")


def test_grouped_batch_int53():
    shapes = synth.batch_shapes(24, seed=12)
    buf, descs = _batch(shapes)
    bi = np.rint(buf).astype(np.int32)
    plan = Plan(descs, 3, wavelet="cdf53", scheme="nonsep", coef_dtype=torch.int32)
    c = plan.forward(torch.from_numpy(bi).cuda())
    torch.cuda.synchronize()
    assert plan.status() == 0
    for g, x in zip(_unpack(c.cpu().numpy(), descs), _unpack(bi, descs)):
        assert np.array_equal(g.astype(np.int64), oracle.forward53i(x.astype(np.int64), 3))


def test_grouped_batch_over_several_launches_and_graph():
    """More images than one launch holds (76): the level's launches overlap,
    the next level waits for all of them; the same under CUDA-graph capture."""
    shapes = synth.batch_shapes(200, seed=13)
    buf, descs = _batch(shapes, seed=14)
    xd = torch.from_numpy(buf).cuda()
    plan = Plan(descs, 3, scheme="reduced")
    ref = plan.forward(xd, torch.zeros_like(xd))
    torch.cuda.synchronize()
    assert plan.status() == 0
    got = _unpack(ref.cpu().numpy(), descs)
    imgs = _unpack(buf, descs)
    for i in range(0, 200, 9):
        assert_fp32_close(got[i], oracle.forward97(imgs[i].astype(np.float64), 3), 3, 255.0, f"image {i}")
    out = torch.zeros_like(xd)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.forward(xd, out, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(g, stream=s):
        plan.forward(xd, out, stream=s)
    for _ in range(3):
        out.zero_()
        g.replay()
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.equal(out, ref)


def test_grouped_batch_dd137():
    """DD 13/7 batches: each image equals its own single-image plan bit for bit
    and the oracle; the inverse reconstructs every image."""
    shapes = synth.batch_shapes(30, seed=31)
    buf, descs = _batch(shapes, seed=32)
    xd = torch.from_numpy(buf).cuda()
    plan = Plan(descs, 3, wavelet="dd137", scheme="nonsep")
    c = plan.forward(xd)
    torch.cuda.synchronize()
    assert plan.status() == 0
    got = _unpack(c.cpu().numpy(), descs)
    imgs = _unpack(buf, descs)
    for i, (o, h, w, p) in enumerate(descs):
        if i % 6:
            continue
        xi = xd[o:o + h * p].view(h, p).contiguous()
        single = Plan.single(h, w, 3, pitch=p, wavelet="dd137", scheme="nonsep").forward(xi)
        assert np.array_equal(single[:, :w].cpu().numpy(), got[i]), f"image {i} {h}x{w}"
        ref = oracle.forward137(imgs[i].astype(np.float64), 3)
        assert np.abs(got[i] - ref).max() <= 1e-3
    rec = plan.inverse(c)
    torch.cuda.synchronize()
    for x, r in zip(imgs, _unpack(rec.cpu().numpy(), descs)):
        assert np.abs(x - r).max() <= 2e-3

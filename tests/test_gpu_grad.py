"""Differentiation: DWT2Function and the wavelet-domain L1 loss.

* gradcheck of the GPU Function (FP32, loose tolerances: the path computes in
  FP32; the FP64 gradcheck pins the oracle's adjoint in test_oracle.py);
* the fused L1 gradient (dwt2_adjoint_l1) against the oracle's transpose
  applied to the same signs;
* central finite differences of the L1 loss along random directions on the
  full 16 x 4096 x 4096 four-level workload, with the error sign flips can
  cause bounded explicitly.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1704_08657_gb300 import synth
from paper_1704_08657_gb300.dwt import Plan, dwt2, l1_detail_loss

pytestmark = pytest.mark.gpu


def test_function_gradcheck_fp32():
    h, w = 24, 20
    plan = Plan.single(h, w, 2)
    x = torch.randn(h, w, device="cuda", generator=torch.Generator("cuda").manual_seed(3)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: dwt2(t, plan), (x,), eps=1e-2, atol=2e-2, rtol=1e-2,
                                    nondet_tol=1e-5)


def test_backward_is_the_adjoint():
    h, w, levels = 300, 260, 4
    plan = Plan.single(h, w, levels)
    x = torch.from_numpy(synth.uniform(h, w, seed=1)).cuda().requires_grad_(True)
    g = torch.randn(h, w, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    (dwt2(x, plan) * g).sum().backward()
    ref = oracle.adjoint97(g.double().cpu().numpy(), levels)
    assert np.abs(x.grad.cpu().numpy() - ref).max() <= 1e-4 * np.abs(ref).max()


def test_l1_gradient_matches_oracle_transpose():
    h, w, levels = 257, 188, 4
    plan = Plan.single(h, w, levels)
    x = torch.from_numpy(synth.noisy(h, w, seed=3)).cuda().requires_grad_(True)
    loss = l1_detail_loss(x, plan)
    loss.backward()
    c = plan.forward(x.detach()).double().cpu().numpy()
    sgn = np.sign(c) / plan.n_detail()
    hl, wl = h, w
    for _ in range(levels):
        hl, wl = (hl + 1) // 2, (wl + 1) // 2
    sgn[:hl, :wl] = 0.0
    ref = oracle.adjoint97(sgn, levels)
    got = x.grad.double().cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    # and the loss value
    det = np.abs(c).sum() - np.abs(c[:hl, :wl]).sum()
    assert abs(float(loss.detach()) - det / plan.n_detail()) <= 1e-6 * det / plan.n_detail()


@pytest.mark.slow
def test_l1_finite_differences_full_size():
    """16 images of 4096 x 4096, four levels: (L(x+hv) - L(x-hv)) / 2h equals
    <grad, v> up to FP32 rounding plus what sign flips between x-hv and x+hv
    can change, bounded by sum over flipped coefficients of (|c+| + |c-|)/(2h n)."""
    n_img, side, levels, hstep = 16, 4096, 4, 1e-2
    shapes = [(side, side)] * n_img
    descs, off = [], 0
    for (hh, ww) in shapes:
        descs.append((off, hh, ww, ww))
        off += hh * ww
    plan = Plan(descs, levels, scheme="reduced")
    gen = torch.Generator("cuda").manual_seed(6)
    x = (torch.randint(0, 256, (off,), device="cuda", generator=gen)).float()
    xg = x.clone().requires_grad_(True)
    l1_detail_loss(xg, plan).backward()
    grad = xg.grad
    n = plan.n_detail()

    def loss64(c):
        from paper_1704_08657_gb300.dwt import _abs_sum_images
        return (_abs_sum_images(c, plan.images) - _abs_sum_images(c, plan.coarsest_ll())) / n

    def detail_mask(c):
        m = torch.ones_like(c, dtype=torch.bool)
        flat = m.view(-1)
        for (o, hh, ww, p) in plan.coarsest_ll():
            flat[o:o + hh * p].view(hh, p)[:, :ww] = False
        return m

    mask = detail_mask(x)
    for k in range(8):
        v = torch.randn(off, device="cuda", generator=gen)
        cp = plan.forward(x + hstep * v)
        cm = plan.forward(x - hstep * v)
        fd = float((loss64(cp) - loss64(cm)) / (2 * hstep))
        ad = float((grad.double() * v.double()).sum())
        flip = (torch.sign(cp) != torch.sign(cm)) & mask
        bound = float(((cp.abs() + cm.abs()).double() * flip).sum()) / (2 * hstep * n)
        assert abs(fd - ad) <= bound + 1e-3 * abs(ad) + 1e-9, (k, fd, ad, bound, int(flip.sum()))
        del cp, cm, v, flip


def test_l1_backward_reads_its_scale_on_the_device():
    """dwt2_adjoint_l1_dev: the upstream gradient stays on the device (no host
    synchronisation in L1DetailLoss.backward), so the call also replays from a
    CUDA graph with a scale written after the capture."""
    from paper_1704_08657_gb300 import abi
    h, w, levels = 300, 260, 3
    plan = Plan.single(h, w, levels)
    x = torch.from_numpy(synth.uniform(h, w, seed=2)).cuda()
    c = plan.forward(x)
    inv_n = 1.0 / plan.n_detail()
    ref = plan.adjoint_l1(c, 2.5 * inv_n)
    sd = torch.tensor([2.5], device="cuda")
    out = torch.full_like(c, float("nan"))
    abi.dwt2_adjoint_l1_dev(plan.handle, c.data_ptr(), out.data_ptr(), sd.data_ptr(), inv_n,
                            plan.workspace.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert torch.allclose(out, ref, rtol=1e-6, atol=0)
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(graph, stream=s):
        abi.dwt2_adjoint_l1_dev(plan.handle, c.data_ptr(), out.data_ptr(), sd.data_ptr(), inv_n,
                                plan.workspace.data_ptr(), s.cuda_stream)
    sd.fill_(-5.0)
    out.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    assert torch.allclose(out, -2.0 * ref, rtol=1e-6, atol=0)
    assert plan.status() == 0
    # and autograd's backward goes through it
    xg = x.clone().requires_grad_(True)
    (3.0 * l1_detail_loss(xg, plan)).backward()
    assert torch.allclose(xg.grad, plan.adjoint_l1(c, 3.0 * inv_n), rtol=1e-6, atol=0)

"""Row bands of one image on the CPU: the partition arithmetic of
dwt2_band_rows / dwt2_band_rects, and two gloo ranks that each transform
their own band with the oracle and together reproduce the whole-image oracle
exactly.

The claim under test: a band that transforms its owned rows widened by
H = a*(2^L - 1) rows (rounded up to a multiple of 2^L) computes every owned
coefficient from image rows only, so its owned coefficients equal the
whole-image coefficients -- with the same arithmetic, bit for bit.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1704_08657_gb300 import abi, build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REACH = {abi.DWT2_CDF97: 4, abi.DWT2_CDF53_INT: 2, abi.DWT2_DD137: 6}


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return abi.load()


def _stitch_np(band_c, full_c, rects):
    for sr, dr, rows, c0, cols in rects:
        full_c[dr:dr + rows, c0:c0 + cols] = band_c[sr:sr + rows, c0:c0 + cols]


def _bands(wav, levels, h, n):
    return [abi.dwt2_band_rows(wav, levels, h, n, b) for b in range(n)]


@pytest.mark.parametrize("wav", [abi.DWT2_CDF97, abi.DWT2_CDF53_INT, abi.DWT2_DD137])
@pytest.mark.parametrize("levels,h,n", [(1, 9, 2), (2, 64, 2), (3, 101, 3), (5, 1000, 4), (4, 513, 5), (5, 4096, 7)])
def test_partition_tiles_the_rows(wav, levels, h, n):
    q = 1 << levels
    halo = -(-REACH[wav] * (q - 1) // q) * q
    bands = _bands(wav, levels, h, n)
    assert bands[0][0] == 0 and bands[-1][1] == h
    for b, (o0, o1, i0, i1) in enumerate(bands):
        assert o1 - o0 >= q
        assert o0 % q == 0 and (o1 % q == 0 or o1 == h)
        assert i0 == max(0, o0 - halo) and i1 == min(h, o1 + halo)
        assert i0 % q == 0  # the band's quads are the image's quads at every level
        if b + 1 < n:
            assert bands[b + 1][0] == o1


def test_partition_rejects_thin_bands():
    with pytest.raises(abi.Dwt2Error):
        abi.dwt2_band_rows(abi.DWT2_CDF97, 5, 40, 2, 0)  # 2 bands of >= 32 rows do not fit in 40
    with pytest.raises(abi.Dwt2Error):
        abi.dwt2_band_rows(abi.DWT2_CDF97, 1, 16, 2, 2)  # band index out of range
    with pytest.raises(abi.Dwt2Error):
        abi.dwt2_band_rows(9, 1, 16, 2, 0)  # unknown wavelet


@pytest.mark.parametrize("levels,h,w,n", [(1, 10, 7, 2), (3, 77, 40, 2), (4, 200, 33, 3), (5, 512, 96, 4)])
def test_rectangles_cover_every_coefficient_once(levels, h, w, n):
    cover = np.zeros((h, w), dtype=np.int32)
    for b in range(n):
        o0, o1, i0, i1 = abi.dwt2_band_rows(abi.DWT2_CDF97, levels, h, n, b)
        for sr, dr, rows, c0, cols in abi.dwt2_band_rects(abi.DWT2_CDF97, levels, h, w, n, b):
            assert 0 <= sr and sr + rows <= i1 - i0  # inside the band's own coefficients
            cover[dr:dr + rows, c0:c0 + cols] += 1
    assert (cover == 1).all()


@pytest.mark.parametrize("wav,fwd", [(abi.DWT2_CDF97, "forward97"), (abi.DWT2_CDF53_INT, "forward53i"),
                                     (abi.DWT2_DD137, "forward137")])
@pytest.mark.parametrize("levels,h,w,n", [(1, 40, 24, 2), (2, 75, 33, 2), (3, 200, 64, 3), (5, 640, 80, 3),
                                          (4, 333, 50, 4)])
def test_band_oracles_reproduce_the_whole_image(wav, fwd, levels, h, w, n):
    x = synth.uniform(h, w, seed=h + w)
    if wav == abi.DWT2_CDF53_INT:
        x = synth.to_int(x).astype(np.int64)
    f = getattr(oracle, fwd)
    ref = f(x, levels)
    got = np.full_like(ref, -7)
    for b in range(n):
        o0, o1, i0, i1 = abi.dwt2_band_rows(wav, levels, h, n, b)
        band_c = f(x[i0:i1], levels)
        _stitch_np(band_c, got, abi.dwt2_band_rects(wav, levels, h, w, n, b))
    assert np.array_equal(got, ref)


def test_band_without_halo_differs():
    # the pin has teeth: a band that starts at its first owned row (no halo)
    # gets its top coarsest-level coefficients wrong
    levels, h, w, n = 3, 200, 48, 2
    x = synth.uniform(h, w, seed=3).astype(np.float64)
    ref = oracle.forward97(x, levels)
    o0, o1, i0, i1 = abi.dwt2_band_rows(abi.DWT2_CDF97, levels, h, n, 1)
    sr, dr, rows, c0, cols = abi.dwt2_band_rects(abi.DWT2_CDF97, levels, h, w, n, 1)[-1]  # the coarsest LL
    good = oracle.forward97(x[i0:i1], levels)
    assert np.array_equal(good[sr, c0:c0 + cols], ref[dr, c0:c0 + cols])
    bad = oracle.forward97(x[o0:i1], levels)
    assert not np.allclose(bad[0, c0:c0 + cols], ref[dr, c0:c0 + cols])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as orc
        from paper_1704_08657_gb300 import abi as a, synth as sy
        h, w, levels = 300, 70, 4
        x = sy.gradient(h, w, seed=9)
        # each rank holds only the rows it transforms
        o0, o1, i0, i1 = a.dwt2_band_rows(a.DWT2_CDF97, levels, h, world, rank)
        band_c = orc.forward97(x[i0:i1].astype(np.float64), levels)
        part = np.zeros((h, w), dtype=np.float64)
        for sr, dr, rows, c0, cols in a.dwt2_band_rects(a.DWT2_CDF97, levels, h, w, world, rank):
            part[dr:dr + rows, c0:c0 + cols] = band_c[sr:sr + rows, c0:c0 + cols]
        t = torch.from_numpy(part)
        dist.all_reduce(t)  # owned rectangles are disjoint: the sum is the stitched pyramid
        ref = orc.forward97(x.astype(np.float64), levels)
        q.put((rank, bool(np.array_equal(t.numpy(), ref)), (o0, o1, i0, i1)))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_transform_one_image():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [True, True]
    (r0, r1) = [r[2] for r in res]
    assert r0[1] == r1[0]  # the owned rows meet
    assert r0[3] > r1[0] and r1[2] < r0[1]  # and the transformed rows overlap by the halos

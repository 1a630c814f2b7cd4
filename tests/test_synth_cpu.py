"""The synthetic input recipes (the stand-ins for the paper's unnamed images):
deterministic per seed, in range, with the shapes and totals the benchmark and
the design notes state."""
import numpy as np

from paper_1704_08657_gb300 import synth


def test_uniform_is_seeded_integers_in_range():
    a, b = synth.uniform(37, 53, seed=1), synth.uniform(37, 53, seed=1)
    assert a.dtype == np.float32 and np.array_equal(a, b)
    assert not np.array_equal(a, synth.uniform(37, 53, seed=2))
    assert a.min() >= 0 and a.max() <= 255 and np.all(a == np.rint(a))


def test_gradient_is_half_noise_plus_ramp():
    h, w = 40, 70
    x = synth.gradient(h, w, seed=2)
    assert x.min() >= 0 and x.max() <= 255
    ramp = 63.75 * (np.arange(h)[:, None] / (h - 1) + np.arange(w)[None, :] / (w - 1))
    half = x.astype(np.float64) - ramp
    assert np.abs(2 * half - np.rint(2 * half)).max() < 1e-4    # 0.5 * integer
    assert half.min() > -1e-4 and half.max() < 127.5 + 1e-4


def test_batch_recipe_512_images():
    shapes = synth.batch_shapes(512, seed=4)
    assert shapes == synth.batch_shapes(512, seed=4)
    sides = np.array(shapes)
    assert sides.min() >= 64 and sides.max() <= 2048 and np.all(sides % 2 == 0)
    assert int((sides[:, 0] * sides[:, 1]).sum()) == 177_416_064  # the bench's batch workload
    buf, descs = synth.batch_pack(shapes[:20], seed=5)
    end = 0
    for (o, h, w, p) in descs:
        assert o % 4 == 0 and p % 4 == 0 and p >= w and o >= end
        end = o + h * p
    assert buf.size >= end

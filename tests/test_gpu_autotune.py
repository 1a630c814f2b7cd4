"""dwt2_autotune: the chosen configuration is one of the candidates, keeps the
results identical (every configuration computes the same values), and a cached
choice is re-applied without timing."""
import json

import numpy as np
import pytest
import torch

import oracle
from paper_1704_08657_gb300 import abi, synth
from paper_1704_08657_gb300.dwt import Plan
from tests.util import assert_fp32_close

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("flags", [0, abi.DWT2_FLAG_PERSISTENT])
def test_autotune_keeps_results(tmp_path, flags):
    h, w, levels = 1500, 1300, 4
    x = torch.from_numpy(synth.gradient(h, w, seed=2)).cuda()
    plan = Plan.single(h, w, levels, scheme="reduced", flags=flags)
    before = plan.forward(x).clone()
    cache = str(tmp_path / "tune.json")
    choice = plan.autotune(x, cache=cache)
    assert choice >= 0
    after = plan.forward(x)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert torch.equal(before, after)
    assert_fp32_close(after.cpu().numpy(), oracle.forward97(x.cpu().numpy().astype(np.float64), levels), levels,
                      255.0, "autotuned")
    table = json.load(open(cache))
    assert table[plan.tune_key()] == choice
    # a second plan applies the cached choice
    p2 = Plan.single(h, w, levels, scheme="reduced", flags=flags)
    assert p2.autotune(x, cache=cache) == choice
    assert torch.equal(p2.forward(x), before)


@pytest.mark.parametrize("flags,bad", [(0, 1 << 12), (0, 63), (abi.DWT2_FLAG_PERSISTENT, 99)])
def test_autotune_rejects_bad_choice(flags, bad):
    # a two-level plan packs 6 bits per level (40 candidates: 5 configurations x
    # 8 segment heights): 2^12 or more, or a field of 40 or more, is not one of
    # its choices
    plan = Plan.single(64, 64, 2, flags=flags)
    x = torch.zeros((64, 64), device="cuda")
    with pytest.raises(abi.Dwt2Error):
        abi.dwt2_autotune(plan.handle, x.data_ptr(), x.data_ptr(), plan.workspace.data_ptr(), 0, bad)


def test_autotune_choice_fields_per_level():
    # every level's field decodes to a valid candidate, and applying a
    # hand-made choice (different candidates per level) keeps the results
    h, w, levels = 1024, 1536, 5
    x = torch.from_numpy(synth.uniform(h, w, seed=4)).cuda()
    plan = Plan.single(h, w, levels, scheme="sep")
    ref = plan.forward(x).clone()
    out = torch.empty_like(x)
    choice = 0
    for lev in range(levels):
        choice |= ((9 * lev + 3) % 32) << (6 * lev)
    assert abi.dwt2_autotune(plan.handle, x.data_ptr(), out.data_ptr(), plan.workspace.data_ptr(), 0, choice) == choice
    assert torch.equal(plan.forward(x), ref)
    assert plan.status() == 0


"""bench.py's reading of the library's tuning choices, on CPU.

The bench decodes a plan's tuning choice (6 bits per level: configuration x
segment height) into the per-level launch configuration it reports and uses to
look up the level-1 kernel's DRAM traffic; its tables must list the library's
compiled forward configurations and candidate segment heights in the
library's order.
"""
import json
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1704_08657_gb300", "csrc")


def _bench():
    sys.argv = [sys.argv[0]]
    import bench
    return bench


def test_configurations_match_the_library():
    src = open(os.path.join(CSRC, "launch.cuh")).read()
    body = src[src.index("#define DWT2_FWD_CFG_LIST(X)"):]
    body = body[:body.index("\n\n")]
    cfgs = [tuple(int(v) for v in m.groups()[1:])
            for m in re.finditer(r"X\((\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)", body)]
    assert tuple(cfgs) == _bench().FWD_CFGS
    n = int(re.search(r"constexpr int N_FWD_CFGS = (\d+);", open(os.path.join(CSRC, "internal.h")).read()).group(1))
    assert n == len(cfgs)


def test_segment_heights_match_the_library():
    src = open(os.path.join(CSRC, "api.cu")).read()
    segs = tuple(int(v) for v in re.search(r"const int TUNE_SEGS\[\] = \{([^}]*)\}", src).group(1).split(","))
    assert segs == _bench().TUNE_SEGS
    assert len(_bench().FWD_CFGS) * len(segs) <= 64  # a level's field holds 6 bits


def test_choice_decoding():
    b = _bench()
    nseg = len(b.TUNE_SEGS)
    fields = [3 * nseg + 0, 3 * nseg + 6, 4 * nseg + 4, 0 * nseg + 3, 2 * nseg + 1]
    choice = sum(f << (6 * i) for i, f in enumerate(fields))
    got = b.tuned_levels(choice, 7, False)
    want = [b.FWD_CFGS[f // nseg] + (b.TUNE_SEGS[f % nseg],) for f in fields]
    assert got == want + [want[-1]] * 2  # levels past the fifth share its field
    assert b.tuned_levels(choice, 5, True) == []  # persistent plans tune no per-level configuration


def test_traffic_table_covers_every_configuration():
    b = _bench()
    d = json.load(open(os.path.join(ROOT, "profiles", "forward_level1_traffic.json")))
    keys = {",".join(str(v) for v in c) for c in b.FWD_CFGS}
    assert set(d["dram_bytes_per_pixel"]) == keys
    # measured DRAM bytes per pixel of one level: near the 8 algorithmic bytes
    assert all(6.0 < v < 10.0 for v in d["dram_bytes_per_pixel"].values())
    assert re.fullmatch(r"[0-9a-f]{16}", d["kernel_hash"])

"""Constant tables inside the CUDA sources, checked against their definitions
on the host (no GPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_screening_rank_to_lane_table():
    # sph_screen.cuh: for a 4-lane group's hit mask `bits` and a rank idx,
    # the lane holding the (idx+1)-th hit, as 2-bit entries indexed by
    # key = 4 bits + idx (keys 0-31 in the first word, 32-63 in the second)
    src = open(os.path.join(ROOT, "paper_2107_07315_gb300", "csrc", "sph_screen.cuh")).read()
    m = re.search(r"key < 32u \? (0x[0-9a-f]+)ull : (0x[0-9a-f]+)ull", src)
    assert m, "table not found"
    words = [int(m.group(1), 16), int(m.group(2), 16)]
    for bits in range(16):
        lanes = [b for b in range(4) if (bits >> b) & 1]
        for idx in range(4):
            key = 4 * bits + idx
            got = (words[key // 32] >> (2 * (key % 32))) & 3
            if idx < len(lanes):
                assert got == lanes[idx], (bits, idx, got)
            else:
                assert got == 0, (bits, idx, got)

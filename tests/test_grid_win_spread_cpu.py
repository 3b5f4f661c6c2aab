"""The window gridding's jump-table spread (paper_2406_01342_gb300/csrc/
grid_win_spread.inc, generated by gen_grid_win_spread.py): the committed
include is what the generator writes, and every case of every kernel width
adds t * (h phi_u)(i) to exactly the accumulators of tile columns a0 + i that
lie inside the 32-column tile (the spread of Sect. 2.2's gridding sum along
u for one visibility), no other register, with the table covering every
column start a0 in [-(W - 1), 31].
"""
import importlib.util
import os
import re

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2406_01342_gb300", "csrc")


def _generator():
    spec = importlib.util.spec_from_file_location("gen_grid_win_spread", os.path.join(CSRC, "gen_grid_win_spread.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _committed_bodies():
    text = open(os.path.join(CSRC, "grid_win_spread.inc")).read()
    out = {}
    for m in re.finditer(r'#define PC_GW_SPREAD_ASM_(\d+) "(.*)"', text):
        out[int(m.group(1))] = m.group(2)
    return out


def test_committed_include_is_the_generators_output():
    gen = _generator()
    bodies = _committed_bodies()
    assert sorted(bodies) == [4, 5, 6, 7]
    for W, body in bodies.items():
        assert body == gen.body(W), W


@pytest.mark.parametrize("W", [4, 5, 6, 7])
def test_every_case_spreads_exactly_the_footprint_columns(W):
    body = _committed_bodies()[W].replace("\\n", "\n").replace("\\t", "")
    # the branch table lists the cases in order, and the dispatch reads %40
    table = re.search(r"gwt: \.branchtargets ([^;]*);", body).group(1).split(", ")
    assert table == [f"gwl{c}" for c in range(32 + W - 1)]
    assert "brx.idx.uni %40, gwt;" in body
    for c in range(32 + W - 1):
        a0 = c - (W - 1)
        line = re.search(rf"^gwl{c}: (.*)$", body, re.M).group(1)
        fmas = re.findall(r"fma\.rn\.f32x2 %(\d+), %(\d+), %(\d+), %(\d+);", line)
        want = {a0 + i: 32 + i for i in range(W) if 0 <= a0 + i < 32}
        got = {}
        for d, hu, t2, acc in fmas:
            d, hu, t2, acc = int(d), int(hu), int(t2), int(acc)
            assert d == acc and 0 <= d < 32          # accumulator in place
            assert t2 == 39                          # the packed pair (t, t)
            assert d not in got                      # each column once
            got[d] = hu
        assert got == want, (W, c)
        # every case but the last leaves through the join label
        assert ("bra.uni gwld;" in line) == (c != 32 + W - 2)

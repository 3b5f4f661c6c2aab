"""Writes grid_win_spread.inc: for each kernel width W, the inline-PTX body
that adds t * (h phi_u)(i) to the accumulators of tile columns a0 + i (i < W,
inside the 32-column tile), dispatched on a0 through a jump table (brx.idx)
instead of a tree of compare-and-branch. Operands: %0..%31 the 32 column
accumulators (packed complex FP32 pairs), %32..%38 h phi_u(i), %39 the packed
pair (t, t), %40 the case index a0 + W - 1.

Run from this directory after changing it: python gen_grid_win_spread.py
"""
import os

T = 32


def body(W):
    n_cases = T + W - 1
    lines = ["{",
             "gwt: .branchtargets " + ", ".join(f"gwl{c}" for c in range(n_cases)) + ";",
             "brx.idx.uni %40, gwt;"]
    for c in range(n_cases):
        a0 = c - (W - 1)
        ops = [f"fma.rn.f32x2 %{a0 + i}, %{32 + i}, %39, %{a0 + i};" for i in range(W) if 0 <= a0 + i < T]
        tail = [] if c == n_cases - 1 else ["bra.uni gwld;"]
        lines.append(f"gwl{c}: " + " ".join(ops + tail))
    lines.append("gwld:")
    lines.append("}")
    return "\\n\\t".join(lines)


def main():
    out = ["// Generated by gen_grid_win_spread.py: jump-table spreading of one slot",
           "// into the column accumulators of a window-gridding lane (grid_win.cu).",
           "#pragma once", ""]
    for W in range(4, 8):
        out.append(f"#define PC_GW_SPREAD_ASM_{W} \"{body(W)}\"")
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "grid_win_spread.inc"), "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()

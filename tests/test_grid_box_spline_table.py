"""The grid box spline weights the sampled stencil uses (the generated device
function in bsf_grid_box_spline.h) against the oracle's exact beta_b: every
triangle of every cell, at random positions on the 2^-10 grid."""
import os
import random
import re
from fractions import Fraction as Fr

from oracle import sampled as sp

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_1109_5114_gb300", "csrc",
                      "bsf_grid_box_spline.h")


def _weights():
    """{tri: [expr for w[0..8]]} parsed from the header's switch."""
    text = open(HEADER).read()
    out, tri = {}, None
    for line in text.splitlines():
        m = re.match(r"\s*(case (\d)|default):", line)
        if m:
            tri = int(m.group(2)) if m.group(2) else 3
            out[tri] = [None] * 9
            continue
        m = re.match(r"\s*w\[(\d)\] = (.*);", line)
        if m and tri is not None:
            out[tri][int(m.group(1))] = m.group(2)
    return out


def test_generated_weights_equal_the_exact_box_spline():
    W = _weights()
    assert sorted(W) == [0, 1, 2, 3] and all(None not in v for v in W.values())
    rng = random.Random(0)
    for _ in range(400):
        U, V = rng.randrange(0, 1024), rng.randrange(0, 1024)
        tri = (0 if U + V <= 1024 else 1) if V <= U else (2 if U + V >= 1024 else 3)
        env = {"U": U, "V": V, "UU": U * U, "UV": U * V, "VV": V * V}
        for i1 in (-1, 0, 1):
            for i2 in (-2, -1, 0):
                got = eval(W[tri][(i1 + 1) * 3 + (i2 + 2)], {}, env)  # noqa: S307 (integer expression)
                want = sp.beta(Fr(-i1) + Fr(U, 1024), Fr(-i2) + Fr(V, 1024), (Fr(1),) * 4) * (1 << sp.WEIGHT_BITS)
                assert got == want, (U, V, i1, i2)


KNIGHT_HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_1109_5114_gb300", "csrc",
                             "bsf_knight_box_spline.h")


def test_second_set_table_equals_the_exact_box_spline():
    text = open(KNIGHT_HEADER).read()
    body = text[text.index("{") + 1:text.rindex("}")]
    table = [int(v) for v in body.replace("\n", " ").split(",") if v.strip()]
    assert len(table) == 193 * 194 // 2
    rng = random.Random(1)
    for _ in range(300):
        a1, a2 = rng.randrange(-200, 201), rng.randrange(-200, 201)   # centred, units of 2^-6
        a, b = max(abs(a1), abs(a2)), min(abs(a1), abs(a2))
        got = table[a * (a + 1) // 2 + b] if a <= 192 else 0
        want = sp.beta_k(Fr(a1, 64), 3 + Fr(a2, 64), (Fr(1),) * 4) * sp.WEIGHT_DEN_K
        assert got == want, (a1, a2)

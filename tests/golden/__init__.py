"""Golden fixtures: values worked by hand from the paper's definitions (each file
cites its passage), and their parser."""
import os
from fractions import Fraction

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def degraf_cases(name: str = "degraf_hand_worked.txt"):
    """[(case, image uint8 [H, W], win_w, win_h, step, expected [(x, y) as Fractions])]."""
    cases, cur, rows = [], None, None
    for raw in open(os.path.join(HERE, name)):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "case":
            cur = {"name": tok[1], "points": {}}
            cases.append(cur)
        elif tok[0] == "window":
            cur["ww"], cur["wh"], cur["step"] = int(tok[1]), int(tok[2]), int(tok[4])
        elif tok[0] == "image":
            cur["W"], cur["H"] = int(tok[1]), int(tok[2])
            rows = cur["rows"] = []
        elif tok[0] == "point":
            k, ox, nx, dx, oy, ny, dy = (int(v) for v in tok[1:])
            cur["points"][k] = (ox + Fraction(nx, dx), oy + Fraction(ny, dy))
        else:
            rows.append([int(v) for v in tok])
    out = []
    for c in cases:
        img = np.array(c["rows"], dtype=np.uint8)
        assert img.shape == (c["H"], c["W"]), c["name"]
        pts = [c["points"][k] for k in range(len(c["points"]))]
        out.append((c["name"], img, c["ww"], c["wh"], c["step"], pts))
    return out

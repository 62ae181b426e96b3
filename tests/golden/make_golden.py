"""Writes golden_cases.json: the FP64 oracle's results for a few small,
formula-defined inputs.  Calls only the oracle package (test infrastructure);
run from the repository root:  python tests/golden/make_golden.py

Each case stores its inputs (float32-exact values), the parameters and the
oracle's outputs (the full rotation curve D(l), l*, s*, d2, and the
uncentred quantiles of the first image), so that the CUDA path can be checked
against stored values and changes to the oracle show up as diffs.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def gaussian(L, cx, cy, sx, sy, rho=0.0):
    """Anisotropic Gaussian on the L x L grid (pixel units, centre (cx, cy))."""
    y, x = np.mgrid[0:L, 0:L].astype(np.float64)
    dx, dy = (x - cx) / sx, (y - cy) / sy
    return np.exp(-0.5 * (dx * dx + dy * dy - 2 * rho * dx * dy) / (1 - rho * rho))


def shifted(img, dr, dc):
    """Integer shift with zero fill."""
    out = np.zeros_like(img)
    L = img.shape[0]
    rs, rd = (slice(0, L - dr), slice(dr, L)) if dr >= 0 else (slice(-dr, L), slice(0, L + dr))
    cs, cd = (slice(0, L - dc), slice(dc, L)) if dc >= 0 else (slice(-dc, L), slice(0, L + dc))
    out[rd, cd] = img[rs, cs]
    return out


def f32(a):
    a = np.asarray(a, dtype=np.float64)
    return (a / a.sum()).astype(np.float32)


def cases():
    A = f32(gaussian(16, 6.5, 8.2, 2.0, 3.0, 0.3) + 0.6 * gaussian(16, 10.0, 6.0, 1.5, 1.5))
    B = f32(shifted(np.rot90(A.astype(np.float64)), 1, -2))  # quarter turn, then shift
    C = f32(gaussian(24, 11.0, 12.5, 3.0, 2.0, -0.4) + 0.5 * gaussian(24, 15.0, 9.0, 2.0, 2.5))
    D = f32(gaussian(24, 12.0, 11.0, 2.5, 3.5, 0.2))
    return [
        dict(name="quarter_turn_shift_16", f=A, g=B, n=16, M=8, translation=1, level_rule=0),
        dict(name="rotation_only_16", f=A, g=B, n=16, M=8, translation=0, level_rule=0),
        dict(name="two_mixtures_24_n12", f=C, g=D, n=12, M=5, translation=1, level_rule=0),
        dict(name="left_levels_24_n20", f=D, g=C, n=20, M=9, translation=0, level_rule=1),
    ]


def main():
    out = []
    for c in cases():
        f, g = c["f"].astype(np.float64), c["g"].astype(np.float64)
        res, D, S = oracle.align_pair(f, g, c["n"], c["M"], level_rule=c["level_rule"],
                                      translation=c["translation"])
        F, _ = oracle.prepare(f)
        Q = oracle.quantiles(oracle.project(F, c["n"]), 2.0 / F.shape[0], c["M"],
                             level_rule=c["level_rule"])
        out.append({
            "name": c["name"], "n": c["n"], "M": c["M"], "translation": c["translation"],
            "level_rule": c["level_rule"], "L": int(f.shape[0]),
            "f": c["f"].tolist(), "g": c["g"].tolist(),
            "D": D.tolist(), "shifts": S.tolist(), "best_l": int(res["best_l"]),
            "d2": float(res["d2"]), "shift": [float(v) for v in res["shift"]],
            "quantiles_f": Q.tolist(),
        })
    with open(os.path.join(HERE, "golden_cases.json"), "w") as fh:
        json.dump({"generator": "tests/golden/make_golden.py (FP64 oracle)", "cases": out}, fh,
                  indent=None, separators=(",", ":"))
        fh.write("\n")


if __name__ == "__main__":
    main()

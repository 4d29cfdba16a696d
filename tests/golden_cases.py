"""Loads the hand-worked fixtures of ``tests/golden/hand_worked.json``."""

import json
import os

import numpy as np

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hand_worked.json")


def cases():
    with open(_PATH) as f:
        return json.load(f)["cases"]


def plane(case):
    dt = np.uint8 if case["bit_depth"] == 8 else np.uint16
    p = np.full((case["height"], case["width"]), case["base"], dt)
    for x0, x1, y0, y1, v in case["paint"]:
        p[y0:y1, x0:x1] = v
    return p


def times(case):
    return np.array(case["times"], np.float32)


def band_masks(case):
    return [sum(1 << (y - 1) for y in cuts) for cuts in case["expect"]["band_cuts"]]

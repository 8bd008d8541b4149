"""Readers for the cited fixtures under tests/golden/."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


def philox_kat():
    out = []
    for line in _lines("philox4x32_10_kat.txt"):
        words = [int(x, 16) for x in line.split()]
        out.append((words[0:4], words[4:6], words[6:10]))
    return out


def table1():
    blocks, cur = {}, None
    for line in _lines("table1_dij.txt"):
        if line.startswith("L "):
            cur = int(line.split()[1])
            blocks[cur] = []
        else:
            blocks[cur].append([float(x) for x in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def d2q5_matrix(theta):
    rows = []
    env = {"sqrt": math.sqrt, "theta": theta, "__builtins__": {}}
    for line in _lines("d2q5_moment_matrix.txt"):
        rows.append([float(eval(cell.strip(), env)) for cell in line.split("|")])
    return np.array(rows)

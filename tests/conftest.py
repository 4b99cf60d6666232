import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_graph_fixture(name):
    """Parses a golden graph file: returns (n, n_labels, src, dst, lab, vlabel)."""
    src, dst, lab = [], [], []
    n = L = 0
    vl = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "V":
                n, L = int(t[1]), int(t[2])
            elif t[0] == "vl":
                vl[int(t[1])] = int(t[2])
            elif t[0] == "e":
                src.append(int(t[1]))
                dst.append(int(t[2]))
                lab.append(int(t[3]))
    vlabel = np.array([vl.get(i, 0) for i in range(n)], dtype=np.uint8) if vl else None
    return (n, L, np.array(src, dtype=np.uint32), np.array(dst, dtype=np.uint32),
            np.array(lab, dtype=np.uint16), vlabel)


def load_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            rows.append([int(x) for x in t])
    return np.array(rows, dtype=np.uint32)


def load_crpq_fixture(name):
    vars_, atoms, tuples = {}, [], []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "var":
                vars_[int(t[1])] = int(t[2])
            elif t[0] == "atom":
                atoms.append((int(t[1]), t[2], int(t[3])))
            elif t[0] == "t":
                tuples.append([int(x) for x in t[1:]])
    var_label = [vars_[i] for i in range(len(vars_))]
    return var_label, atoms, np.array(tuples, dtype=np.uint32)

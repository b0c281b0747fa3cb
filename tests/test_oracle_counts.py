"""Pins the MMBF counting of the oracle to the paper's Table ntmmbfs."""
import os

import numpy as np

from oracle.counts import mmbf_count

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ntmmbfs.txt")


def _rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                a, b, c, n1, n4, ratio = line.split()
                rows.append((int(a), int(b), int(c), int(n1), int(n4), float(ratio)))
    return rows


def test_table_ntmmbfs_exact():
    rows = _rows()
    assert len(rows) == 6
    for a, b, c, n1, n4, ratio in rows:
        assert mmbf_count((a, b, c), (1, 1, 1)) == n1
        assert mmbf_count((a, b, c), (4, 4, 1)) == n4
        assert abs(n4 / n1 - ratio) < 1e-4

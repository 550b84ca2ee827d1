"""Values the paper prints, checked against the readings the code takes.

tests/golden/table1_alpha.txt holds Table 1 of Sec. 5.2.  Its alpha column
fixes what alpha means: the number of references attached to bridge vectors
divided by the number of bridge vectors n^P (the quantity ann_index_get_info
reports as alpha), not a share of the N references."""
from __future__ import annotations

import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_alpha.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, N, P, n, ref, alpha = line.split()
                rows.append((name, int(N), int(P), int(n), int(ref), alpha))
    return rows


def printed_interval(text):
    """The interval a printed decimal stands for (half a unit of its last digit)."""
    half = 0.5 * 10.0 ** -(len(text.split(".")[1]) if "." in text else 0)
    return float(text) - half, float(text) + half


def consistent(value_lo, value_hi, text):
    lo, hi = printed_interval(text)
    return value_lo <= hi and value_hi >= lo


def test_alpha_is_references_per_bridge_vector():
    rows = table1()
    assert [r[0] for r in rows] == ["SIFT", "GIST", "HOG"]
    for name, N, P, n, ref, alpha in rows:
        # #reference is printed rounded to thousands
        lo, hi = (ref - 500) / n ** P * 100, (ref + 500) / n ** P * 100
        assert consistent(lo, hi, alpha), name


def test_alpha_is_not_a_share_of_the_references():
    for name, N, P, n, ref, alpha in table1():
        lo, hi = (ref - 500) / N * 100, (ref + 500) / N * 100
        assert not consistent(lo, hi, alpha), name

"""The power-trace schedule of the subset kernel, checked on the host.

The kernel takes, for each half photon number h, a fixed list of operations
from the table `c_sched` in csrc/haf_subsets.cu: products
buf[k] = buf[a] X buf[b] (R_{p+q} = R_p X R_q) and traces tr(X buf[a]) or
tr(X buf[a] X buf[b]). This test reads that table and replays it with the
power held by each buffer: every trace k = 1..h must come out exactly once
with power k, a product must not write one of its operands, and every buffer
index of a row must fit the number of buffers a lane group running that row
keeps (`sched_nbuf` in csrc/gbs_internal.cuh).
"""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1908_10070_gb300", "csrc")


def _table():
    src = open(os.path.join(CSRC, "haf_subsets.cu")).read()
    i = src.index("__constant__ SchedOp c_sched")
    j = src.index("};", i)
    rows = {}
    for ln in src[i:j].split("\n"):
        if "// h = " not in ln:
            continue
        h = int(ln.split("// h = ")[1])
        ops = [(k, int(a), int(b), int(c)) for k, a, b, c in re.findall(r"\{(k\w+), (-?\d+), (-?\d+), (-?\d+)\}", ln)]
        rows[h] = ops
    return rows


def _nbuf(hs):
    """sched_nbuf from gbs_internal.cuh: its packed table (3 bits per row)."""
    src = open(os.path.join(CSRC, "gbs_internal.cuh")).read()
    i = src.index("inline int sched_nbuf(int hs) {")
    body = src[i:src.index("}", i)]
    k = int(re.search(r"(0x[0-9a-fA-F]+)ull", body).group(1), 16)
    return (k >> (3 * hs)) & 7


def _replay(ops):
    buf = {0: 1}
    got = {}
    for kind, x, y, z in ops:
        if kind == "kEnd":
            break
        if kind == "kProd":
            assert y in buf and z in buf, ("operand not formed", x, y, z)
            assert x not in (y, z), ("product writes its operand", x, y, z)
            buf[x] = buf[y] + buf[z]
        elif kind == "kTr1":
            got.setdefault(x, []).append(buf[y])
        else:
            got.setdefault(x, []).append(buf[y] + buf[z])
    used = [x for kind, x, y, z in ops if kind == "kProd"] + [0]
    return got, max(used)


def test_every_trace_once_with_its_power():
    rows = _table()
    assert sorted(rows) == list(range(0, 17))
    for h, ops in rows.items():
        got, _ = _replay(ops)
        assert sorted(got) == list(range(1, h + 1)), (h, got)
        for k, powers in got.items():
            assert powers == [k], (h, k, powers)


def test_pair_sum_product_comes_first():
    """The kernel forms R_2 from the pair sums only for the op buf[1] = buf[0] X buf[0]."""
    for h, ops in _table().items():
        prods = [op for op in ops if op[0] == "kProd"]
        if h >= 3:
            assert prods[0] == ("kProd", 1, 0, 0), (h, prods[0])


@pytest.mark.parametrize("hs", range(0, 17))
def test_buffers_fit_the_lane_group(hs):
    """A lane group running schedule row hs keeps sched_nbuf(hs) matrices:
    every buffer index of the row fits, and the count is the row's own (the
    largest index plus one), so no group is sized for a row it does not run."""
    ops = _table()[hs]
    nb = _nbuf(hs)
    top = 0
    for kind, x, y, z in ops:
        if kind == "kEnd":
            break
        top = max(top, x if kind == "kProd" else 0, y, z)
    assert top + 1 == nb, (hs, top, nb)


def test_products_per_h():
    """The fewest products whose powers F satisfy F + F >= {1..h} (R_2 counted)."""
    want = {1: 0, 2: 0, 3: 1, 4: 1, 5: 2, 6: 2, 7: 3, 8: 3, 9: 3, 10: 3, 11: 4, 12: 4, 13: 4, 14: 4, 15: 5, 16: 5}
    for h, ops in _table().items():
        if h == 0:
            continue
        assert sum(1 for op in ops if op[0] == "kProd") == want[h], h

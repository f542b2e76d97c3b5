"""Host model of the marching eta pass's step schedule (`march_col` in csrc/sweep.cuh).

A CTA of EW warps walks a column segment [s0, s1) EW rows per step; warp w of the step at row r
stages node r + K + w into a ring of ERING row slots, then takes, in the per-interface layout,
the interface and output r - 1 + w, or, in the centre layout (FP64 one-midpoint schemes), the
centre r - 1 + w and the interface and output r - 2 + w.  Each lane is one column, so all data
moves along a column between warps, through three shared-memory rings: staged nodes, Q+ of
each centre (centre layout) and h of each interface.

The phases of a step are separated by block barriers (__syncthreads).  The model builds the
happens-before order of one segment from program order and the barriers, where a synchronisation
point is either a block barrier ("full") or a hand-off from warp to warp ("chain": warp w
waits until warp w - 1 has arrived, then arrives itself, so that after its wait it follows
every earlier phase of warps 0 .. w - 1; a weaker point the tests use to show that the block
barriers cannot be thinned that way everywhere), and checks, for the kernel's segment lengths
and eight-step ones, every column length up to a segment and a few of two and three segments
(first, inner and last segments), and stencil half-widths 2 (WENOIU3/5) and 3 (WENOIU7):
* every ring row a phase reads was written before the read, and every other row written to
  the same slot is ordered before that write or after the read;
* every centre, interface and output of the segment is taken exactly once, within the step
  count the kernel computes.

EW and ERING are read from the header so that the model follows the kernel's constants.
"""
import os
import re

import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_1810_11103_gb300", "csrc", "sweep.cuh")


def _const(name):
    with open(HDR) as f:
        m = re.search(r"constexpr int %s = (\d+);" % name, f.read())
    assert m, name
    return int(m.group(1))


EW = _const("EW")
ERING = _const("ERING")
NMP = 1

# phases and the synchronisation after each, per layout
LAYOUTS = {
    # per-interface layout (the float paths): two block barriers per step
    "barriers": [("stage", "full"), ("iface", "full"), ("out", None)],
    # centre layout (FP64 one-midpoint schemes): three block barriers per step
    "centre": [("stage", "full"), ("centre", "full"), ("iface", "full"), ("out", None)],
}


class Order:
    """Nodes in construction (topological) order with their ancestor sets as bit masks."""

    def __init__(self):
        self.anc = []

    def node(self, preds):
        a = 0
        for p in preds:
            if p is not None:
                a |= self.anc[p] | (1 << p)
        self.anc.append(a)
        return len(self.anc) - 1

    def before(self, a, b):
        return (self.anc[b] >> a) & 1 == 1


def schedule(s0, s1, n, H, K, layout):
    """Accesses of one segment: writes[ring] = [(row, node)], reads = [(ring, row, node)]."""
    centre = layout.startswith("centre")
    phases = LAYOUTS[layout]
    lag = 2 if centre else 1
    steps = (s1 - s0 + 2 * NMP - 1 + (1 if centre else 0) + EW - 1) // EW
    order = Order()
    writes = {"node": [], "qp": [], "h": []}
    reads = []
    taken = {"iface": [], "out": [], "centre": []}
    last = [None] * EW                                   # each warp's latest node

    def staged(m):
        return m <= s1 + 3 and m <= n + 3

    for w in range(EW):                                  # start-up: rows below s0 + K
        last[w] = order.node([])
        if w < K + NMP + H and staged(s0 - NMP - H + w):
            writes["node"].append((s0 - NMP - H + w, last[w]))

    def phase(name, t, w, nd):
        r = s0 + EW * t
        if name == "stage":
            m = r + K + w
            if staged(m):
                writes["node"].append((m, nd))
        elif name == "centre":
            c = r - 1 + w
            if c <= s1:
                taken["centre"].append(c)
                reads.extend(("node", x, nd) for x in range(c - H, c + H + 1))
                writes["qp"].append((c, nd))
        elif name == "iface":
            q = r - NMP - (1 if centre else 0) + w
            if s0 - NMP <= q <= s1 + NMP - 2:
                taken["iface"].append(q)
                # both sides' stencils (per-interface layout), the midpoint metrics and the
                # central part of h (q - 2 .. q + 3; q - 3 .. q + 4 for WENOIU7)
                lo, hi = (q - 3, q + 4) if H == 3 else (q - 2, q + 3)
                reads.extend(("node", x, nd) for x in range(lo, hi + 1))
                if centre:
                    reads.append(("qp", q, nd))
                writes["h"].append((q, nd))
            s = r - lag + w
            if s0 <= s < s1:
                reads.append(("node", s, nd))            # the output's stage state, read here
        elif name == "out":
            s = r - lag + w
            if s0 <= s < s1:
                taken["out"].append(s)
                reads.extend([("h", s, nd), ("h", s - 1, nd)])

    for t in range(steps):
        for name, sync in phases:
            for w in range(EW):
                last[w] = order.node([last[w]])
                phase(name, t, w, last[w])
            if sync == "full":
                b = order.node(last)
                last = [b] * EW
            elif sync == "chain":
                arrived = None
                for w in range(EW):
                    waited = order.node([last[w], arrived])      # wait for warp w - 1
                    arrived = order.node([waited])               # then arrive for warp w + 1
                    last[w] = arrived
    return order, writes, reads, taken


def hazards(order, writes, reads):
    bad = []
    for ring, row, nd in reads:
        slot = [(r, wn) for (r, wn) in writes[ring] if r % ERING == row % ERING]
        mine = [wn for (r, wn) in slot if r == row]
        if len(mine) != 1 or not order.before(mine[0], nd):
            bad.append((ring, "not visible", row))
            continue
        for r, wn in slot:
            if r != row and not (order.before(wn, mine[0]) or order.before(nd, wn)):
                bad.append((ring, "overwritten", row, r))
    return bad


def _segments(seg):
    # every segment length up to a full one, and columns of two to three segments
    for n in list(range(1, seg + 3)) + [2 * seg - 1, 2 * seg, 2 * seg + 1, 3 * seg - 2]:
        for s0 in range(0, n, seg):
            yield n, s0, min(n, s0 + seg)


# the kernel's segments (sixteen steps in FP64, 32 in the float paths) and eight-step ones
@pytest.mark.parametrize("layout,steps", [("barriers", 32), ("centre", 16), ("barriers", 8), ("centre", 8)])
@pytest.mark.parametrize("H,K", [(2, 2), (3, 3)])
def test_eta_march_schedule(layout, H, K, steps):
    seg = steps * EW - 1 - (1 if layout.startswith("centre") else 0)
    for n, s0, s1 in _segments(seg):
        order, writes, reads, taken = schedule(s0, s1, n, H, K, layout)
        assert hazards(order, writes, reads) == [], (layout, n, s0, s1)
        assert sorted(taken["iface"]) == list(range(s0 - 1, s1)), (n, s0)
        assert sorted(taken["out"]) == list(range(s0, s1)), (n, s0)
        if layout.startswith("centre"):
            assert sorted(taken["centre"]) == list(range(s0 - 1, s1 + 1)), (n, s0)


@pytest.mark.parametrize("layout,weaker", [
    ("centre", [("stage", "full"), ("centre", None), ("iface", "full"), ("out", None)]),
    ("centre", [("stage", "full"), ("centre", "full"), ("iface", None), ("out", None)]),
    ("centre", [("stage", "chain"), ("centre", "full"), ("iface", "full"), ("out", None)]),
    ("barriers", [("stage", "full"), ("iface", None), ("out", None)]),
    ("barriers", [("stage", None), ("iface", "full"), ("out", None)]),
    ("barriers", [("stage", "chain"), ("iface", "chain"), ("out", None)]),
])
def test_eta_march_schedule_catches_a_missing_barrier(layout, weaker):
    # a barrier dropped, or the staging barrier weakened to a hand-off, must show up as a hazard
    keep = LAYOUTS[layout]
    try:
        LAYOUTS[layout] = weaker
        order, writes, reads, _ = schedule(0, 62, 200, 2, 2, layout)
        assert hazards(order, writes, reads)
    finally:
        LAYOUTS[layout] = keep


def test_eta_march_schedule_catches_a_short_ring():
    # a ring of 8 row slots, fewer than the rows a step reads and stages, must fail
    global ERING
    keep = ERING
    try:
        ERING = 8
        order, writes, reads, _ = schedule(0, 62, 200, 3, 3, "centre")
        assert hazards(order, writes, reads)
    finally:
        ERING = keep

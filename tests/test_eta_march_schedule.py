"""Host model of the marching eta pass's step schedule (`march_col` in csrc/sweep.cuh).

A CTA of EW warps walks a column segment [s0, s1) EW rows per step; warp w of the step at row r
stages node r + K + w into a ring of ERING row slots, then (FP64 one-midpoint schemes) takes
the centre r - 1 + w, the interface r - 2 + w and the output r - 2 + w, or (per-interface
layout) the interface and output r - 1 + w.  Block barriers split a step into barrier
intervals: staging | centres | interfaces | outputs, where the outputs of step t share an
interval with the staging of step t + 1.  The model checks, for columns of 1 to 129, 255, 256
and 299 rows (every segment length up to a full segment, first, inner and last segments) and
stencil half-widths 2 (WENOIU3/5) and 3 (WENOIU7):

* every row a phase reads from a ring (node ring, Q+ ring, h ring) was written in an earlier
  interval and no other row overwrites its slot up to and including the reading interval;
* every interface s0 - 1 .. s1 - 1, every output s0 .. s1 - 1 and (centre layout) every
  centre s0 - 1 .. s1 is taken exactly once, within the step count the kernel computes.

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


def schedule(s0, s1, n, H, K, centre, centre_barrier=True):
    """Writes and reads of one segment: (ring, row, interval) triples, and what was taken."""
    lag = 2 if centre else 1
    steps = (s1 - s0 + 2 * NMP - 1 + (1 if centre else 0) + EW - 1) // EW
    writes = {"node": [], "qp": [], "h": []}
    reads = []
    taken = {"iface": [], "out": [], "centre": []}

    def staged(m):
        return m <= s1 + 3 and m <= n + 3

    for w in range(EW):                                  # start-up rows below s0 + K
        if w < K + NMP + H and staged(s0 - NMP - H + w):
            writes["node"].append((s0 - NMP - H + w, 0))
    for t in range(steps):
        r = s0 + EW * t
        if centre:   # stage | centres | interfaces | outputs: three barriers per step
            i_stage, i_centre, i_iface, i_out = 3 * t, 3 * t + 1, 3 * t + 2, 3 * t + 3
            if not centre_barrier:
                i_iface = i_centre
        else:        # stage | interfaces | outputs: two barriers per step
            i_stage, i_iface, i_out = 2 * t, 2 * t + 1, 2 * t + 2
        for w in range(EW):
            m = r + K + w
            if staged(m):
                writes["node"].append((m, i_stage))
            if centre:
                c = r - 1 + w
                if c <= s1:
                    taken["centre"].append(c)
                    reads += [("node", x, i_centre) for x in range(c - H, c + H + 1)]
                    writes["qp"].append((c, i_centre))
            q = r - NMP - (1 if centre else 0) + w
            if s0 - NMP <= q <= s1 + NMP - 2:
                taken["iface"].append(q)
                lo, hi = (q - 3, q + 4) if H == 3 else (q - 2, q + 3)
                reads += [("node", x, i_iface) for x in range(lo, hi + 1)]
                if centre:
                    reads.append(("qp", q, i_iface))
                writes["h"].append((q, i_iface))
            s = r - lag + w
            if s0 <= s < s1:
                taken["out"].append(s)
                reads += [("node", s, i_iface), ("h", s, i_out), ("h", s - 1, i_out)]
    return writes, reads, taken


def hazards(writes, reads):
    bad = []
    for ring, row, iv in reads:
        hist = [(i, r) for (r, i) in writes[ring] if r % ERING == row % ERING]
        mine = [i for (i, r) in hist if r == row and i < iv]
        if not mine:
            bad.append((ring, "not visible", row, iv))
            continue
        # from the interval of the row's write up to the read, no other row in the slot
        if any(max(mine) <= i <= iv and r != row for (i, r) in hist):
            bad.append((ring, "overwritten", row, iv))
    return bad


@pytest.mark.parametrize("centre", [True, False])
@pytest.mark.parametrize("H,K", [(2, 2), (3, 3)])
def test_eta_march_schedule(centre, H, K):
    seg = 8 * EW - 1 - (1 if centre else 0)
    for n in list(range(1, 130)) + [255, 256, 299]:
        for s0 in range(0, n, seg):
            s1 = min(n, s0 + seg)
            writes, reads, taken = schedule(s0, s1, n, H, K, centre)
            assert hazards(writes, reads) == [], (n, s0, s1)
            assert sorted(taken["iface"]) == list(range(s0 - 1, s1)), (n, s0)
            assert sorted(taken["out"]) == list(range(s0, s1)), (n, s0)
            if centre:
                assert sorted(taken["centre"]) == list(range(s0 - 1, s1 + 1)), (n, s0)


def test_eta_march_schedule_catches_a_missing_barrier():
    # without the barrier between the centres and the interfaces, Q+ from the warp below is
    # read in the interval that writes it
    writes, reads, _ = schedule(0, 62, 200, 2, 2, True, centre_barrier=False)
    assert any(ring == "qp" for ring, *_ in hazards(writes, reads))


def test_eta_march_schedule_catches_a_short_ring():
    # a ring of 8 row slots, fewer than the rows a step reads and stages, must fail
    global ERING
    keep = ERING
    try:
        ERING = 8
        writes, reads, _ = schedule(0, 62, 200, 3, 3, True)
        assert hazards(writes, reads)
    finally:
        ERING = keep

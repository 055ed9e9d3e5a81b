"""A CPU model of the shared-memory pipeline of the two-stage 2D kernel
(paper_1109_1027_gb300/csrc/stage2d_fused.cu), in place of a race checker:
for every block height it replays which ring slot each iteration of the
walk writes (or fills by TMA), waits for and reads, and checks that every
read finds the row it expects, written or waited for before the CTA barrier
that precedes the read and not overwritten since.  The ring sizes and the
lag are read from the kernel source, so the model follows them.

Schedule (iteration `it`, one CTA barrier at its top; stage A runs output
row q = it, stage B output row e = it - LAG):
  * stage-A input ring (SA slots, TMA): rows 0..SA-1 issued before the walk,
    row it+SA issued after the barrier of iteration it; iteration it waits
    for row it+4 before its barrier; the prologue reads rows 0..3, iteration
    it reads rows it+1..it+4 (edge lanes) and it+3, it+4 (main threads);
  * stage-A output ring (SY slots, written by the CTA): row q written at
    iteration q; stage B's prologue (iteration LAG-1) reads rows 0..3 and
    iteration it >= LAG reads rows it-3..it-1;
  * F_A fifo (NF slots, per thread): row q written at iteration q and read
    at iteration q + 3 by the same thread;
  * epilogue rings (2 slots, TMA): stage A's row q issued at iteration q-1
    (row 0 before the walk) and read at q; stage B's row e issued at
    iteration e + LAG - 1 and read at e + LAG."""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1109_1027_gb300", "csrc", "stage2d_fused.cu")


def _const(name):
    with open(SRC) as f:
        m = re.search(r"constexpr int %s = (\d+);" % name, f.read())
    assert m, name
    return int(m.group(1))


SA, SY, NF, LAG = _const("SA"), _const("SY"), _const("NF"), _const("LAG")


class Ring:
    """Slots of one ring: which row each holds and when it became readable
    (the iteration whose top barrier orders the write before later reads)."""

    def __init__(self, name, nslots):
        self.name, self.n = name, nslots
        self.row = [None] * nslots
        self.ready = [None] * nslots        # first iteration at which the row may be read
        self.pending = {}                   # row -> last iteration that will read it

    def put(self, row, it, ready_at):
        s = row % self.n
        old = self.row[s]
        if old is not None:
            last = self.pending.get(old, -1)
            # the slot is overwritten at iteration `it` (after its barrier):
            # every read of the old row must have happened before iteration it
            assert last < it, f"{self.name}: row {old} still read at {last}, overwritten by row {row} at {it}"
        self.row[s] = row
        self.ready[s] = ready_at

    def read(self, row, it):
        s = row % self.n
        assert self.row[s] == row, f"{self.name}: iteration {it} reads row {row}, slot holds {self.row[s]}"
        assert self.ready[s] is not None and self.ready[s] <= it, \
            f"{self.name}: row {row} read at {it} before it is ordered ({self.ready[s]})"


def _replay(nrows):
    nA, mA = nrows + 4, nrows + 8
    nit = nA + LAG - 1
    # planned reads (iteration by row), to check overwrites against
    reads_in, reads_y, reads_f = {}, {}, {}

    def plan(d, row, it):
        d[row] = max(d.get(row, -1), it)

    for m in range(4):
        plan(reads_in, m, -1)                               # prologue
    for it in range(nA):
        for m in range(it + 1, it + 5):
            plan(reads_in, m, it)
    for q in range(4):
        plan(reads_y, q, LAG - 1)
    for it in range(LAG, nrows + LAG):
        for q in range(it - 3, it):
            plan(reads_y, q, it)
    for q in range(nA):
        plan(reads_f, q, q + 3)

    rin, ry, rf = Ring("input", SA), Ring("A output", SY), Ring("F_A fifo", NF)
    rin.pending, ry.pending, rf.pending = reads_in, reads_y, reads_f
    issued = set()
    waited_by = {}                                          # input row -> iteration whose barrier follows its wait
    nxt = 0
    for m in range(min(SA, mA)):
        rin.put(m, -1, ready_at=None)
        issued.add(m)
        nxt += 1
    for m in range(4):
        waited_by[m] = -1
        rin.ready[m % SA] = -1
    for m in range(4):
        rin.read(m, -1)
    for it in range(nit + 1):
        a_on = it < nA
        if a_on:
            m = it + 4
            assert m in issued, f"row {m} waited at {it} before it was issued"
            waited_by[m] = it
            rin.ready[m % SA] = it
        # after the barrier: producer issues
        if a_on and nxt < mA:
            rin.put(nxt, it, ready_at=None)
            issued.add(nxt)
            nxt += 1
        if a_on:
            for m in range(it + 1, it + 5):
                rin.read(m, it)
            ry.put(it, it, ready_at=it + 1)
            rf.put(it, it, ready_at=it)                     # same thread: program order
        if it == LAG - 1:
            for q in range(4):
                ry.read(q, it)
        elif LAG <= it < nrows + LAG:
            for q in range(it - 3, it):
                ry.read(q, it)
            rf.read(it - 3, it)
    assert nxt == mA, "every input row is issued"
    assert all(waited_by.get(m) is not None for m in range(mA)), "every input row is waited for"


@pytest.mark.parametrize("nrows", list(range(1, 81)) + [128, 255])
def test_fused_pipeline_has_no_slot_conflicts(nrows):
    _replay(nrows)


def test_the_model_catches_a_ring_too_small():
    """The model is not vacuous: with one slot fewer in the output ring the
    stage-B prologue would read a row that stage A has already overwritten."""
    global SY
    saved = SY
    try:
        SY = saved - 1
        with pytest.raises(AssertionError):
            _replay(20)
    finally:
        SY = saved

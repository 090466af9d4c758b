"""A CPU model of the strided sweeps' TMA schedule (TmaColumnIO in
gp_sweep_tma.cuh driven by solve_segment in gp_sweep.cuh): which box each
read takes, when boxes are issued and waited, and which ring slot a box
occupies.  It follows the solve's calls (start, need, val, vals, put) for one
segment of one line and checks, for every chunk length B, window W, line
length and segment cut the kernels accept:
  - every read hits a box that was waited for and still sits in its slot
    (a slot is refilled only with the box two past the newest one read);
  - a box's node coordinate is never below -1 (node 0, read as the TMA
    fill) and no read passes the segment's copy limit;
  - every interior position of the line is written exactly once over all
    segments, and nothing outside [0, n).
This checks the schedule, not the kernel: the GPU parity tests check that."""
import pytest

RC = 4  # kRingChunks


class IO:
    def __init__(self, B, n, tb, te, writes):
        self.B, self.n, self.tb, self.te = B, n, tb, te
        self.writes = writes
        self.slot = [None] * RC

    def issue(self):
        b = self.issued
        y = self.s0 + b * self.B
        assert y >= -1
        self.slot[b % RC] = b
        self.issued += 1

    def start(self, first, lim):
        self.s0, self.limit, self.issued, self.ready = first, lim, 0, 0
        while self.issued < RC - 1 and self.s0 + self.issued * self.B < self.limit:
            self.issue()

    def need(self, p_end):
        c = (p_end - 1 - self.s0) // self.B
        assert p_end - 1 - self.s0 >= 0
        if c < self.ready:
            return
        assert self.issued > c, "need of a box the pattern has not issued"
        while self.issued <= c:
            self.issue()
        self.ready = c + 1
        while self.issued <= c + RC - 2 and self.s0 + self.issued * self.B < self.limit:
            self.issue()

    def read(self, p):
        b = (p - self.s0) // self.B
        assert 0 <= b < self.ready, ("read of a box not waited for", p, b, self.ready)
        assert self.slot[b % RC] == b, ("read of a refilled slot", p, b)
        assert p < self.limit

    def put(self, t0, q):
        p = t0 + q
        assert self.tb <= p < self.te
        self.writes[p] = self.writes.get(p, 0) + 1

    def flush(self, t0, count):
        assert 0 <= count


def solve_segment(io, n, tb, te, B, W):
    """The position pattern of solve_segment (and window_chunk)."""
    tw = tb - (W + 1) if tb > W + 1 else 0
    e = min(te + W, n)
    io.start(tw - 1, e + 2)
    io.need(tw + 2)
    for p in (tw - 1, tw, tw + 1):
        io.read(p)
    for t in range(tw, tb):
        io.need(t + 3)
        io.read(t + 2)
    m = e - tb
    for q in range(W):
        if q < m:
            io.need(tb + q + 3)
            io.read(tb + q + 2)
    t0 = tb
    while t0 + B + W <= e:
        io.need(t0 + W + 2 + B)
        for q in range(B):
            io.read(t0 + W + 2 + q)
        for q in range(B - 1, -1, -1):
            io.put(t0, q)
        io.flush(t0, B)
        t0 += B
    rem = e - t0
    assert 0 <= rem < B + W
    io.need(e + 2)
    for q in range(W, B + W):
        if q < rem:
            io.read(t0 + q + 2)
    for q in range(B + W - 1, -1, -1):
        if q < rem and t0 + q < te:
            io.put(t0, q)
    io.flush(t0, min(rem, te - t0))


def segment_cut(n, B, override):
    """choose_segments for a strided axis."""
    if override > 0:
        length = min(n, override)
    else:
        want = max(1, (n + 127) // 128)
        length = (n + want - 1) // want
        length = min((length + B - 1) // B * B, n)
    length = max(1, length)
    return length, (n + length - 1) // length


@pytest.mark.parametrize("B", [8, 16])
@pytest.mark.parametrize("W", [4, 8, 16])
@pytest.mark.parametrize("override", [0, 5, 13, 24, 40])
def test_line_tma_schedule(B, W, override):
    for n in list(range(1, 70)) + [127, 128, 129, 200, 255, 256, 257, 318, 398, 478]:
        seg_len, n_seg = segment_cut(n, B, override)
        writes = {}
        for s in range(n_seg):
            tb = s * seg_len
            te = n if s == n_seg - 1 else tb + seg_len
            solve_segment(IO(B, n, tb, te, writes), n, tb, te, B, W)
        assert sorted(writes) == list(range(n)), (n, seg_len)
        assert all(v == 1 for v in writes.values()), (n, seg_len)

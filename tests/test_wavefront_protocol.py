"""The GPU wavefront's progress protocol is serialisable (Section III-A).

Host model of the bulge kernel's waits: a row-bulge (R, s) of a stage (bw, d)
runs three segments,
  1. loads, right reflector, row updates            -> publishes 2s+1 ("half")
  2. left reflector on the columns loaded up front
  3. the left panel's tail columns (after a second wait) -> publishes 2s+2
and sweep R waits only on sweep R-1's progress word: before segment 1 for
`pre_target(s)`, before segment 3 for `tail_target(s)`.  This test takes the
element footprint of every segment straight from the geometry of the chase,
derives what each segment is guaranteed to follow (waits compose through the
earlier sweeps' own waits), and checks that every pair of segments of
different sweeps that touch a common element runs in sweep order -- the
order of the sequential oracle.  It also checks that weakening a wait breaks
this, so the model is not vacuous.
"""
import itertools

import pytest


def sweep_steps(n, bw, d, R):
    bwp = bw - d
    s = 0
    while R + bwp + s * bw < n - 1:
        s += 1
    return s


def geometry(n, bw, d, R, s, tail_start):
    c = R + (bw - d) + s * bw
    m = min(d + 1, n - c)
    r0 = R if s == 0 else c - bw
    jmax = min(n - 1, c + m - 1 + bw)
    ncols = jmax - c
    pre_hi = min(tail_start, ncols + 1)
    right = {(i, j) for i in range(r0, c + m) for j in range(c, c + m)}
    left_pre = {(i, c + jj) for i in range(c, c + m) for jj in range(0, pre_hi)}
    tail = {(i, c + jj) for i in range(c, c + m) for jj in range(pre_hi, ncols + 1)}
    seg1 = right | {(i, c + jj) for i in range(c, c + m) for jj in range(m, pre_hi)}
    seg2 = left_pre | {(i, j) for (i, j) in right if i >= c}
    return [seg1, seg2, tail]


class Protocol:
    """Wait targets of the kernel (progress values of sweep R-1, relative to
    the stage base), and the left-panel offset where the tail starts."""

    def __init__(self, kind="kernel"):
        self.kind = kind
        self.final_wait = kind != "no_final_wait"

    def targets(self, n, bw, d, R, s):
        nsp = sweep_steps(n, bw, d, R - 1) if R > 0 else 0
        split = bw - d >= 2
        if split:
            pre = 2 * min(s + 1, nsp)
            tail = 2 * (s + 1) + (1 if bw - d >= 3 else 2) if s + 1 < nsp else 2 * nsp
            tail_start = bw - 1
            if self.kind == "weak_tail":
                tail = 2 * min(s + 1, nsp)
            if self.kind == "weak_tail_bw2" and bw - d == 2 and s + 1 < nsp:
                tail = 2 * (s + 1) + 1
        else:
            pre = 2 * min(s + 2, nsp)
            tail = 2 * (s + 2) + 1 if s + 2 < nsp else 2 * nsp
            tail_start = d + bw
            if self.kind == "lag2_no_tail":
                tail, tail_start = 0, 1 << 30
        return pre, tail, tail_start


def check(n, b, tw, proto):
    bw = b
    while bw > 1:
        d = min(tw, bw - 1)
        check_stage(n, bw, d, proto)
        bw -= d


def check_stage(n, bw, d, proto):
    nsweeps = n - 1
    steps = [sweep_steps(n, bw, d, R) for R in range(nsweeps)]
    # know[R][(s, seg)] = per earlier sweep R', the progress value of R' known
    # complete when segment seg of (R, s) starts
    know = {}
    pub = {}   # (R, value) -> knowledge vector at the time R published value
    segs = {}
    for R in range(nsweeps):
        k = {}
        for s in range(steps[R]):
            pre, tail, tail_start = proto.targets(n, bw, d, R, s)
            segs[(R, s)] = geometry(n, bw, d, R, s, tail_start)
            if R > 0:
                k = merge(k, wait_knowledge(pub, R - 1, pre))
            know[(R, s, 0)] = dict(k)
            know[(R, s, 1)] = dict(k)
            pub[(R, 2 * s + 1)] = dict(k)
            has_tail = bool(segs[(R, s)][2])
            if R > 0 and has_tail:
                k = merge(k, wait_knowledge(pub, R - 1, tail))
            know[(R, s, 2)] = dict(k)
            if R > 0 and s == steps[R] - 1 and proto.final_wait:
                # a sweep publishes its completion only once its predecessor is
                # complete, so completion passes the whole chain on
                k = merge(k, wait_knowledge(pub, R - 1, 2 * steps[R - 1]))
            pub[(R, 2 * s + 2)] = dict(k)
        if steps[R] == 0:
            pub[(R, 0)] = dict(k)
    # every conflicting pair of segments of sweeps R1 < R2 must be ordered
    owners = {}
    for (R, s), sg in segs.items():
        for g, elems in enumerate(sg):
            for e in elems:
                owners.setdefault(e, []).append((R, s, g))
    for e, lst in owners.items():
        for (R1, s1, g1), (R2, s2, g2) in itertools.combinations(sorted(lst), 2):
            if R1 == R2:
                continue
            need = 2 * s1 + (1 if g1 == 0 else 2)
            got = know[(R2, s2, g2)].get(R1, 0)
            assert got >= need, (n, bw, d, e, (R1, s1, g1), (R2, s2, g2), got, need)


def wait_knowledge(pub, Rp, value):
    """Waiting for sweep Rp's progress >= value teaches Rp's state then."""
    # the smallest published value >= `value` carries the knowledge (values
    # are published in increasing order; waiting for v means seeing some v' >= v,
    # and the guarantee is the one of v itself)
    k = {Rp: value}
    best = None
    for (R, v), kn in pub.items():
        if R == Rp and v >= value and (best is None or v < best[0]):
            best = (v, kn)
    if best is not None:
        k = merge(k, best[1])
    return k


def merge(a, b):
    out = dict(a)
    for key, v in b.items():
        out[key] = max(out.get(key, 0), v)
    return out


CASES = [(n, b, tw) for n in (24, 37, 50) for (b, tw) in
         ((2, 1), (3, 2), (4, 3), (5, 2), (6, 4), (8, 3), (9, 8), (12, 5), (16, 15), (7, 6))]


@pytest.mark.parametrize("n,b,tw", CASES)
def test_kernel_protocol_is_serialisable(n, b, tw):
    check(n, b, tw, Protocol("kernel"))


@pytest.mark.parametrize("kind,b,tw", [("weak_tail", 8, 3), ("weak_tail_bw2", 6, 4),
                                       ("no_final_wait", 5, 2),
                                       ("lag2_no_tail", 5, 4), ("lag2_no_tail", 9, 8)])
def test_weakened_waits_are_caught(kind, b, tw):
    with pytest.raises(AssertionError):
        check(40, b, tw, Protocol(kind))

"""Host model of the group kernel's schedule (one CTA chases K consecutive
sweeps of a stage through a shared-memory window, Section III-A dependency
distance).

Per group g (sweeps R0 = gK .. R0+K-1) and step s, with c = R0 + bw' + s bw:
  W1   wait: group g-1 completed step s
  LD1  load the window except the carried block and the tail columns
  U    right reflectors of every member, applied to the rows above c
  Ln   per member: right reflector on the rows >= c, left reflector on the
       near columns c .. c+K+d-1 (the near warps; runs alongside ST1 .. LD2)
  ST1  store the rows above c;               publish "step s upper done"
  W2   wait: group g-1 did the upper part of step s+1 (or finished)
  LD2  load the tail columns and the next step's carried block
  Lf   per member: left reflector on the far columns >= c+K+d
  ST2  store everything but the carried block; publish "step s complete"
(the last step stores the carried block too and publishes only once group
g-1 has finished).  Ln is placed before ST1 here; in the kernel it overlaps
ST1, W2 and LD2, which touch none of its cells (checked below: its cells are
resident after LD1 and no other group reaches them before "step s complete").

The model checks, for every stage of small matrices:
  * cross-group: every pair of operations of different groups that touch a
    common element is ordered as in the sequential oracle by the waits;
  * within a group: every pair ordered differently from the sequential
    oracle is a right reflector and a left reflector whose common block holds
    neither one's generating vector and is transformed whole by both, so the
    two commute (equal in exact arithmetic);
  * the window: every element an operation touches is in shared memory at
    that moment, every modified element is written back, and no other group
    touches an element between our load and our store of it;
and it replays the schedule numerically against the oracle.  Weakened
variants of the protocol must fail the checks.
"""
import itertools

import numpy as np
import pytest

import bandgen
import oracle


def sweep_steps(n, bw, d, R):
    c0 = R + bw - d
    return 0 if c0 >= n - 1 else (n - 2 - c0) // bw + 1


def group_size(bw, d, K):
    """Members per group on this stage (0: the stage needs the per-sweep
    kernel).  3K + d <= bw keeps group g-2's step s+2 out of group g's
    window at step s (nothing orders the two), which also gives 2K + d < bw
    for the tail columns and K <= bw - d for the first step's bulge rows."""
    return max(0, min(K, (bw - d) // 3))


class Model:
    def __init__(self, n, bw, d, K, variant="kernel"):
        self.n, self.bw, self.d, self.K, self.variant = n, bw, d, K, variant
        self.bwp = bw - d
        nact = max(0, n - 1 - self.bwp)
        self.G = (nact + K - 1) // K
        self.nact = nact

    # ------------------------------------------------------------ geometry
    def members(self, g):
        R0 = g * self.K
        return R0, min(self.K, self.nact - R0)

    def steps(self, g):
        R0, _ = self.members(g)
        return sweep_steps(self.n, self.bw, self.d, R0)

    def origin(self, g, s):
        return g * self.K + self.bwp + s * self.bw

    def clip(self, cells):
        n = self.n
        return {(i, j) for (i, j) in cells if 0 <= i < n and 0 <= j < n}

    def regions(self, g, s):
        """Window regions of group g, step s, in matrix coordinates."""
        K, d, bw, bwp = self.K, self.d, self.bw, self.bwp
        c = self.origin(g, s)
        Kp = K if g > 0 else 0
        top = (lambda X: max(0, X - d) - (bwp if s == 0 else bw))
        V = {(c + I, c + X) for X in range(K + d) for I in range(top(X), min(K - 1, X) + d + 1)}
        carried_in = set()
        if s > 0:
            carried_in = {(c + I, c + X) for X in range(K + d)
                          for I in range(top(X), top(X) + K + d) if I < -bw + K + d}
        Vup = {(i, j) for (i, j) in V if i < c}
        Vlo = V - Vup
        Hn = {(c + I, c + X) for X in range(K + d, bw - Kp) for I in range(0, K + d)}
        lo2 = bw - Kp if self.variant != "tail_late_only" else bw
        L2 = {(c + I, c + X) for X in range(lo2, bw + K + d)
              for I in range(max(0, X - d - bw), K + d)}
        Ht = {(c + I, c + X) for X in range(K + d, bw) for I in range(0, K + d)} - Hn
        carried_out = {(c + I, c + X) for X in range(bw, bw + K + d)
                       for I in range(max(0, X - d - bw), K + d)}
        ld1 = self.clip((V - carried_in) | Hn)
        if self.variant == "tail_late_only":
            ld1 |= self.clip(Ht)
        return dict(c=c, V=self.clip(V), Vup=self.clip(Vup), Vlo=self.clip(Vlo),
                    carried_in=self.clip(carried_in), ld1=ld1, ld2=self.clip(L2),
                    st1=self.clip(Vup), st2=self.clip(Vlo | Hn | Ht),
                    carried_out=self.clip(carried_out))

    def ops(self, g, s):
        """Operations of group g at step s in program order: (phase, kind, R,
        rows, cols, gen-cells, footprint) with the right reflectors split into
        gen, upper and lower parts (one reflector id per (R, s, side))."""
        n, bw, d, bwp = self.n, self.bw, self.d, self.bwp
        R0, kk = self.members(g)
        c = self.origin(g, s)
        act = [j for j in range(kk) if s < sweep_steps(n, bw, d, R0 + j)]
        # near columns: c .. c+K+d-1 (the "near_wide" variant wrongly takes the
        # tail columns too, before the wait that protects them)
        xnear = c + self.K + d if self.variant != "near_wide" else c + bw + self.K + d
        U, L, F = [], [], []
        for j in act:
            cj = c + j
            m = min(d + 1, n - cj)
            r0 = R0 + j if s == 0 else cj - bw
            cols = range(cj, cj + m)
            gen = {(r0, x) for x in cols}
            rid = (R0 + j, s, "R")
            full = {(i, x) for i in range(r0, cj + m) for x in cols}
            U.append(("U", "R", rid, gen, gen))
            up = {(i, x) for i in range(r0 + 1, min(c, cj + m)) for x in cols}
            U.append(("U", "R", rid, gen, up))
            lo = {(i, x) for i in range(max(c, r0 + 1), cj + m) for x in cols}
            L.append(("L", "R", rid, gen, lo))
            jmax = min(n - 1, cj + m - 1 + bw)
            lid = (R0 + j, s, "L")
            lgen = {(i, cj) for i in range(cj, cj + m)}
            lfull = {(i, x) for i in range(cj, cj + m) for x in range(cj, jmax + 1)}
            L.append(("L", "L", lid, lgen, {(i, x) for (i, x) in lfull if x < xnear}))
            far = {(i, x) for (i, x) in lfull if x >= xnear}
            if far:
                F.append(("F", "L", lid, lgen, far))
            self.full[rid] = full
            self.full[lid] = lfull
            self.gen[rid] = gen
            self.gen[lid] = lgen
        return U + L + F

    # ------------------------------------------------------------ schedule
    def run(self):
        """Knowledge-vector execution of every group's program."""
        self.full, self.gen = {}, {}
        self.events = []          # (g, index, kind, payload, knowledge)
        pub = {}                  # (g, value) -> knowledge when published
        for g in range(self.G):
            S = self.steps(g)
            Sp = self.steps(g - 1) if g > 0 else 0
            know = {}

            def wait(value):
                nonlocal know
                if g == 0:
                    return
                best = None
                for (gg, v), kn in pub.items():
                    if gg == g - 1 and v >= value and (best is None or v < best[0]):
                        best = (v, kn)
                assert best is not None, ("wait never satisfied", g, value)
                know = merge(know, best[1])
                know = merge(know, {g - 1: value})

            def publish(v):
                pub[(g, v)] = merge(know, {g: v})
                self.events.append((g, "PUB", v, dict(know)))

            for s in range(S):
                reg = self.regions(g, s)
                w1 = 2 * (s + 1)
                if self.variant == "weak_w1" and s > 0:
                    w1 = 2 * s + 1
                wait(w1)
                self.events.append((g, "LD", (s, "ld1", reg["ld1"]), dict(know)))
                ops = self.ops(g, s)
                for phase in ("U", "L"):
                    for op in ops:
                        if op[0] == phase:
                            self.events.append((g, "OP", (s,) + op, dict(know)))
                self.events.append((g, "ST", (s, "st1", reg["st1"]), dict(know)))
                publish(2 * s + 1)
                if self.variant != "no_w2":
                    wait(2 * (s + 1) + 1 if s + 1 < Sp else 2 * Sp)
                self.events.append((g, "LD", (s, "ld2", reg["ld2"]), dict(know)))
                for op in ops:
                    if op[0] == "F":
                        self.events.append((g, "OP", (s,) + op, dict(know)))
                st2 = set(reg["st2"])
                if s == S - 1:
                    st2 |= reg["carried_out"]
                self.events.append((g, "ST", (s, "st2", st2), dict(know)))
                if s == S - 1 and g > 0 and self.variant != "no_final_wait":
                    wait(2 * Sp)
                publish(2 * (s + 1))
        self.pub = pub

    # -------------------------------------------------------------- checks
    def next_pub(self, g, idx):
        """Knowledge value of group g published after its event idx."""
        for e in self.events[idx:]:
            if e[0] == g and e[1] == "PUB":
                return e[2]
        return None

    def check(self):
        self.run()
        ev = self.events
        # index events per group in program order
        per = {}
        for k, e in enumerate(ev):
            per.setdefault(e[0], []).append(k)
        seq_key = lambda rid: (rid[0], rid[1], 0 if rid[2] == "R" else 1)
        opsl = [(k, e) for k, e in enumerate(ev) if e[1] == "OP"]
        cells = {}
        for k, e in opsl:
            for cell in e[2][5]:
                cells.setdefault(cell, []).append(k)
        # pairwise order of conflicting parts
        for cell, ks in cells.items():
            for k1, k2 in itertools.combinations(ks, 2):
                e1, e2 = ev[k1], ev[k2]
                rid1, rid2 = e1[2][3], e2[2][3]
                if rid1 == rid2:
                    continue
                g1, g2 = e1[0], e2[0]
                if g1 != g2:
                    # the op of the smaller group must happen before the other
                    (ka, ea), (kb, eb) = ((k1, e1), (k2, e2)) if g1 < g2 else ((k2, e2), (k1, e1))
                    v = self.next_pub(ea[0], ka)
                    assert v is not None and eb[3].get(ea[0], -1) >= v, \
                        ("cross-group order", cell, ea[2][:4], eb[2][:4])
                    continue
                # same group: program order k1 < k2
                if seq_key(rid1) <= seq_key(rid2):
                    continue
                assert self.commutes(rid1, rid2, e1, e2), ("reordered", cell, rid1, rid2)
        self.check_window()

    def commutes(self, rid_a, rid_b, ea, eb):
        # one right and one left reflector; common block misses both
        # generating vectors and each transforms the whole block
        kinds = {rid_a[2], rid_b[2]}
        if kinds != {"R", "L"}:
            return False
        r, l = (rid_a, rid_b) if rid_a[2] == "R" else (rid_b, rid_a)
        fr, fl = self.full[r], self.full[l]
        common = fr & fl
        if common & self.gen[r] or common & self.gen[l]:
            return False
        rows_r = {i for (i, _) in fr}
        cols_r = {j for (_, j) in fr}
        rows_l = {i for (i, _) in fl}
        cols_l = {j for (_, j) in fl}
        if not (rows_l <= rows_r and cols_r <= cols_l):
            return False
        # the left reflector is not applied between two parts of the right one
        parts = [k for k, e in enumerate(self.events) if e[1] == "OP" and e[2][3] == r]
        lpos = [k for k, e in enumerate(self.events) if e[1] == "OP" and e[2][3] == l]
        return all(k < min(parts) or k > max(parts) for k in lpos)

    def check_window(self):
        ev = self.events
        # residency: per group, the set of cells in shared memory over time
        owner_ops = {}
        for k, e in enumerate(ev):
            if e[1] == "OP":
                for cell in e[2][5]:
                    owner_ops.setdefault(cell, []).append(k)
        for g in range(self.G):
            resident = {}
            dirty = set()
            for k, e in enumerate(ev):
                if e[0] != g:
                    continue
                if e[1] == "LD":
                    for cell in e[2][2]:
                        assert cell not in resident, ("loaded twice", g, cell)
                        resident[cell] = k
                elif e[1] == "OP":
                    for cell in e[2][5]:
                        assert cell in resident, ("not resident", g, e[2][:4], cell)
                        dirty.add(cell)
                elif e[1] == "ST":
                    for cell in e[2][2]:
                        assert cell in resident, ("store of a cell not loaded", g, cell)
                        kl = resident.pop(cell)
                        dirty.discard(cell)
                        # no other group touches the cell between load and store
                        for ko in owner_ops.get(cell, []):
                            go = ev[ko][0]
                            if go == g:
                                continue
                            if go < g:
                                v = self.next_pub(go, ko)
                                assert v is not None and ev[kl][3].get(go, -1) >= v, \
                                    ("predecessor touches window", g, cell, ev[ko][2][:4])
                            else:
                                v = self.next_pub(g, k)
                                assert ev[ko][3].get(g, -1) >= v, \
                                    ("successor touches window", g, cell, ev[ko][2][:4])
            assert not dirty, ("modified, never stored", g, sorted(dirty)[:5])
            assert not resident, ("loaded, never stored", g, sorted(resident)[:5])


def merge(a, b):
    out = dict(a)
    for key, v in b.items():
        out[key] = max(out.get(key, -1), v)
    return out


def stages(b, tw):
    bw = b
    while bw > 1:
        d = min(tw, bw - 1)
        yield bw, d
        bw -= d


CASES = [(n, b, tw, K) for (n, b, tw, K) in [
    (40, 12, 3, 2), (47, 12, 3, 4), (60, 16, 4, 3), (53, 20, 5, 2), (64, 24, 8, 4),
    (70, 18, 2, 5), (45, 9, 2, 2), (90, 30, 10, 6), (33, 14, 4, 1), (61, 40, 16, 3)]]


@pytest.mark.parametrize("n,b,tw,K", CASES)
def test_group_protocol(n, b, tw, K):
    checked = 0
    for bw, d in stages(b, tw):
        k = group_size(bw, d, K)
        if k == 0:
            continue
        Model(n, bw, d, k).check()
        checked += 1
    assert checked > 0


@pytest.mark.parametrize("variant", ["weak_w1", "no_w2", "no_final_wait", "tail_late_only", "near_wide"])
def test_weakened_group_protocol_is_caught(variant):
    with pytest.raises(AssertionError):
        for (n, b, tw, K) in [(40, 12, 3, 2), (60, 16, 4, 3), (64, 24, 8, 4)]:
            for bw, d in stages(b, tw):
                k = group_size(bw, d, K)
                if k:
                    Model(n, bw, d, k, variant).check()


def test_group_size_limits():
    # 3K + d <= bw, and the final stage (bw' = 1) is never grouped
    assert group_size(128, 32, 64) == 32
    assert group_size(64, 32, 64) == 10
    assert group_size(32, 31, 8) == 0
    assert group_size(35, 32, 8) == 1
    assert group_size(34, 32, 8) == 0


# ----------------------------------------------------------- numeric replay

def _larfg(x):
    """Householder vector with the LAPACK larfg contract (test model only)."""
    alpha = x[0]
    xi = np.linalg.norm(x[1:])
    if xi == 0.0:
        return 0.0, np.concatenate(([1.0], np.zeros(len(x) - 1))), alpha
    beta = -np.copysign(np.hypot(alpha, xi), alpha if alpha != 0 else 1.0)
    tau = (beta - alpha) / beta
    v = np.concatenate(([1.0], x[1:] / (alpha - beta)))
    return tau, v, beta


def replay(a, b, tw, K):
    """The group kernel's order on a dense matrix: groups one after another
    (a linearisation the waits allow), each step-major with the U / L split."""
    a = a.copy()
    n = a.shape[0]
    for bw, d in stages(min(b, n - 1), tw):
        k = group_size(bw, d, K)
        bwp = bw - d
        if k == 0:       # per-sweep order
            groups = [[R] for R in range(n - 1)]
        else:
            nact = max(0, n - 1 - bwp)
            groups = [list(range(g, min(g + k, nact))) for g in range(0, nact, k)]
        for mem in groups:
            S = sweep_steps(n, bw, d, mem[0])
            for s in range(S):
                c = mem[0] + bwp + s * bw
                act = [R for R in mem if s < sweep_steps(n, bw, d, R)]
                refl = {}
                for R in act:                                  # phase U
                    cj = R + bwp + s * bw
                    m = min(d + 1, n - cj)
                    r0 = R if s == 0 else cj - bw
                    tau, v, beta = _larfg(a[r0, cj:cj + m])
                    a[r0, cj:cj + m] = 0.0
                    a[r0, cj] = beta
                    rows = slice(r0 + 1, min(c, cj + m))
                    a[rows, cj:cj + m] -= tau * np.outer(a[rows, cj:cj + m] @ v, v)
                    refl[R] = (tau, v, r0)
                for R in act:                                  # phase L
                    cj = R + bwp + s * bw
                    m = min(d + 1, n - cj)
                    tau, v, r0 = refl[R]
                    rows = slice(max(c, r0 + 1), cj + m)
                    a[rows, cj:cj + m] -= tau * np.outer(a[rows, cj:cj + m] @ v, v)
                    tau, v, beta = _larfg(a[cj:cj + m, cj])
                    a[cj:cj + m, cj] = 0.0
                    a[cj, cj] = beta
                    jmax = min(n - 1, cj + m - 1 + bw)
                    cols = slice(cj + 1, jmax + 1)
                    a[cj:cj + m, cols] -= tau * np.outer(v, v @ a[cj:cj + m, cols])
    return np.diag(a).copy(), np.diag(a, 1).copy(), a


@pytest.mark.parametrize("n,b,tw,K", [(70, 20, 5, 3), (64, 24, 8, 4), (90, 30, 10, 6), (50, 12, 3, 2)])
def test_group_order_matches_oracle(n, b, tw, K):
    ab = bandgen.random_band(n, b, seed=n + b)
    d0, e0, _ = oracle.band_to_bidiag(ab, b, tw)
    d, e, a = replay(bandgen.dense_from_band(ab, b), b, tw, K)
    # bidiagonal: everything else exactly zero
    assert np.count_nonzero(np.triu(a, 2)) == 0 and np.count_nonzero(np.tril(a, -1)) == 0
    scale = np.max(np.abs(d0))
    assert np.max(np.abs(np.abs(d) - np.abs(d0))) <= 1e-12 * scale
    assert np.max(np.abs(np.abs(e) - np.abs(e0))) <= 1e-12 * scale


def test_group_size_limit_is_needed():
    # one member more than 3K + d <= bw allows breaks the checks
    with pytest.raises(AssertionError):
        Model(47, 12, 3, 4).check()

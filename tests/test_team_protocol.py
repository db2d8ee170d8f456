"""Host model of the team kernel: the last bandwidth-reduction stage
(bw -> 1, Section III-A dependency distance of three row-bulges), W sweeps per
CTA side by side on a circular shared-memory band window, an IO warp that
owns the columns.

The model replays the kernel's actions, each atomic, in random orders that
respect exactly the kernel's waits, with several groups (CTAs) at once:
  team j, step s, right half:  j > 0: team j-1 completed step s+1;
                               j = 0: the right panel's columns are loaded
  team j, step s, left half:   j = 0: its columns are loaded; j > 0: team j-1
                               applied the right reflector of step s+2; on the
                               last step team j-1 is complete
  IO store:  columns left of every team's next row-bulge -> band, publish
  IO load:   columns the previous group released, into free slots
The window addressing is the kernel's (slot x mod C, band offset + 2bw - 1).
The stage starts from the oracle's band after the earlier stages and ends
where the oracle ends; the model's d and e must match the oracle's to
rounding, for every seed.  A variant with the release point of the first
version (the last team only) must fail.
"""
import random

import numpy as np
import pytest

import bandgen
import oracle


def sweep_steps(n, bw, d, R):
    c0 = R + bw - d
    return 0 if c0 >= n - 1 else (n - 2 - c0) // bw + 1


def _larfg(x):
    alpha = x[0]
    xi = np.linalg.norm(x[1:])
    if xi == 0.0:
        v = np.zeros(len(x))
        v[0] = 1.0
        return 0.0, v, alpha
    beta = -np.copysign(np.hypot(alpha, xi), alpha if alpha != 0 else 1.0)
    return (beta - alpha) / beta, np.concatenate(([1.0], x[1:] / (alpha - beta))), beta


class Stage:
    def __init__(self, work, n, bw, top, W, rng, variant="kernel"):
        self.band = work          # (n, ld): element (i, x) at band[x, i - x + top]
        self.n, self.bw, self.d, self.top, self.W = n, bw, bw - 1, top, W
        self.P = 3 * bw - 1 + ((3 * bw - 1) & 1)
        self.C = (2 * W + 3) * bw
        self.rng, self.variant = rng, variant
        nact = n - 2
        self.G = (nact + W - 1) // W if nact > 0 else 0
        self.pub = [-1] * self.G          # first column not released (-1: none yet)
        self.groups = [self._group(g) for g in range(self.G)]

    def _group(self, g):
        n, bw, d, W = self.n, self.bw, self.d, self.W
        R0 = g * W
        kk = min(W, n - 2 - R0)
        return dict(g=g, R0=R0, kk=kk, win=np.full(self.C * self.P, np.nan),
                    tprog=[0] * kk, ld=R0 + 1, st=R0 + 1,
                    step=[0] * kk, half=[0] * kk,
                    ns=[sweep_steps(n, bw, d, R0 + j) for j in range(kk)])

    # window address of element (i, x)
    def at(self, x, i):
        return (x % self.C) * self.P + (i - x + 2 * self.bw - 1)

    def geom(self, R, s):
        c = R + 1 + s * self.bw
        m = min(self.d + 1, self.n - c)
        r0 = R if s == 0 else c - self.bw
        jmax = min(self.n - 1, c + m - 1 + self.bw)
        return c, m, r0, jmax

    # ----------------------------------------------------------- actions
    def team_ready(self, G, j):
        s, h = G["step"][j], G["half"][j]
        if s >= G["ns"][j]:
            return False
        c, m, r0, jmax = self.geom(G["R0"] + j, s)
        nsp = G["ns"][j - 1] if j > 0 else 0
        if h == 0:
            if j == 0:
                return G["ld"] >= c + m
            return G["tprog"][j - 1] >= 2 * min(s + 2, nsp)
        if j == 0:
            return G["ld"] >= jmax + 1
        ok = True
        if c + self.d + self.bw <= jmax:
            ok = G["tprog"][j - 1] >= (2 * (s + 2) + 1 if s + 2 < nsp else 2 * nsp)
        if s == G["ns"][j] - 1:
            ok = ok and G["tprog"][j - 1] >= 2 * nsp
        return ok

    def team_act(self, G, j):
        s, h = G["step"][j], G["half"][j]
        R = G["R0"] + j
        c, m, r0, jmax = self.geom(R, s)
        win, at = G["win"], self.at
        if h == 0:
            idx = [at(c + t, r0) for t in range(m)]
            tau, v, beta = _larfg(win[idx].copy())
            win[idx] = 0.0
            win[idx[0]] = beta
            for r in range(r0 + 1, c + m):
                ri = [at(c + t, r) for t in range(m)]
                w = win[ri] @ v
                win[ri] -= tau * w * v
            G["tprog"][j] = 2 * s + 1
            G["half"][j] = 1
        else:
            idx = [at(c, c + t) for t in range(m)]
            tau, v, beta = _larfg(win[idx].copy())
            win[idx] = 0.0
            win[idx[0]] = beta
            for x in range(c + 1, jmax + 1):
                ci = [at(x, c + t) for t in range(m)]
                w = v @ win[ci]
                win[ci] -= tau * w * v
            G["tprog"][j] = 2 * (s + 1)
            G["half"][j] = 0
            G["step"][j] = s + 1
        assert not np.isnan(win[idx]).any()

    def release_point(self, G):
        if self.variant == "last_team_only":
            j = G["kk"] - 1
            p = G["tprog"][j] >> 1
            return self.n if p >= G["ns"][j] else G["R0"] + j + 1 + p * self.bw
        rel = self.n
        for j in range(G["kk"]):
            p = G["tprog"][j] >> 1
            if p < G["ns"][j]:
                rel = min(rel, G["R0"] + j + 1 + p * self.bw)
        return rel

    def io_store_ready(self, G):
        return min(self.release_point(G), G["ld"]) > G["st"]

    def io_store(self, G):
        to = min(self.release_point(G), G["ld"])
        for x in range(G["st"], to):
            for o in range(3 * self.bw - 1):
                i = x + o - (2 * self.bw - 1)
                val = G["win"][(x % self.C) * self.P + o]
                if 0 <= i < self.n:
                    self.band[x, i - x + self.top] = val
        G["st"] = to
        self.pub[G["g"]] = to

    def avail(self, G):
        return self.n if G["g"] == 0 else self.pub[G["g"] - 1]

    def io_load_ready(self, G):
        to = min(self.avail(G), self.n, G["st"] + self.C, G["ld"] + self.bw)
        return to > G["ld"]

    def io_load(self, G):
        to = min(self.avail(G), self.n, G["st"] + self.C, G["ld"] + self.bw)
        for x in range(G["ld"], to):
            for o in range(3 * self.bw - 1):
                i = x + o - (2 * self.bw - 1)
                G["win"][(x % self.C) * self.P + o] = self.band[x, i - x + self.top] \
                    if 0 <= i < self.n else 0.0
        G["ld"] = to

    def run(self, max_active=3):
        """Random interleaving; at most max_active groups in flight (persistent
        CTAs), claimed in order."""
        next_g, active = 0, []
        while next_g < self.G or active:
            while len(active) < max_active and next_g < self.G:
                active.append(self.groups[next_g])
                next_g += 1
            acts = []
            for G in active:
                for j in range(G["kk"]):
                    if self.team_ready(G, j):
                        acts.append((self.team_act, G, j))
                if self.io_store_ready(G):
                    acts.append((self.io_store, G, None))
                if self.io_load_ready(G):
                    acts.append((self.io_load, G, None))
            assert acts, "deadlock"
            f, G, j = acts[self.rng.randrange(len(acts))]
            f(G, j) if j is not None else f(G)
            active = [G for G in active if G["st"] < self.n]


def _last_stage_input(n, b, tw, seed):
    ab = bandgen.random_band(n, b, seed=seed)
    bcl = min(b, n - 1)
    st = 0
    bw = bcl
    while bw - min(tw, bw - 1) > 1:
        bw -= min(tw, bw - 1)
        st += 1
    _, _, _, work = oracle.band_to_bidiag(ab, b, tw, max_stages=st, return_work=True)
    return ab, work, bw, bcl + tw


@pytest.mark.parametrize("n,b,tw,W,seed", [(60, 6, 5, 3, 1), (80, 9, 8, 4, 2), (45, 12, 4, 2, 3),
                                           (71, 5, 2, 5, 4), (50, 17, 16, 3, 5), (33, 3, 2, 4, 6),
                                           (90, 16, 8, 2, 7)])
def test_team_stage_matches_oracle(n, b, tw, W, seed):
    ab, work, bw, top = _last_stage_input(n, b, tw, seed)
    d0, e0, _ = oracle.band_to_bidiag(ab, b, tw)
    scale = max(np.max(np.abs(d0)), 1e-300)
    for trial in range(3):
        band = work.copy()
        Stage(band, n, bw, top, W, random.Random(100 * seed + trial)).run()
        d = np.array([band[i, top] for i in range(n)])
        e = np.array([band[i + 1, top - 1] for i in range(n - 1)])
        assert np.max(np.abs(np.abs(d) - np.abs(d0))) <= 1e-12 * scale
        assert np.max(np.abs(np.abs(e) - np.abs(e0))) <= 1e-12 * scale


def test_release_at_last_team_only_is_caught():
    # the first version released columns left of the last team's next
    # row-bulge; at a group's first step the earlier teams are further left
    n, b, tw, W = 60, 6, 5, 3
    ab, work, bw, top = _last_stage_input(n, b, tw, 1)
    d0, e0, _ = oracle.band_to_bidiag(ab, b, tw)
    band = work.copy()
    Stage(band, n, bw, top, W, random.Random(5), variant="last_team_only").run()
    d = np.array([band[i, top] for i in range(n)])
    assert not np.allclose(np.abs(d), np.abs(d0), rtol=0, atol=1e-10 * np.max(np.abs(d0)))

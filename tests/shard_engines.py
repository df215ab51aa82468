"""The oracle as the per-shard engine of the sharded protocol
(paper_1411_1702_gb300/shard.py), for CPU tests of the protocol.

Each shard is an oracle filter over its own slots whose random streams are
keyed by the global slot (or_config.slot0).  The cumulative weights use tiles
of one particle, so the gathered tile totals are the weights themselves and
their running sum is the oracle's own sequential c, bit for bit: a sharded run
must then resample exactly the parents a single oracle filter resamples.
Test infrastructure only.
"""
import math

import numpy as np

import oracle
from paper_1411_1702_gb300 import shard as SH


class OracleShard:
    tile = 1

    def __init__(self, w, n_all, first, n):
        self.o = oracle.Filter(w, N=n, slot0=first)
        self.o.shard_init()
        self.w, self.n_all, self.first, self.n = w, n_all, first, n
        R = 3 * w.d + w.p + 2
        self.info = dict(record=R, tiles=n, tiles_all=n_all, total=n_all, first=first)
        self.send = np.zeros(n_all * R)
        self.recv = np.zeros(n * R)
        self.pending = False      # Step 1's moments come first
        self.parents = None

    # Steps 2, 3a
    def stage1(self, t, y):
        self.t, self.y = t, np.asarray(y, dtype=np.float64)
        self.tab, self.S = self.o.substeps(t)
        assert self.o.stage1(self.tab, self.S, self.y) == oracle.OK
        wk = self.o.work()
        self.lg, self.ll1 = wk["lg"], wk["ll1"]
        fin = np.isfinite(self.lg)
        return float(np.max(self.lg[fin])) if fin.any() else -math.inf

    def scan(self, M):
        # g_k = exp(lg_k - M), with the C library's exp (math.exp), as the
        # oracle's own scan forms it
        g = np.array([math.exp(v - M) if math.isfinite(v) else 0.0 for v in self.lg])
        return g, float(g[-1])

    def offsets(self, tiles_all, cl_last):
        acc = 0.0
        c = np.empty(len(tiles_all))
        for k, v in enumerate(tiles_all):
            acc += float(v)
            c[k] = acc
        self.c_local = c[self.first:self.first + self.n]
        return c, float(c[-1]), self.o.resample_u()

    def resample(self, lo, hi, i_fb, u, total):
        st = self.o.state()
        d, p, R = self.w.d, self.w.p, self.info["record"]
        for j, i in enumerate(range(lo, hi)):
            if i >= i_fb:
                l = int(np.searchsorted(self.c_local, total, side="left"))
            else:
                l = int(np.searchsorted(self.c_local, SH.threshold(i, u, self.n_all, total), side="right"))
            r = self.send[j * R:(j + 1) * R]
            r[0:d], r[d:2 * d], r[2 * d:3 * d] = st["x"][l], st["h1"][l], st["h2"][l]
            r[3 * d:3 * d + p] = st["phi"][l]
            r[3 * d + p] = self.ll1[l]
            r[3 * d + p + 1] = l + self.first
        return self.send

    # Steps 3c-5 from the received parents
    def stage2(self):
        d, p, R = self.w.d, self.w.p, self.info["record"]
        rec = self.recv.reshape(self.n, R)
        self.saved = self.o.state()
        self.o.set_state(x=rec[:, 0:d], h1=rec[:, d:2 * d], h2=rec[:, 2 * d:3 * d],
                         phi=rec[:, 3 * d:3 * d + p])
        self.o.set_ll1(rec[:, 3 * d + p])
        self.parents = rec[:, 3 * d + p + 1].astype(np.int64)
        assert self.o.stage2(self.tab, self.S, self.y, np.arange(self.n, dtype=np.int32)) == oracle.OK
        self.pending = True
        lw = self.o.pending_lw()
        fin = np.isfinite(lw)
        return float(np.max(lw[fin])) if fin.any() else -math.inf

    def moments(self, M):
        self.M = M
        return self.o.shard_sums(self.pending, M)

    def commit(self, sums):
        assert self.o.shard_commit(self.pending, self.M, sums, self.t if self.pending else 0.0) == oracle.OK
        self.pending = False

    def abort(self):
        if getattr(self, "saved", None) is not None and self.pending:
            self.o.set_state(**self.saved)
        self.pending = False

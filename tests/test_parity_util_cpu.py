"""CPU checks of the parity checker itself (tests/parity_util.py).

check_epoch compares the CUDA library with the oracle; here a second oracle
filter stands in for the library, so the checker's bounds can be exercised
without a GPU: two identical implementations must pass, and a planted slip
in the stand-in's Step 5 (the child's first-stage log-likelihood in place of
the parent's) or in its propagated state must fail.  The stand-in is test
scaffolding only; it is never a fallback for the library.
"""
import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import workloads as W
from parity_util import check_epoch


class OracleStandIn:
    """The calls of the library's Filter that check_epoch makes, served by
    the oracle, with optional planted slips."""

    def __init__(self, w, slip=None):
        self.o = oracle.Filter(w)
        self.o.init()
        self.slip = slip
        self.est = None

    def pf_get_ensemble(self):
        return self.o.state()

    def pf_estimates(self):
        if self.est is not None:
            return self.est
        m = self.o.moments()
        return m["phibar"], m["C"], m["xbar"]

    def pf_get_history(self):
        return self.o.history()

    def pf_get_work(self):
        wk = self.o.work()
        wk["idx"] = self._idx
        return wk

    def pf_stats(self):
        wk = self.pf_get_work()
        return dict(unique_parents=len(np.unique(wk["idx"])), ess=self.o.moments()["ess"])

    def pf_assimilate(self, t, y):
        o = self.o
        tab, S = o.substeps(t)
        assert o.stage1(tab, S, y) == oracle.OK
        assert o.cumulative() == oracle.OK
        wk = o.work()
        idx = oracle.resample_systematic(wk["c"], o.resample_u())
        assert o.stage2(tab, S, y, idx) == oracle.OK
        assert o.commit(t) == oracle.OK
        self._idx = idx
        self.est = None
        if self.slip is None:
            return
        st = o.state()
        if self.slip == "step5_child_ll1":
            lw = st["lw"] + wk["ll1"][idx] - wk["ll1"]
            lw -= np.max(lw) + np.log(np.sum(np.exp(lw - np.max(lw))))
            st["lw"] = lw
        elif self.slip == "state":
            st["x"] = st["x"] * (1.0 + 1e-8)
        o.set_state(**st)
        wt = np.exp(st["lw"])
        pb = np.average(st["phi"], axis=0, weights=wt)
        self.est = (pb, np.cov(st["phi"].T, aweights=wt, bias=True),
                    np.average(st["x"], axis=0, weights=wt))


def _run(w, slip, epochs):
    g = OracleStandIn(w, slip)
    o = oracle.Filter(w)
    o.init()
    out = []
    for k in range(epochs):
        out.append(check_epoch(g, o, w.t_obs[k], w.y_obs[k]))
        g.o.set_moments(*g.pf_estimates()[:2])
    return out


@pytest.mark.parametrize("name,N", [("linear2", 700), ("robertson", 900)])
def test_identical_implementations_pass(oracle_lib, name, N):
    w = W.get(name, N=N, T=4)
    for errs in _run(w, None, 3):
        assert errs["x"] == 0.0 and errs["w"] == 0.0 and errs["dlw"] == 0.0
        # the derived ceilings are tight enough to mean something
        print(name, errs["tol"])
        assert errs["tol"]["lw"] < 1e-6 and errs["tol"]["w"] < 1e-6


@pytest.mark.parametrize("slip", ["step5_child_ll1", "state"])
def test_planted_slips_fail(oracle_lib, slip):
    w = W.robertson(N=900, T=4)
    with pytest.raises(AssertionError):
        _run(w, slip, 2)

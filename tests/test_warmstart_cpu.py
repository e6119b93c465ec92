"""Host logic of the warm-start evaluation (paper_1405_2232_gb300.warmstart),
with the batched solver, the network and the handoff replaced by stand-ins:
every arm is run on the same cases with the parameters it names (start at
rest or at u = 0, predicted or initial temperature), and the summary counts
and medians are those of the per-case records.  CPU only."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1405_2232_gb300 import inputs as I  # noqa: E402
from paper_1405_2232_gb300 import lb  # noqa: E402
from paper_1405_2232_gb300 import unet as UN  # noqa: E402
from paper_1405_2232_gb300 import warmstart as WS  # noqa: E402


class _FakeBatch:
    def __init__(self, L):
        self.L = L

    def fields(self, d):
        return np.full((self.L, self.L), 0.1), np.full((self.L, self.L), 0.07)

    def close(self):
        pass


def test_evaluate_runs_every_arm_with_its_start(monkeypatch):
    calls = []
    rng = np.random.default_rng(0)
    n, L = 8, 32

    def fake_solve(params, rhos, Ts, cap, device_inputs=False, chunk_rows=None):
        calls.append((tuple(p.init_balanced for p in params), device_inputs, len(rhos)))
        st = rng.choice([lb.LB_OK, lb.LB_ERR_PSI_DOMAIN, lb.LB_ERR_NOT_CONVERGED], size=n).astype(np.int32)
        st[:3] = lb.LB_OK  # some cases converge in every arm
        steps = rng.integers(100, cap, size=n)
        return steps, np.zeros(n), st, 1.0, _FakeBatch(L)

    fb_calls = []

    def fake_fallback(pw, warm, pp, plain, cap, probe, chunk_rows=None):
        fb_calls.append((tuple(p.init_balanced for p in pw), tuple(p.init_balanced for p in pp), probe))
        st = np.full(n, lb.LB_OK, dtype=np.int32)
        return rng.integers(100, cap, size=n), np.zeros(n), st, 1.0, 2

    t_scales = []

    def fake_warm(N, H, W, pred, norm, r0, t0, r, t):
        t_scales.append(norm["t_dev_scale"])
        r.copy_(r0)
        t.copy_(t0)

    real_device = torch.device
    monkeypatch.setattr(WS, "solve", fake_solve)
    monkeypatch.setattr(WS, "solve_with_fallback", fake_fallback)
    monkeypatch.setattr(WS, "_sync", lambda: None)
    monkeypatch.setattr(WS, "predict", lambda net, X, batch: torch.zeros((X.shape[0], L, L, 2)))
    monkeypatch.setattr(UN, "warm_fields", fake_warm)
    monkeypatch.setattr(torch, "device", lambda s: real_device("cpu"))
    doms, masks = I.warm_start_cases(n, L=L, seed=6)
    ev = WS.evaluate(None, doms, masks, 80000, probe=3000)

    # plain, plain at rest, warm at rest, warm (initial T) at rest; the fallback
    # arm starts warm at rest and restarts plain (u = 0)
    assert [c[0] for c in calls] == [(0,) * n, (1,) * n, (1,) * n, (1,) * n]
    assert [c[1] for c in calls] == [False, False, True, True]
    assert fb_calls == [((1,) * n, (0,) * n, 3000)]
    assert t_scales == [I.UNET_NORM["t_dev_scale"], 0.0]
    pc = ev.pop("per_case")
    json.dumps(ev)
    json.dumps(pc)
    arms = ("plain", "plain_balanced", "warm", "warm_T0", "warm_fallback")
    for arm in arms:
        st = np.array(pc["status_" + arm])
        a = ev[arm]
        assert a["converged"] + a["failed"] + a["capped"] == n
        assert a["converged"] == int(np.sum(st == lb.LB_OK))
        assert a["capped"] == int(np.sum(st == lb.LB_ERR_NOT_CONVERGED))
    assert ev["warm_fallback"]["restarts"] == 2
    allc = np.all([np.array(pc["status_" + k]) == lb.LB_OK for k in arms], axis=0)
    assert ev["all_arms_converged"] == int(allc.sum()) >= 3
    for arm, med in ev["median_steps_all_arms"].items():
        assert med == float(np.median(np.array(pc["steps_" + arm])[allc]))
    p_st, p_steps = np.array(pc["status_plain"]), np.array(pc["steps_plain"])
    for arm, v in ev["vs_plain"].items():
        both = (p_st == lb.LB_OK) & (np.array(pc["status_" + arm]) == lb.LB_OK)
        assert v["both_converged"] == int(both.sum())
        assert v["steps_ratio"] == pytest.approx(np.array(pc["steps_" + arm])[both].sum() / p_steps[both].sum())


class _FakeRunBatch:
    """Stand-in of lb.Batch for the fallback schedule: domains 0, 1 converge
    during the probe, 2 fails, 3 is still relaxing."""

    log = []

    def __init__(self, params, rhos, Ts, device_inputs=False):
        self.n = len(params)
        _FakeRunBatch.log.append(("init", device_inputs))

    def run(self, tol, K, max_steps):
        _FakeRunBatch.log.append(("run", max_steps))
        st = np.array([lb.LB_OK, lb.LB_OK, lb.LB_ERR_PSI_DOMAIN, lb.LB_ERR_NOT_CONVERGED], dtype=np.int32)
        return np.full(self.n, max_steps), np.zeros(self.n), st

    def restart(self, d, rho, T, init_balanced=0):
        _FakeRunBatch.log.append(("restart", d, init_balanced))

    def close(self):
        pass


def test_fallback_restarts_what_did_not_converge(monkeypatch):
    monkeypatch.setattr(lb, "Batch", _FakeRunBatch)
    _FakeRunBatch.log.clear()
    pw = [lb.lb_params_default(init_balanced=1) for _ in range(4)]
    pp = [lb.lb_params_default(init_balanced=0) for _ in range(4)]
    fields = ([np.zeros((64, 64))] * 4, [np.zeros((64, 64))] * 4)
    steps, resid, st, wall, nr = WS.solve_with_fallback(pw, fields, pp, fields, 10000, 1500)
    assert nr == 2
    assert _FakeRunBatch.log == [("init", False), ("run", 1500), ("restart", 2, 0), ("restart", 3, 0),
                                 ("run", 8500)]

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

    t_scales = []

    def fake_warm(N, H, W, pred, norm, r0, t0, r, t):
        t_scales.append(norm["t_dev_scale"])
        r.copy_(r0)
        t.copy_(t0)

    real_device = torch.device
    monkeypatch.setattr(WS, "solve", fake_solve)
    monkeypatch.setattr(WS, "_sync", lambda: None)
    monkeypatch.setattr(WS, "predict", lambda net, X, batch: torch.zeros((X.shape[0], L, L, 2)))
    monkeypatch.setattr(UN, "warm_fields", fake_warm)
    monkeypatch.setattr(torch, "device", lambda s: real_device("cpu"))
    doms, masks = I.warm_start_cases(n, L=L, seed=6)
    ev = WS.evaluate(None, doms, masks, 80000)

    # plain, plain at rest, warm at rest, warm at u = 0, warm (initial T) at rest
    assert [c[0] for c in calls] == [(0,) * n, (1,) * n, (1,) * n, (0,) * n, (1,) * n]
    assert [c[1] for c in calls] == [False, False, True, True, True]
    assert t_scales == [I.UNET_NORM["t_dev_scale"], 0.0]
    pc = ev.pop("per_case")
    json.dumps(ev)
    json.dumps(pc)
    for arm in ("plain", "plain_balanced", "warm", "warm_T0", "warm_unbalanced"):
        st = np.array(pc["status_" + arm])
        a = ev[arm]
        assert a["converged"] + a["failed"] + a["capped"] == n
        assert a["converged"] == int(np.sum(st == lb.LB_OK))
        assert a["capped"] == int(np.sum(st == lb.LB_ERR_NOT_CONVERGED))
    allc = np.all([np.array(pc["status_" + k]) == lb.LB_OK
                   for k in ("plain", "plain_balanced", "warm", "warm_T0", "warm_unbalanced")], axis=0)
    assert ev["all_arms_converged"] == int(allc.sum()) >= 3
    for arm, med in ev["median_steps_all_arms"].items():
        assert med == float(np.median(np.array(pc["steps_" + arm])[allc]))

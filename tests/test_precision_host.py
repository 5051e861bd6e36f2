"""Host logic of the FP32-against-FP64 driver (no GPU): lockstep sampling, the metrics
and the stop at a non-finite state, with the library replaced by a stand-in whose two
'precisions' decay the state at slightly different rates."""
import math
import types

import pytest

torch = pytest.importorskip("torch")
from paper_2207_11571_gb300 import precision_run  # noqa: E402


class _Event:
    def __init__(self, **kw):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 1.0


def _fake_dg(diverge_fp32_below=None):
    ctxs = {}

    def create(K, P, Re, Mach, Pr, les, precision=0, volume_flux=0):
        ctxs[len(ctxs) + 1] = {"N": K ** 3 * (P + 1) ** 3, "fp32": precision == 1}
        return len(ctxs)

    def init(c, q, pert):
        q.copy_(torch.ones_like(q) + pert)

    def step(c, q, h, n, net, stream):
        rate = 0.01 * (1.0 + (1e-6 if ctxs[c]["fp32"] else 0.0))
        q.mul_(1.0 - rate * h * n)
        if diverge_fp32_below is not None and ctxs[c]["fp32"] and float(q[0]) < diverge_fp32_below:
            q.fill_(float("nan"))

    def diagnostics(c, q, raise_nonfinite=True):
        ke = float(q.view(5, -1)[1:4].pow(2).sum()) / 2
        return {"ke": ke, "dke_dt": -0.02 * ke, "nonfinite": int(not math.isfinite(ke))}

    return types.SimpleNamespace(DG_PREC_FP32=1, DG_PREC_FP64=0, dg_create=create,
                                 dg_sizes=lambda c: (ctxs[c]["N"], 0), dg_init_tgv=init,
                                 dg_stable_dt=lambda c, q, cfl: 3e-3, dg_autotune=lambda c, q, dt: (2, 0.1),
                                 dg_rk3_step=step, dg_diagnostics=diagnostics, dg_destroy=lambda c: None)


@pytest.fixture
def on_host(monkeypatch):
    empty = torch.empty
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: None)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self: self)
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **k: empty(*a, **k))
    return monkeypatch


def test_lockstep_samples_and_metrics(on_host):
    on_host.setattr(precision_run, "dg", _fake_dg())
    r = precision_run.run(2, 1, t_end=0.2, sample=0.05)
    assert r["history"]["t"] == pytest.approx([0.0, 0.05, 0.1, 0.15, 0.2])
    assert r["t_reached"] == pytest.approx(0.2) and r["diverged_at"] is None
    assert r["steps"] == 4 * math.ceil(0.05 / 3e-3)
    # the two runs decay at rates 1e-6 apart: KE differs by ~2 * 0.01 * 1e-6 * t
    assert 0 < r["ke_rel_max"] < 1e-8 and r["momentum_rel_l2_at_end"] < 1e-8
    assert r["ms_per_step"]["fp32"] == pytest.approx(4 / r["steps"])


def test_stops_at_the_first_non_finite_sample(on_host):
    on_host.setattr(precision_run, "dg", _fake_dg(diverge_fp32_below=0.9985))
    r = precision_run.run(2, 1, t_end=10.0, sample=0.1)
    assert r["diverged_at"] == {"fp32": pytest.approx(0.2)}
    assert r["t_reached"] == pytest.approx(0.1) and r["momentum_rel_l2_at_end"] is None
    assert math.isfinite(r["ke_rel_max"]) and math.isfinite(r["dissipation_rel_l2"])

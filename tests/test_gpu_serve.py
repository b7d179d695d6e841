"""Serving loop: every served result matches the FP64 oracle and the same
request run alone (to the split-precision tolerance), the device-memory
budget bounds what is in flight, and requests overlap on the device across
slots."""
import numpy as np
import pytest
import torch

from paper_1908_06096_gb300 import inputs
from tests.conftest import per_field_max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _payload(st_mod, plan, T, nf, direction, seed):
    if direction == "inv":
        return torch.from_numpy(inputs.spectra(T, nf, seed=seed)).to(torch.float32).pin_memory()
    g = inputs.grid_noise(plan.npts, nf, seed=seed)
    return torch.from_numpy(g).to(torch.float32).pin_memory()


@pytest.mark.parametrize("budget_mb", [1024, 3])
def test_served_results_match_oracle_and_alone(st_mod, oracle_mod, budget_mb):
    from paper_1908_06096_gb300 import serve
    Ts = (31, 63, 255)
    srv = serve.Server(Ts, precision="bf16x3", slots=2, max_fields=12, budget_bytes=budget_mb << 20,
                       keep_results=True)
    rng = np.random.default_rng(7)
    reqs = []
    t = 0.0
    for i in range(40):
        T = int(rng.choice(Ts)) if i else 255          # at least one T255 request
        nf = int(rng.integers(1, 6))
        d = "inv" if rng.integers(0, 2) == 0 else "dir"
        t += float(rng.exponential(2e-4))
        reqs.append(serve.Request(i, t, T, nf, d, _payload(st_mod, srv.base[T], T, nf, d, 900 + i)))
    stats = srv.run(reqs)
    assert stats["requests"] == 40
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    alone = {T: st_mod.Plan(T, "regular", precision="bf16x3", max_fields=8) for T in Ts}
    geo = {}
    for T, p in alone.items():
        rows = oracle_mod.grid_rows("regular", p.nlat, p.nlon)
        mu, w = oracle_mod.gauss(p.nlat)
        geo[T] = (rows, mu, w)
    for r in reqs:
        p = alone[r.T]
        rows, mu, w = geo[r.T]
        x = r.payload.to("cuda")
        ref = p.inv(x) if r.direction == "inv" else p.dir(x)
        got = r.result.view(ref.shape).double().numpy()
        assert per_field_max_rel(got, ref.double().cpu().numpy()) <= 2e-5, (r.rid, r.T, r.direction)
        xin = r.payload.double().numpy()
        if r.direction == "inv":
            oref = oracle_mod.inv_trans(r.T, rows, mu, xin.reshape(r.nfields, -1, 2))
            err = per_field_max_rel(got, oref)
        else:
            oref = oracle_mod.dir_trans(r.T, rows, mu, w, xin.reshape(r.nfields, -1))
            err = per_field_max_rel(got[..., 0] + 1j * got[..., 1], oref)
        assert err < 2e-5, (r.rid, r.T, r.direction, err)
    for p in alone.values():
        p.close()
    srv.close()


def test_admission_never_exceeds_budget(st_mod):
    from paper_1908_06096_gb300 import serve
    srv = serve.Server((63,), precision="bf16x3", slots=3, max_fields=16, budget_bytes=0)
    p = srv.base[63]
    one_field = srv.footprint(serve.Request(0, 0.0, 63, 1, "inv", torch.empty(0)))
    srv.budget = 5 * one_field           # room for five fields in flight
    peak = {"v": 0}
    orig = srv._launch

    def spy(slot, batch, ev):
        inflight = sum(srv.footprint(r) for s in srv.slots for r in s.busy) + \
            sum(srv.footprint(r) for r in batch)
        peak["v"] = max(peak["v"], inflight)
        return orig(slot, batch, ev)

    srv._launch = spy
    reqs = [serve.Request(i, 0.0, 63, 2, "inv", _payload(st_mod, p, 63, 2, "inv", i)) for i in range(12)]
    stats = srv.run(reqs)
    assert stats["requests"] == 12
    assert 0 < peak["v"] <= srv.budget
    assert 0 < stats["peak_inflight_bytes"] <= srv.budget
    # latencies are measured from arrival on the run's own clock
    assert 0 < stats["p50_ms"] <= stats["max_ms"] < 60_000
    srv.close()

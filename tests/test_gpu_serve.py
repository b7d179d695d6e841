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


# arena for request payloads: roomy, or just above the largest request (T255,
# 5 fields: about 4 MB) so that admission has to hold requests back
@pytest.mark.parametrize("arena_mb", [1024, 6])
def test_served_results_match_oracle_and_alone(st_mod, oracle_mod, arena_mb):
    from paper_1908_06096_gb300 import serve
    Ts = (31, 63, 255)
    srv = serve.Server(Ts, precision="bf16x3", slots=2, max_fields=12, arena_bytes=arena_mb << 20,
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


def test_admission_defers_when_the_device_budget_would_be_exceeded(st_mod):
    """Resident tables and workspaces count against the device budget; a
    request whose input and output do not fit what is left waits until
    requests in flight complete, and resident + in-flight never exceeds the
    budget."""
    from paper_1908_06096_gb300 import serve
    probe = serve.Server((63,), precision="bf16x3", slots=3, max_fields=16, arena_bytes=1 << 20)
    resident = probe.resident_bytes
    one = probe.footprint(serve.Request(0, 0.0, 63, 2, "inv", torch.empty(0)))
    probe.close()
    # room for one two-field request in flight (and not for two)
    budget = resident + one + one // 2
    srv = serve.Server((63,), precision="bf16x3", slots=3, max_fields=16, budget_bytes=budget)
    assert srv.resident_bytes == resident
    p = srv.base[63]
    peak = {"v": 0}
    orig = srv._launch

    def spy(slot, batch, blocks):
        peak["v"] = max(peak["v"], srv.arena.used * srv.arena.buf.element_size())
        return orig(slot, batch, blocks)

    srv._launch = spy
    reqs = [serve.Request(i, 0.0, 63, 2, "inv", _payload(st_mod, p, 63, 2, "inv", i)) for i in range(12)]
    stats = srv.run(reqs)
    assert stats["requests"] == 12
    assert stats["requests_deferred_for_memory"] > 0
    assert 0 < peak["v"] <= budget - resident
    assert stats["resident_bytes"] + stats["peak_inflight_bytes"] <= stats["budget_bytes"] == budget
    # latencies are measured from arrival on the run's own clock
    assert 0 < stats["p50_ms"] <= stats["max_ms"] < 60_000
    srv.close()


def test_budget_below_resident_is_refused(st_mod):
    from paper_1908_06096_gb300 import serve
    with pytest.raises(serve.AdmissionError):
        serve.Server((31,), precision="bf16x3", slots=1, max_fields=4, budget_bytes=4096)

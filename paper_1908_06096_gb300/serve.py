"""Continuous-batching server for spherical-harmonic transforms.

Requests (truncation T, number of fields, inverse or direct, host payload)
arrive over time.  The server keeps, per truncation, one set of Legendre
tables and FFT data resident on the device, and several slots; a slot is a
CUDA stream with its own workspace (a plan sharing the resident tables, see
st_plan_create_shared) and its own device staging buffers.  Whenever a slot is
free, the oldest waiting request is taken together with later waiting requests
of the same truncation and direction, as many as fit the slot's field budget
and the server's device-memory budget (admission by footprint), copied in,
transformed in one call, and copied out.  Slots run concurrently, so work of
requests that arrived while others were on the device overlaps with it.

Latency of a request = completion (a CUDA event after its result reached host
memory) - arrival.  The paper has no serving layer; this is the systems side
of running the transform (ESCAPE D3.3 section 4.2.3's "reusable arrays":
everything resident, nothing allocated per request).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import st


@dataclass
class Request:
    rid: int
    t_arrival: float          # seconds from the start of the run
    T: int
    nfields: int
    direction: str            # "inv" or "dir"
    payload: torch.Tensor     # pinned host tensor: spectra [nf, nspec, 2] or grid [nf, npts]
    t_done: float | None = None
    result: torch.Tensor | None = None


@dataclass
class _Slot:
    idx: int
    stream: torch.cuda.Stream
    plans: dict
    d_spec: torch.Tensor
    d_grid: torch.Tensor
    d_out: torch.Tensor
    h_out: torch.Tensor
    busy: list = field(default_factory=list)   # requests in flight
    bytes: int = 0
    event: torch.cuda.Event | None = None
    kind: tuple | None = None


class Server:
    def __init__(self, truncations, precision: str = "bf16x3", grid: str = "regular", slots: int = 4,
                 max_fields: int = 137, budget_bytes: int = 32 << 30, keep_results: bool = False):
        self.precision = precision
        self.max_fields = max_fields
        self.budget = budget_bytes
        self.keep = keep_results
        self.base = {T: st.Plan(T, grid, precision=precision, max_fields=1) for T in truncations}
        self.dtype = next(iter(self.base.values())).dtype
        es = 8 if self.dtype == torch.float64 else 4
        max_spec = max(p.nspec for p in self.base.values()) * 2 * max_fields
        max_grid = max(p.npts for p in self.base.values()) * max_fields
        self.slots = []
        for k in range(slots):
            plans = {T: st.Plan(T, share_with=b, max_fields=max_fields) for T, b in self.base.items()}
            d_spec = torch.empty(max_spec, dtype=self.dtype, device="cuda")
            d_grid = torch.empty(max_grid, dtype=self.dtype, device="cuda")
            d_out = torch.empty(max(max_spec, max_grid), dtype=self.dtype, device="cuda")
            h_out = torch.empty(max(max_spec, max_grid), dtype=self.dtype).pin_memory()
            self.slots.append(_Slot(k, torch.cuda.Stream(), plans, d_spec, d_grid, d_out, h_out))
        self.resident_bytes = sum(int(p.info.device_bytes) for p in self.base.values()) + \
            sum(int(pl.info.device_bytes) for s in self.slots for pl in s.plans.values()) + \
            slots * (max_spec + max_grid + max(max_spec, max_grid)) * es
        torch.cuda.synchronize()

    def footprint(self, r: Request) -> int:
        """Device bytes a request occupies while in flight (input + output)."""
        p = self.base[r.T]
        es = 8 if self.dtype == torch.float64 else 4
        return r.nfields * (p.nspec * 2 + p.npts) * es

    def close(self):
        for s in self.slots:
            for p in s.plans.values():
                p.close()
        for p in self.base.values():
            p.close()

    # ------------------------------------------------------------------
    def _launch(self, slot: _Slot, batch: list, t0_event: torch.cuda.Event):
        T, direction = batch[0].T, batch[0].direction
        plan = slot.plans[T]
        nf = sum(r.nfields for r in batch)
        with torch.cuda.stream(slot.stream):
            if direction == "inv":
                per_in, per_out = plan.nspec * 2, plan.npts
                src = slot.d_spec[:nf * per_in].view(nf, plan.nspec, 2)
                dst = slot.d_out[:nf * per_out].view(nf, plan.npts)
            else:
                per_in, per_out = plan.npts, plan.nspec * 2
                src = slot.d_grid[:nf * per_in].view(nf, plan.npts)
                dst = slot.d_out[:nf * per_out].view(nf, plan.nspec, 2)
            off = 0
            for r in batch:
                src.view(-1)[off * per_in:(off + r.nfields) * per_in].copy_(r.payload.view(-1), non_blocking=True)
                off += r.nfields
            if direction == "inv":
                plan.inv(src, out=dst, stream=slot.stream)
            else:
                plan.dir(src, out=dst, stream=slot.stream)
            slot.h_out[:nf * per_out].copy_(dst.view(-1), non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(slot.stream)
        slot.busy = batch
        slot.event = ev
        slot.kind = (T, direction, per_out)

    def _complete(self, slot: _Slot, t0_event: torch.cuda.Event):
        # seconds from the start of the run, on the device clock
        t_done = t0_event.elapsed_time(slot.event) * 1e-3
        T, direction, per_out = slot.kind
        off = 0
        for r in slot.busy:
            r.t_done = t_done
            if self.keep:
                r.result = slot.h_out[off * per_out:(off + r.nfields) * per_out].clone()
            off += r.nfields
        done = slot.busy
        slot.busy = []
        slot.event = None
        return done

    def run(self, requests: list) -> dict:
        """Serve `requests` (any order; arrivals from t_arrival); returns
        latency statistics.  Waiting requests are queued per (T, direction);
        a free slot takes the oldest waiting request and the following ones of
        its queue that fit."""
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        queues: dict = collections.OrderedDict()
        nwait = 0
        inflight_bytes = 0
        finished = []
        t0_event = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0_event.record()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        foot = {}
        peak_inflight = 0
        while pending or nwait or any(s.busy for s in self.slots):
            now = time.perf_counter() - t0
            while pending and pending[0].t_arrival <= now:
                r = pending.popleft()
                queues.setdefault((r.T, r.direction), collections.deque()).append(r)
                nwait += 1
            for s in self.slots:
                if s.busy and s.event.query():
                    for r in self._complete(s, t0_event):
                        inflight_bytes -= foot.pop(r.rid)
                        finished.append(r)
            for s in self.slots:
                if s.busy or not nwait:
                    continue
                key = min((k for k, q in queues.items() if q), key=lambda k: queues[k][0].t_arrival)
                q = queues[key]
                head = q[0]
                fh = self.footprint(head)
                if inflight_bytes + fh > self.budget and inflight_bytes > 0:
                    break  # admission by footprint: wait for memory to free up
                # (a request larger than the whole budget runs alone)
                batch, nf, fb = [q.popleft()], head.nfields, fh
                while q:
                    r = q[0]
                    f = self.footprint(r)
                    if nf + r.nfields > self.max_fields or inflight_bytes + fb + f > self.budget:
                        break
                    batch.append(q.popleft())
                    nf += r.nfields
                    fb += f
                nwait -= len(batch)
                for r in batch:
                    foot[r.rid] = self.footprint(r)
                inflight_bytes += fb
                peak_inflight = max(peak_inflight, inflight_bytes)
                self._launch(s, batch, t0_event)
            if not nwait and pending and not any(s.busy for s in self.slots):
                dt = pending[0].t_arrival - (time.perf_counter() - t0)
                if dt > 2e-4:
                    time.sleep(dt - 1e-4)
        torch.cuda.synchronize()
        wall = max(r.t_done for r in finished) - min(r.t_arrival for r in finished)
        lat = np.array([r.t_done - r.t_arrival for r in finished])
        fields = sum(r.nfields for r in finished)
        return {"requests": len(finished), "fields": fields, "wall_s": wall,
                "field_transforms_per_s": fields / wall, "requests_per_s": len(finished) / wall,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3),
                "peak_inflight_bytes": int(peak_inflight)}


def make_requests(specs, payloads) -> list:
    """specs: dicts from inputs.serve_requests; payloads[(T, direction)] is a
    pinned host tensor with at least max_fields fields, sliced per request."""
    out = []
    for i, s in enumerate(specs):
        p = payloads[(s["T"], s["direction"])]
        out.append(Request(i, s["t"], s["T"], s["nfields"], s["direction"], p[:s["nfields"]]))
    return out

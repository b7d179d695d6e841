"""Continuous-batching server for spherical-harmonic transforms.

Requests (truncation T, number of fields, inverse or direct, host payload)
arrive over time.  The server keeps, per truncation, one set of Legendre
tables and FFT data resident on the device, and several slots; a slot is a
CUDA stream with its own workspace (a plan per truncation sharing the
resident tables, see st_plan_create_shared).  Whenever a slot is free, the
oldest waiting request is taken together with later waiting requests of the
same truncation and direction, as many as fit the slot's field limit and the
device budget, copied in, transformed in one call, and copied out.  Slots run
concurrently, so work of requests that arrived while others were on the
device overlaps with it.

Device memory is accounted as a whole against ``budget_bytes``:
  resident = tables + every slot's plan workspaces (allocated at start-up),
  arena    = budget - resident, one device buffer that holds the inputs and
             outputs of the requests in flight.
A batch is admitted only when its input and output fit in the arena's free
space (first fit); otherwise it waits until completed requests release
theirs.  So at any time  resident + in-flight bytes <= budget.

Latency of a request = completion (a CUDA event after its result reached host
memory) - arrival.  The paper has no serving layer; this is the systems side
of running the transform (ESCAPE D3.3 section 4.2.3's "reusable arrays":
everything resident, nothing allocated per request).
"""
from __future__ import annotations

import bisect
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


class Arena:
    """First-fit allocator over one device buffer (element offsets).  Blocks
    are rounded up to 64 elements so that every block starts 256-byte
    aligned."""

    ALIGN = 64

    def __init__(self, nelem: int, dtype):
        self.buf = torch.empty(max(nelem, self.ALIGN), dtype=dtype, device="cuda")
        self.size = self.buf.numel()
        self.free = [(0, self.size)]          # sorted (offset, length)
        self.used = 0
        self.peak = 0

    def alloc(self, n: int):
        n = (n + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    del self.free[i]
                else:
                    self.free[i] = (off + n, ln - n)
                self.used += n
                self.peak = max(self.peak, self.used)
                return off, n
        return None

    def release(self, off: int, n: int):
        self.used -= n
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, n))
        # merge with the neighbours
        if i + 1 < len(self.free) and off + n == self.free[i + 1][0]:
            self.free[i] = (off, n + self.free[i + 1][1])
            del self.free[i + 1]
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == off:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            del self.free[i]

    def view(self, off: int, n: int):
        return self.buf[off:off + n]


@dataclass
class _Slot:
    idx: int
    stream: torch.cuda.Stream
    plans: dict
    h_out: torch.Tensor
    busy: list = field(default_factory=list)   # requests in flight
    blocks: list = field(default_factory=list)  # arena blocks of the batch in flight
    event: torch.cuda.Event | None = None
    kind: tuple | None = None


class AdmissionError(RuntimeError):
    pass


class Server:
    def __init__(self, truncations, precision: str = "bf16x3", grid: str = "regular", slots: int = 4,
                 max_fields: int = 137, budget_bytes: int | None = None, arena_bytes: int | None = None,
                 keep_results: bool = False):
        """budget_bytes: device bytes the server may hold in all (resident
        tables and workspaces plus the request arena).  If None, the budget is
        the resident bytes plus arena_bytes (default 8 GiB)."""
        self.precision = precision
        self.max_fields = max_fields
        self.keep = keep_results
        self.base = {T: st.Plan(T, grid, precision=precision, max_fields=1) for T in truncations}
        self.dtype = next(iter(self.base.values())).dtype
        self.es = 8 if self.dtype == torch.float64 else 4
        max_spec = max(p.nspec for p in self.base.values()) * 2 * max_fields
        max_grid = max(p.npts for p in self.base.values()) * max_fields
        self.slots = []
        for k in range(slots):
            plans = {T: st.Plan(T, share_with=b, max_fields=max_fields) for T, b in self.base.items()}
            h_out = torch.empty(max(max_spec, max_grid), dtype=self.dtype).pin_memory()
            self.slots.append(_Slot(k, torch.cuda.Stream(), plans, h_out))
        # base plans hold the shared tables (and a one-field workspace each)
        self.resident_bytes = sum(int(p.info.device_bytes) for p in self.base.values()) + \
            sum(int(pl.info.device_bytes) for s in self.slots for pl in s.plans.values())
        if budget_bytes is None:
            budget_bytes = self.resident_bytes + (8 << 30 if arena_bytes is None else arena_bytes)
        self.budget = int(budget_bytes)
        arena = self.budget - self.resident_bytes
        if arena <= 0:
            self.close()
            raise AdmissionError(f"device budget {self.budget} B is below the resident {self.resident_bytes} B")
        self.arena = Arena(arena // self.es, self.dtype)
        torch.cuda.synchronize()

    def footprint(self, r: Request) -> int:
        """Device bytes a request occupies while in flight (input + output)."""
        p = self.base[r.T]
        return r.nfields * (p.nspec * 2 + p.npts) * self.es

    def close(self):
        for s in getattr(self, "slots", []):
            for p in s.plans.values():
                p.close()
        for p in self.base.values():
            p.close()

    # ------------------------------------------------------------------
    def _reserve(self, batch: list):
        """Arena blocks for a batch's input and output, or None if they do not
        fit the free space now."""
        T, direction = batch[0].T, batch[0].direction
        p = self.base[T]
        nf = sum(r.nfields for r in batch)
        n_in = nf * (p.nspec * 2 if direction == "inv" else p.npts)
        n_out = nf * (p.npts if direction == "inv" else p.nspec * 2)
        a = self.arena.alloc(n_in)
        if a is None:
            return None
        b = self.arena.alloc(n_out)
        if b is None:
            self.arena.release(*a)
            return None
        return a, b

    def _launch(self, slot: _Slot, batch: list, blocks):
        T, direction = batch[0].T, batch[0].direction
        plan = slot.plans[T]
        nf = sum(r.nfields for r in batch)
        (ia, na), (oa, no) = blocks
        with torch.cuda.stream(slot.stream):
            if direction == "inv":
                per_in, per_out = plan.nspec * 2, plan.npts
                src = self.arena.view(ia, nf * per_in).view(nf, plan.nspec, 2)
                dst = self.arena.view(oa, nf * per_out).view(nf, plan.npts)
            else:
                per_in, per_out = plan.npts, plan.nspec * 2
                src = self.arena.view(ia, nf * per_in).view(nf, plan.npts)
                dst = self.arena.view(oa, nf * per_out).view(nf, plan.nspec, 2)
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
        slot.blocks = [(ia, na), (oa, no)]
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
        for blk in slot.blocks:
            self.arena.release(*blk)
        done = slot.busy
        slot.busy = []
        slot.blocks = []
        slot.event = None
        return done

    def run(self, requests: list) -> dict:
        """Serve `requests` (any order; arrivals from t_arrival); returns
        latency statistics.  Waiting requests are queued per (T, direction);
        a free slot takes the oldest waiting request and the following ones of
        its queue that fit the slot's field limit and the arena."""
        for r in requests:
            if self.footprint(r) > self.arena.size * self.es:
                raise AdmissionError(f"request {r.rid} needs {self.footprint(r)} B, more than the arena holds")
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        queues: dict = collections.OrderedDict()
        nwait = 0
        finished = []
        deferred = set()                       # requests that waited for device memory
        self.arena.peak = self.arena.used
        t0_event = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0_event.record()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while pending or nwait or any(s.busy for s in self.slots):
            now = time.perf_counter() - t0
            while pending and pending[0].t_arrival <= now:
                r = pending.popleft()
                queues.setdefault((r.T, r.direction), collections.deque()).append(r)
                nwait += 1
            for s in self.slots:
                if s.busy and s.event.query():
                    finished.extend(self._complete(s, t0_event))
            for s in self.slots:
                if s.busy or not nwait:
                    continue
                key = min((k for k, q in queues.items() if q), key=lambda k: queues[k][0].t_arrival)
                q = queues[key]
                batch = [q[0]]
                nf = q[0].nfields
                for r in list(q)[1:]:
                    if nf + r.nfields > self.max_fields:
                        break
                    batch.append(r)
                    nf += r.nfields
                # admission by device memory: shrink the batch until its input
                # and output fit the arena's free space; if not even the head
                # request fits, it waits for in-flight requests to complete
                blocks = None
                while batch:
                    blocks = self._reserve(batch)
                    if blocks is not None:
                        break
                    batch.pop()
                if blocks is None:
                    deferred.add(q[0].rid)
                    break
                for _ in batch:
                    q.popleft()
                nwait -= len(batch)
                self._launch(s, batch, blocks)
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
                "peak_inflight_bytes": int(self.arena.peak * self.es),
                "resident_bytes": int(self.resident_bytes), "budget_bytes": int(self.budget),
                "requests_deferred_for_memory": len(deferred)}


def make_requests(specs, payloads) -> list:
    """specs: dicts from inputs.serve_requests; payloads[(T, direction)] is a
    pinned host tensor with at least max_fields fields, sliced per request."""
    out = []
    for i, s in enumerate(specs):
        p = payloads[(s["T"], s["direction"])]
        out.append(Request(i, s["t"], s["T"], s["nfields"], s["direction"], p[:s["nfields"]]))
    return out

"""Continuous-batching server for residual and adjoint evaluations (not in the paper).

Requests (a mesh, its field and coefficients, and the kind of evaluation) arrive over
time. The scheduler admits them as soon as an execution slot is free and the device
arena can hold their footprint; admitted requests run on per-slot CUDA streams, so
uploads, kernels and downloads of different requests overlap on the device while
new ones keep arriving. Latency is measured from arrival to the moment the host sees
the request's completion event.

Pieces:
  Arena           ctypes wrapper of libfem's host-side first-fit arena (fem_arena_*)
  Request         one evaluation with pinned host inputs and pinned host results
  footprint()     device bytes a request needs (every array rounded to 256 B)
  GpuExecutor     gives a request one arena block of a preallocated device buffer and
                  launches it with one native call (fem_serve_launch: upload, kernels,
                  download, event on the slot's stream); polls all events in one call
  Scheduler       the real-time admission loop (FIFO, optional backfill); it talks to
                  the executor through try_admit / launch / poll only
  request_log()   the served stream as records; save_request_log / replay_arrivals
                  store it and serve the same arrivals again
"""

from __future__ import annotations

import collections
import ctypes
import dataclasses
import gc
import math
import statistics
import time
from typing import Dict, List, Optional

import numpy as np
import torch

from . import binding
from .binding import value_dtype

ALIGN = 256


# ----------------------------------------------------------------------------- arena


class Arena:
    """Offsets into one device buffer, managed by libfem's native first-fit allocator."""

    def __init__(self, capacity: int, alignment: int = ALIGN):
        L = binding.lib()
        P = ctypes.c_void_p
        for name, args, res in (("fem_arena_create", [ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(P)], ctypes.c_int),
                                ("fem_arena_destroy", [P], None),
                                ("fem_arena_alloc", [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
                                ("fem_arena_free", [P, ctypes.c_int64], ctypes.c_int),
                                ("fem_arena_free_bytes", [P], ctypes.c_int64),
                                ("fem_arena_largest_free", [P], ctypes.c_int64),
                                ("fem_arena_capacity", [P], ctypes.c_int64)):
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        self._L = L
        self._h = P()
        st = L.fem_arena_create(int(capacity), int(alignment), ctypes.byref(self._h))
        if st != 0:
            raise binding.FemError("fem_arena_create", st, L.fem_last_error().decode())

    def alloc(self, nbytes: int) -> Optional[int]:
        off = ctypes.c_int64()
        st = self._L.fem_arena_alloc(self._h, int(nbytes), ctypes.byref(off))
        if st == -4:
            return None
        if st != 0:
            raise binding.FemError("fem_arena_alloc", st, self._L.fem_last_error().decode())
        return int(off.value)

    def free(self, offset: int) -> None:
        st = self._L.fem_arena_free(self._h, int(offset))
        if st != 0:
            raise binding.FemError("fem_arena_free", st, self._L.fem_last_error().decode())

    @property
    def free_bytes(self) -> int:
        return int(self._L.fem_arena_free_bytes(self._h))

    @property
    def largest_free(self) -> int:
        return int(self._L.fem_arena_largest_free(self._h))

    @property
    def capacity(self) -> int:
        return int(self._L.fem_arena_capacity(self._h))

    def __del__(self):
        try:
            if self._h:
                self._L.fem_arena_destroy(self._h)
                self._h = ctypes.c_void_p()
        except Exception:
            pass


# ----------------------------------------------------------------------------- native launch

SERVE_SLOTS = {"coords": 0, "conn": 1, "u": 2, "K": 3, "lam": 3, "mu": 4, "adj": 5, "out": 6, "dK": 6, "du": 7,
               "scratch": 8, "node_ptr": 9, "node_idx": 10, "work": 11}
KINDS = {"residual": 0, "adjoint": 1, "selftest": 2}
# error bits of a request's status word (the library's device error bits)
STATUS_TEXT = {1: "timeout: a bounded device-side wait gave up (outputs incomplete)",
               2: "bad mesh: a vertex id outside [0, n_verts) or a cell with det J = 0"}


class ServeRequestDesc(ctypes.Structure):
    """ctypes mirror of fem_serve_request (include/fem.h)."""

    _fields_ = [("kind", ctypes.c_int32), ("physics", ctypes.c_int32), ("dim", ctypes.c_int32),
                ("n_q", ctypes.c_int32), ("prec", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n_cells", ctypes.c_int64), ("n_verts", ctypes.c_int64),
                ("qpts", ctypes.c_void_p), ("qw", ctypes.c_void_p),
                ("host_in", ctypes.c_void_p), ("in_bytes", ctypes.c_int64),
                ("host_out", ctypes.c_void_p * 2), ("out_bytes", ctypes.c_int64 * 2),
                ("offset", ctypes.c_int64 * 12), ("block_bytes", ctypes.c_int64), ("host_status", ctypes.c_void_p)]


class ServeResult(ctypes.Structure):
    """ctypes mirror of fem_serve_result (include/fem.h)."""

    _fields_ = [("t_arrive", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("status", ctypes.c_int32), ("bits", ctypes.c_uint32)]


# fem_serve_result.status
NATIVE_STATUS = {0: "done", 1: "rejected", 2: "failed", 3: "failed"}


def _serve_lib():
    L = binding.lib()
    if not getattr(L, "_serve_ready", False):
        P = ctypes.c_void_p
        L.fem_serve_event_create.argtypes = [ctypes.POINTER(P)]
        L.fem_serve_event_create.restype = ctypes.c_int
        L.fem_serve_event_destroy.argtypes = [P]
        L.fem_serve_event_destroy.restype = None
        L.fem_serve_events_query.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.fem_serve_events_query.restype = ctypes.c_int
        L.fem_serve_launch.argtypes = [ctypes.POINTER(ServeRequestDesc), P, P, P]
        L.fem_serve_launch.restype = ctypes.c_int
        L.fem_serve_run.argtypes = [ctypes.POINTER(ServeRequestDesc), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_int, P, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_int, ctypes.POINTER(ServeResult)]
        L.fem_serve_run.restype = ctypes.c_int
        L.fem_serve_request_bytes.argtypes = []
        L.fem_serve_request_bytes.restype = ctypes.c_int64
        if L.fem_serve_request_bytes() != ctypes.sizeof(ServeRequestDesc):
            raise RuntimeError("fem_serve_request layout differs between libfem and this binding")
        L._serve_ready = True
    return L


# ----------------------------------------------------------------------------- requests


@dataclasses.dataclass
class Request:
    rid: int
    kind: str  # "residual" or "adjoint" (adjoint: Laplacian only)
    physics: str  # "laplacian" or "elasticity"
    dim: int
    n_cells: int
    n_verts: int
    qpts: np.ndarray
    qw: np.ndarray
    host: Dict[str, torch.Tensor]  # pinned inputs: coords, conn, u, K | lam, mu, adj
    prec: str = "mixed"
    arrival: float = 0.0  # seconds after the start of the stream
    status: str = "pending"
    t_arrive: float = math.nan
    t_admit: float = math.nan
    t_done: float = math.nan
    result: Dict[str, torch.Tensor] = dataclasses.field(default_factory=dict)
    error: str = ""
    _arrays: Optional[list] = dataclasses.field(default=None, repr=False, compare=False)
    _footprint: Optional[int] = dataclasses.field(default=None, repr=False, compare=False)
    host_block: Optional[torch.Tensor] = dataclasses.field(default=None, repr=False, compare=False)
    input_bytes: int = 0
    _offsets: Optional[dict] = dataclasses.field(default=None, repr=False, compare=False)
    desc: Optional[ServeRequestDesc] = dataclasses.field(default=None, repr=False, compare=False)
    # page-locked word the request's kernels report their error bits into (zeroed before
    # each launch, read after completion); status_np is a numpy view of it (cheap to read)
    status_host: Optional[torch.Tensor] = dataclasses.field(default=None, repr=False, compare=False)
    status_np: Optional[np.ndarray] = dataclasses.field(default=None, repr=False, compare=False)

    def build_desc(self) -> ServeRequestDesc:
        """The request as the native launcher sees it (built once; the tensors it points
        into are owned by the request)."""
        d = ServeRequestDesc()
        d.kind = KINDS[self.kind]
        d.physics = 0 if self.physics == "laplacian" else 1
        d.dim, d.n_q, d.prec = self.dim, int(self.qw.shape[0]), binding.precision(self.prec)
        d.n_cells, d.n_verts = self.n_cells, self.n_verts
        d.qpts, d.qw = self.qpts.ctypes.data, self.qw.ctypes.data
        d.host_in = self.host_block.data_ptr() if self.host_block is not None else None
        d.in_bytes = self.input_bytes
        outs = {"residual": ["out"], "adjoint": ["dK", "du"], "selftest": []}[self.kind]
        for k, name in enumerate(outs):
            t = self.result[name]
            d.host_out[k] = t.data_ptr() if t.numel() else None
            d.out_bytes[k] = t.numel() * t.element_size()
        for name, off in self.offsets().items():
            d.offset[SERVE_SLOTS[name]] = off
        d.block_bytes = footprint(self)
        if self.status_host is None:
            self.status_host = torch.zeros(1, dtype=torch.int32, pin_memory=True)
            self.status_np = self.status_host.numpy()
        d.host_status = self.status_host.data_ptr()
        self.desc = d
        return d

    def device_status(self) -> int:
        """Error bits the request's kernels reported (valid once it has completed)."""
        return 0 if self.status_np is None else int(self.status_np[0])

    @property
    def n_comp(self) -> int:
        return 1 if self.physics == "laplacian" else self.dim

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrive

    def device_arrays(self):
        """(name, shape, dtype) of every device array the request needs (computed once)."""
        if self._arrays is None:
            self._arrays = self._device_arrays()
        return self._arrays

    def offsets(self) -> Dict[str, int]:
        """Byte offset of every array inside the request's device block (computed once)."""
        if self._offsets is None:
            off, self._offsets = 0, {}
            for name, shape, dt in self.device_arrays():
                self._offsets[name] = off
                off += (_nbytes(shape, dt) + ALIGN - 1) // ALIGN * ALIGN
        return self._offsets

    def _device_arrays(self):
        if self.kind == "selftest":
            return [("scratch", (1,), torch.int32)]  # no arrays used: a minimal arena block
        d, C, V, nq = self.dim, self.n_cells, self.n_verts, int(self.qw.shape[0])
        dt = value_dtype(self.prec)
        arrs = [("coords", (d, V), torch.float64), ("conn", (d + 1, C), torch.int32),
                ("u", (V,) if self.physics == "laplacian" else (d, V), dt)]
        if self.physics == "laplacian":
            arrs.append(("K", (nq, C), dt))
        else:
            arrs += [("lam", (nq, C), dt), ("mu", (nq, C), dt)]
        if self.kind == "residual":
            arrs.append(("out", ((d + 1) * self.n_comp, C), dt))
        else:
            arrs += [("adj", (d + 1, C), dt), ("dK", (nq, C), dt), ("du", (V,), dt), ("scratch", (d + 1, C), dt),
                     ("node_ptr", (V + 1,), torch.int32), ("node_idx", ((d + 1) * C,), torch.int32),
                     ("work", (max(1, binding.lib().fem_node2cell_work_size(V)),), torch.int32)]
        return arrs

    def alloc_results(self):
        dt = value_dtype(self.prec)
        d, C, V, nq = self.dim, self.n_cells, self.n_verts, int(self.qw.shape[0])
        if self.kind == "selftest":
            self.result = {}
        elif self.kind == "residual":
            self.result = {"out": torch.empty(((d + 1) * self.n_comp, C), dtype=dt, pin_memory=True)}
        else:
            self.result = {"dK": torch.empty((nq, C), dtype=dt, pin_memory=True),
                           "du": torch.empty(V, dtype=dt, pin_memory=True)}


_ELEMENT_BYTES = {torch.float64: 8, torch.float32: 4, torch.int32: 4, torch.uint8: 1}


def _nbytes(shape, dtype) -> int:
    n = 1
    for s in shape:
        n *= int(s)
    return n * _ELEMENT_BYTES[dtype]


def footprint(req: Request) -> int:
    """Device bytes of a request: every array rounded up to the 256-byte alignment
    (computed once per request)."""
    if req._footprint is None:
        req._footprint = sum((_nbytes(s, t) + ALIGN - 1) // ALIGN * ALIGN for _, s, t in req.device_arrays())
    return req._footprint


def make_request(rid, case, kind, prec="mixed", arrival=0.0, adj=None) -> Request:
    """A request from a workloads.Case (values rounded to the precision's storage type).
    Its inputs live in one pinned host block laid out like the leading (input) part of
    the request's device block, so admission uploads them with a single copy."""
    dt = value_dtype(prec)
    c = case if prec == "fp64" else case.rounded_to_f32()
    if kind == "adjoint" and c.physics != "laplacian":
        raise ValueError("adjoint requests are Laplacian only")
    values = {"coords": c.mesh.coords, "conn": c.mesh.conn, "u": c.u}
    if c.physics == "laplacian":
        values["K"] = c.K
    else:
        values["lam"], values["mu"] = c.lam, c.mu
    if kind == "adjoint":
        values["adj"] = c.adj if adj is None else adj
    r = Request(rid, kind, c.physics, c.dim, c.n_cells, c.n_verts, np.ascontiguousarray(c.rule.points),
                np.ascontiguousarray(c.rule.weights), {}, prec=prec, arrival=arrival)
    layout = r.device_arrays()[:len(values)]
    assert [name for name, _, _ in layout] == list(values), "inputs lead the device layout"
    r.input_bytes = sum((_nbytes(sh, t) + ALIGN - 1) // ALIGN * ALIGN for _, sh, t in layout)
    r.host_block = torch.empty(max(1, r.input_bytes), dtype=torch.uint8, pin_memory=True)
    off = 0
    for name, shape, t in layout:
        nb = _nbytes(shape, t)
        view = r.host_block[off:off + nb].view(t).view(shape)
        view.copy_(torch.from_numpy(np.ascontiguousarray(values[name])).to(t))
        r.host[name] = view
        off += (nb + ALIGN - 1) // ALIGN * ALIGN
    r.alloc_results()
    r.build_desc()
    return r


def make_selftest_request(rid, arrival=0.0) -> Request:
    """A request whose only kernel is the bounded-wait self-test (a wait that nothing
    completes, given up after 1 ms): it always comes back failed with the timeout bit, and
    the requests around it are unaffected. For tests of the failure path."""
    r = Request(rid, "selftest", "laplacian", 3, 0, 0, np.zeros((1, 3)), np.ones(1), {}, prec="mixed",
                arrival=arrival)
    r.input_bytes = 0
    r.alloc_results()
    r.build_desc()
    return r


# ----------------------------------------------------------------------------- executor


class GpuExecutor:
    """Runs admitted requests: one CUDA stream and one completion event per slot; each
    request's arrays sit in one arena block of the preallocated buffer, and its launch is
    one native call. Nothing is allocated per request."""

    def __init__(self, device="cuda", capacity: int = 4 << 30, n_slots: int = 8, nvtx: bool = False):
        self.device = torch.device(device)
        self.nvtx = nvtx  # an NVTX range per request launch (for a timeline profiler)
        self.pool = torch.empty(int(capacity), dtype=torch.uint8, device=self.device)
        self.arena = Arena(capacity)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_slots)]
        self.free_slots = list(range(n_slots))
        self.inflight: Dict[int, tuple] = {}  # rid -> (req, slot, offsets, event)
        self.launches = 0
        self.capacity = self.arena.capacity
        self.pool_ptr = self.pool.data_ptr()
        self._L = _serve_lib()
        self.events = []
        for _ in range(n_slots):  # one completion event per slot, reused
            e = ctypes.c_void_p()
            st = self._L.fem_serve_event_create(ctypes.byref(e))
            if st != 0:
                raise binding.FemError("fem_serve_event_create", st, self._L.fem_last_error().decode())
            self.events.append(e)

    @property
    def n_slots(self) -> int:
        return len(self.streams)

    def fits_ever(self, req: Request) -> bool:
        return footprint(req) <= self.capacity

    def full(self) -> bool:
        """No free slot: nothing can be admitted until a request completes."""
        return not self.free_slots

    def try_admit(self, req: Request):
        if not self.free_slots:
            return None
        # one arena block per request, its arrays at 256-byte boundaries (Request.offsets)
        base = self.arena.alloc(footprint(req))
        if base is None:
            return None
        return self.free_slots.pop(), [base], base

    def launch(self, req: Request, admitted) -> None:
        """Upload, kernels, download and completion event of one request on its slot's
        stream: one native call (fem_serve_launch) with pointers into the request's block."""
        slot, offs, base = admitted
        desc = req.desc if req.desc is not None else req.build_desc()
        req.status_np[0] = 0  # the kernels only set bits
        if self.nvtx:
            torch.cuda.nvtx.range_push(f"{req.kind} {req.physics}{req.dim}d rid={req.rid} cells={req.n_cells}")
        st = self._L.fem_serve_launch(ctypes.byref(desc), ctypes.c_void_p(self.pool_ptr + base), self.events[slot],
                                      ctypes.c_void_p(self.streams[slot].cuda_stream))
        if self.nvtx:
            torch.cuda.nvtx.range_pop()
        if st != 0:
            self.arena.free(base)
            self.free_slots.append(slot)
            raise binding.FemError("fem_serve_launch", st, self._L.fem_last_error().decode())
        # residual: 1 kernel; adjoint: list build (7 kernels) + element + gather; self-test: 1
        self.launches += 9 if req.kind == "adjoint" else 1
        self.inflight[req.rid] = (req, slot, offs, None)

    def poll(self) -> List[Request]:
        if not self.inflight:
            return []
        rids = list(self.inflight)
        n = len(rids)
        evs = (ctypes.c_void_p * n)(*[self.events[self.inflight[r][1]] for r in rids])
        done = (ctypes.c_int * n)()
        st = self._L.fem_serve_events_query(evs, n, done)
        if st != 0:
            raise binding.FemError("fem_serve_events_query", st, self._L.fem_last_error().decode())
        out = []
        for k, rid in enumerate(rids):
            if done[k]:
                req, slot, offs, _ = self.inflight.pop(rid)
                for o in offs:
                    self.arena.free(o)
                self.free_slots.append(slot)
                bits = req.device_status()
                if bits:
                    req.error = "; ".join(t for b, t in STATUS_TEXT.items() if bits & b) or f"device error bits {bits}"
                out.append(req)
        return out

    def __del__(self):
        try:
            for e in getattr(self, "events", []):
                self._L.fem_serve_event_destroy(e)
        except Exception:
            pass

    def busy(self) -> bool:
        return bool(self.inflight)


# ----------------------------------------------------------------------------- scheduler


@dataclasses.dataclass
class ServeStats:
    n: int
    n_done: int
    n_rejected: int
    n_failed: int
    makespan_s: float
    cells: int
    cells_per_s: float
    req_per_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    max_inflight: int
    arrival_rate: float

    def as_dict(self):
        return dataclasses.asdict(self)


class Scheduler:
    """Real-time continuous batching: requests join a FIFO queue when their arrival time
    passes and are admitted whenever a slot and enough arena memory are free; with
    backfill, a later request that fits may overtake a head that does not."""

    def __init__(self, executor, backfill: bool = True, clock=time.perf_counter, idle_sleep: float = 0.0):
        self.ex = executor
        self.backfill = backfill
        self.clock = clock
        self.idle_sleep = idle_sleep

    def run(self, requests: List[Request], arrival_rate: float = math.nan) -> ServeStats:
        # a real-time loop: Python's cyclic garbage collector is paused while it runs (its
        # full passes over a large heap would stall admissions for milliseconds)
        gc_was_enabled = gc.isenabled()
        gc.collect()
        gc.disable()
        try:
            return self._run(requests, arrival_rate)
        finally:
            if gc_was_enabled:
                gc.enable()

    def _run(self, requests: List[Request], arrival_rate: float) -> ServeStats:
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue: collections.deque = collections.deque()
        n, finished, max_inflight = len(requests), 0, 0
        full = getattr(self.ex, "full", None)
        t0 = self.clock()
        while finished < n:
            now = self.clock()
            while pending and pending[0].arrival <= now - t0:
                r = pending.popleft()
                r.t_arrive = t0 + r.arrival
                if not self.ex.fits_ever(r):  # can never run: rejected on arrival
                    r.status, r.error = "rejected", "footprint exceeds the device arena"
                    r.t_done = self.clock()
                    finished += 1
                    continue
                r.status = "queued"
                queue.append(r)
            progressed = False
            i = 0
            while i < len(queue):
                if full is not None and full():
                    break  # no slot: no request in the queue can be admitted now
                r = queue[i]
                adm = self.ex.try_admit(r)
                if adm is not None:
                    del queue[i]
                    r.t_admit = self.clock()
                    r.status = "running"
                    self.ex.launch(r, adm)
                    progressed = True
                    continue
                if not self.backfill:
                    break
                i += 1
            max_inflight = max(max_inflight, len(getattr(self.ex, "inflight", ())))
            for r in self.ex.poll():
                r.t_done = self.clock()
                r.status = "failed" if r.error else "done"
                finished += 1
                progressed = True
            if not progressed:
                if pending and not queue and not self.ex.busy():
                    wait = pending[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 1e-3))
                elif self.idle_sleep > 0:
                    time.sleep(self.idle_sleep)
                # idle_sleep = 0: poll again at once (a short sleep costs the timer slack,
                # ~50 us on Linux, on every completion)
        return _stats(requests, self.clock() - t0, arrival_rate, max_inflight)


class NativeScheduler:
    """The same scheduling as Scheduler (FIFO by arrival, admission when a slot and arena
    memory are free, optional backfill), run as one native call (fem_serve_run) over the
    whole stream: the host does no per-request work in Python. Uses the executor's device
    pool and slot count; the call creates its own streams and events and its own arena over
    the pool, so the executor must have nothing in flight."""

    def __init__(self, executor, backfill: bool = True):
        self.ex = executor
        self.backfill = backfill
        self._L = _serve_lib()

    def run(self, requests: List[Request], arrival_rate: float = math.nan) -> ServeStats:
        if getattr(self.ex, "inflight", None):
            raise RuntimeError("the executor has requests in flight")
        n = len(requests)
        descs = (ServeRequestDesc * max(1, n))()
        foot = (ctypes.c_int64 * max(1, n))()
        arr = (ctypes.c_double * max(1, n))()
        for k, r in enumerate(requests):
            descs[k] = r.desc if r.desc is not None else r.build_desc()
            foot[k] = footprint(r)
            arr[k] = float(r.arrival)
        res = (ServeResult * max(1, n))()
        st = self._L.fem_serve_run(descs, foot, arr, n, ctypes.c_void_p(self.ex.pool_ptr), self.ex.capacity, ALIGN,
                                   self.ex.n_slots, 1 if self.backfill else 0, res)
        if st != 0:
            raise binding.FemError("fem_serve_run", st, self._L.fem_last_error().decode())
        # the loop's own clock starts after its streams are made: place it at the end of the call
        span = max((res[k].t_done for k in range(n)), default=0.0)
        base = time.perf_counter() - span
        at = lambda x: math.nan if x < 0 else base + x
        for k, r in enumerate(requests):
            x = res[k]
            r.t_arrive, r.t_admit, r.t_done = at(x.t_arrive), at(x.t_admit), at(x.t_done)
            r.status = NATIVE_STATUS.get(x.status, "failed")
            r.error = ""
            if x.status == 1:
                r.error = "footprint exceeds the device arena"
            elif x.status == 2:
                bits = int(x.bits)
                r.error = "; ".join(t for b, t in STATUS_TEXT.items() if bits & b) or f"device error bits {bits}"
            elif x.status == 3:
                r.error = "launch refused (argument error)"
        # most requests in flight at once, from the admission and completion times
        ev = sorted([(x.t_admit, 1) for x in res[:n] if x.t_admit >= 0] +
                    [(x.t_done, -1) for x in res[:n] if x.t_admit >= 0])
        cur = peak = 0
        for _, d in ev:
            cur += d
            peak = max(peak, cur)
        return _stats(requests, span, arrival_rate, max_inflight=peak)


def _stats(requests, span, arrival_rate, max_inflight) -> ServeStats:
    n = len(requests)
    done = [r for r in requests if r.status == "done"]
    lat = sorted(r.latency * 1e3 for r in done) or [math.nan]
    cells = sum(r.n_cells for r in done)

    def pct(p):
        k = max(0, min(len(lat) - 1, int(math.ceil(p / 100.0 * len(lat))) - 1))
        return lat[k]

    return ServeStats(n=n, n_done=len(done), n_rejected=sum(r.status == "rejected" for r in requests),
                      n_failed=sum(r.status == "failed" for r in requests),
                      makespan_s=span, cells=cells, cells_per_s=cells / span if span > 0 else math.nan,
                      req_per_s=len(done) / span if span > 0 else math.nan, p50_ms=pct(50), p99_ms=pct(99),
                      mean_ms=statistics.mean(lat) if done else math.nan, max_inflight=max_inflight,
                      arrival_rate=arrival_rate)


def request_log(requests, t0: float = None) -> List[dict]:
    """The served stream as plain records (arrival, admission and completion times in s
    from the first arrival, status, size), for saving beside a run and replaying it."""
    reqs = list(requests)
    if t0 is None:
        t0 = min((r.t_arrive for r in reqs if not math.isnan(r.t_arrive)), default=0.0)
    rel = lambda t: None if t is None or math.isnan(t) else t - t0
    return [{"rid": r.rid, "kind": getattr(r, "kind", None), "physics": getattr(r, "physics", None),
             "n_cells": r.n_cells, "arrival": r.arrival, "t_arrive": rel(r.t_arrive), "t_admit": rel(r.t_admit),
             "t_done": rel(r.t_done), "status": r.status, "error": r.error} for r in reqs]


def save_request_log(path: str, requests) -> None:
    import json

    with open(path, "w") as f:
        json.dump(request_log(requests), f)


def replay_arrivals(path: str, requests) -> None:
    """Set each request's arrival time from a saved log (matched by rid), so the same
    stream can be served again."""
    import json

    with open(path) as f:
        arrivals = {rec["rid"]: rec["arrival"] for rec in json.load(f)}
    for r in requests:
        if r.rid in arrivals:
            r.arrival, r.status = float(arrivals[r.rid]), "pending"


def poisson_arrivals(n: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps of mean 1/rate."""
    rng = np.random.Generator(np.random.Philox(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=n)) if rate > 0 else np.zeros(n)

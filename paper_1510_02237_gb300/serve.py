"""Continuous-batching request loop for KSE-Parareal solves on one GPU.

Requests (an initial value, a problem and K) arrive over time.  A request is
admitted as soon as a solver slot for its problem shape is free, or can be
created within the device-memory budget (slot footprint from
``parareal_footprint_bytes``: iterates, fine images and the Krylov basis),
the in-flight limit and the SM budget (the grid-synchronised kernels of the
solves in flight, each on its slot's SM limit, fit on the GPU side by side).
Every completed solve's handle is asked whether a device-side wait gave up
(counted in ``device_errors``).  Each slot owns a solver handle with its own CUDA
stream, device input/output buffers and pinned host staging buffers, so
admitted requests run side by side on the device while later ones keep
arriving.  A request's latency runs from its arrival to the moment its
result is back in host memory.

All computation happens in the library's kernels; this module only
schedules, and it allocates only when it creates a slot.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import (PR_FP32, PR_FP32X, PR_FP64, PR_PROJ_SPLIT_BF16, PararealError, Solver, new_stream,
               parareal_autotune, parareal_footprint_bytes, parareal_solve, parareal_status)


@dataclass
class Result:
    index: int
    arrival: float
    admitted: float
    done: float
    qT: np.ndarray

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Slot:
    key: tuple
    solver: Solver
    stream: object
    u0_dev: object
    qT_dev: object
    u0_host: object
    qT_host: object
    bytes: int
    sms: int = 0            # SMs its grid-synchronised kernels use
    busy: bool = False


@dataclass
class ServeStats:
    completed: int = 0
    makespan_s: float = 0.0
    peak_inflight: int = 0
    peak_bytes: int = 0
    slots_created: int = 0
    device_errors: int = 0   # completed solves whose handle reported a device-side wait that gave up
    latencies_s: list = field(default_factory=list)

    def summary(self) -> dict:
        lat = np.array(self.latencies_s) * 1e3
        return {"completed": self.completed, "solves_per_s": self.completed / max(self.makespan_s, 1e-9),
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "mean_ms": float(lat.mean()) if len(lat) else None, "makespan_s": self.makespan_s,
                "peak_inflight": self.peak_inflight, "peak_device_bytes": self.peak_bytes,
                "slots_created": self.slots_created, "device_errors": self.device_errors}


def default_sm_limit(d: int, sms: int) -> int:
    """SMs for a handle's grid-synchronised kernels: about one SM per 2048
    state values (at least 4), so small problems leave room for others.  On a
    saturated request stream (grids 64x32..512x256) this served 3-5 % more
    solves/s than one SM per 4096 values (more solves side by side, each on
    fewer SMs) and 10-12 % more than one per 8192."""
    return int(max(4, min(sms, d // 2048)))


def batch_sm_limit(d: int, sms: int) -> int:
    """SMs per instance when a known batch of solves runs as one graph: the
    request loop's share (64 uneven instances: 0.93 s against 1.05 s with one
    SM per 4096 state values; one per 1024, or shares proportional to each
    instance's fine work, were 1.0-1.04 s)."""
    return default_sm_limit(d, sms)


class Server:
    """Admit, run and complete requests; see the module docstring."""

    def __init__(self, budget_bytes: float = 150e9, max_inflight: int = 16, mode: str = "mixed",
                 sm_limit=default_sm_limit, autotune: bool = True, sms: int | None = None):
        """sms: the SM count the admission shares out (default: the current
        device's)."""
        import torch
        if mode not in self.MODES:
            raise ValueError(f"mode must be one of {self.MODES}")
        self.torch = torch
        self.budget = float(budget_bytes)
        self.max_inflight = int(max_inflight)
        self.mode = mode
        self.sm_limit = sm_limit
        self.autotune = autotune
        self.sms = int(sms) if sms else \
            torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        self.slots = collections.defaultdict(list)
        self.bytes = 0

    # ---------------------------------------------------------------- slots
    MODES = ("fp64", "fp64_tc", "mixed")

    def solver_options(self, p) -> dict:
        """Options of the handles this server creates for problem p (also what
        reproduces a served result with a handle of one's own).

        mode 'fp64': plain FP64.  'fp64_tc': FP64 fine sweep and correction,
        the subspace products Q^T V and V - Q C (and the image update
        Z - D C) on the BF16 tensor cores with FP32 accumulation and exact
        split digits (FP64-accurate, so the final
        accuracy equals the plain FP64 solve's).  'mixed': additionally FP32
        tendencies in the fine sweep and an FP32 correction (fastest; its
        accuracy depends on the input's conditioning)."""
        opt = {}
        if self.mode == "mixed":
            opt.update(fine_prec=PR_FP32X, corr_prec=PR_FP32)
        if self.mode in ("mixed", "fp64_tc") and (3 * p.nx * p.ny) % 8 == 0:
            opt.update(proj_prec=PR_PROJ_SPLIT_BF16)
        if self.sm_limit:
            opt["sm_limit"] = self.sm_limit(p.d, self.sms)
        return opt

    def _options(self, p, K_max):
        return dict(self.solver_options(p), K_max=K_max)

    def _key(self, inst):
        p = inst.problem
        return (p.nx, p.ny, p.n_slices, p.n_f, p.n_g, p.U, p.V, p.c_s, p.nu_f, p.nu_c, p.n_sound)

    def _acquire(self, inst, inflight: int, sms_used: int = 0):
        if inflight >= self.max_inflight:
            return None
        # SM admission: the grid-synchronised kernels of all solves in flight
        # fit on the GPU side by side
        p = inst.problem
        need = self.solver_options(p).get("sm_limit", 0) or self.sms
        if inflight and sms_used + need > self.sms:
            return None
        key = self._key(inst)
        for s in self.slots[key]:
            if not s.busy:
                return s
        K_max = min(p.n_slices, 8)
        opt = self._options(p, K_max)
        nbytes = parareal_footprint_bytes(p.nx, p.ny, p.n_slices, **opt)
        if self.bytes + nbytes > self.budget:
            self._evict(nbytes)
            if self.bytes + nbytes > self.budget:
                return None
        torch = self.torch
        stream = new_stream()
        solver = Solver(p, stream=stream, **opt)
        if self.autotune:   # fine-step launch shape, timed once per problem shape (cached)
            parareal_autotune(solver.h)
        slot = _Slot(key, solver, stream, torch.empty(p.d, dtype=torch.float64, device="cuda"),
                     torch.empty(p.d, dtype=torch.float64, device="cuda"),
                     torch.empty(p.d, dtype=torch.float64).pin_memory(),
                     torch.empty(p.d, dtype=torch.float64).pin_memory(), nbytes, need)
        self.slots[key].append(slot)
        self.bytes += nbytes
        self.stats.slots_created += 1
        return slot

    def _evict(self, need: int):
        """Free idle slots (largest first) until `need` more bytes fit."""
        idle = [s for v in self.slots.values() for s in v if not s.busy]
        idle.sort(key=lambda s: -s.bytes)
        for s in idle:
            if self.bytes + need <= self.budget:
                break
            s.solver.close()
            self.slots[s.key].remove(s)
            self.bytes -= s.bytes

    def close(self):
        for v in self.slots.values():
            for s in v:
                s.solver.close()
        self.slots.clear()
        self.bytes = 0

    # ---------------------------------------------------------------- loop
    def run(self, requests, realtime: bool = True):
        """Serve a list of (arrival_s, Instance).  Returns (results, stats)."""
        torch = self.torch
        self.stats = ServeStats()
        order = sorted(range(len(requests)), key=lambda i: requests[i][0])
        pending = collections.deque(order)
        waiting = collections.deque()
        inflight = []
        results = [None] * len(requests)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0 if realtime else float("inf")
        while pending or waiting or inflight:
            t = now()
            while pending and requests[pending[0]][0] <= t:
                waiting.append(pending.popleft())
            # completions
            still = []
            for (i, slot, ev, t_adm) in inflight:
                if ev.query():
                    t_done = now() if realtime else 0.0
                    try:
                        parareal_status(slot.solver.h)   # the stream is idle: no wait
                    except PararealError:
                        self.stats.device_errors += 1
                    results[i] = Result(i, requests[i][0], t_adm, t_done, slot.qT_host.numpy().copy())
                    slot.busy = False
                    self.stats.completed += 1
                    self.stats.latencies_s.append(t_done - requests[i][0])
                else:
                    still.append((i, slot, ev, t_adm))
            inflight = still
            # admissions in arrival order (a request that does not fit waits)
            while waiting:
                i = waiting[0]
                inst = requests[i][1]
                slot = self._acquire(inst, len(inflight), sum(sl.sms for (_, sl, _, _) in inflight))
                if slot is None:
                    break
                waiting.popleft()
                slot.busy = True
                q0 = inst.initial_value().ravel()
                slot.u0_host.numpy()[:] = q0
                with torch.cuda.stream(slot.stream):
                    slot.u0_dev.copy_(slot.u0_host, non_blocking=True)
                parareal_solve(slot.solver.h, slot.u0_dev, inst.K, qT=slot.qT_dev, report=False)
                with torch.cuda.stream(slot.stream):
                    slot.qT_host.copy_(slot.qT_dev, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(slot.stream)
                inflight.append((i, slot, ev, now() if realtime else 0.0))
            self.stats.peak_inflight = max(self.stats.peak_inflight, len(inflight))
            self.stats.peak_bytes = max(self.stats.peak_bytes, self.bytes)
            if not inflight and not waiting and pending and realtime:
                time.sleep(max(0.0, min(0.01, requests[pending[0]][0] - now())))
            elif inflight:
                time.sleep(0.0002)
        self.stats.makespan_s = time.perf_counter() - t0
        return results, self.stats

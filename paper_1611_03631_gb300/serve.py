"""Continuous-batching server of robot mapping sessions on one GPU.

Each session is a robot that streams posed scans at its own rate and, after every scan, asks
for distances and gradients at a batch of points near its trajectory (the planner's query of
the paper's Sec. VII). The server keeps every admitted session's TSDF/ESDF map resident on the
device and advances all sessions that have a scan waiting with one batched step
(``vbx_batch_step``): a request that arrives while the GPU works joins the next step, so the
batch changes from step to step (continuous batching). Sessions are admitted in arrival order
when a slot is free and their map fits the device-memory budget; a finished session's map is
reset and reused by the next session of the same kind, or freed to make room for another kind.

The per-map arithmetic does not depend on which other maps share a step, so a session's map
and query results are the same alone and in the mix.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from . import vbx


@dataclasses.dataclass
class SessionSpec:
    sid: int
    kind: str  # key of the scan pool
    seq: int  # sequence index inside the pool kind
    offset: int  # first frame of the sequence
    n_scans: int
    rate_hz: float
    start: float  # arrival time of the session (s since the run started)


def poisson_sessions(
    n: int,
    kinds: List[str],
    seqs_per_kind: Dict[str, int],
    frames_per_seq: Dict[str, int],
    sessions_per_s: float,
    scans_per_session: int,
    rate_range=(10.0, 30.0),
    seed: int = 5,
) -> List[SessionSpec]:
    """Sessions arriving as a Poisson process, each streaming scans at U(rate_range) Hz."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / sessions_per_s))
        kind = kinds[int(rng.integers(0, len(kinds)))]
        out.append(
            SessionSpec(
                sid=i,
                kind=kind,
                seq=int(rng.integers(0, seqs_per_kind[kind])),
                offset=int(rng.integers(0, frames_per_seq[kind])),
                n_scans=scans_per_session,
                rate_hz=float(rng.uniform(*rate_range)),
                start=t,
            )
        )
    return out


class ScanPool:
    """Pre-generated scan sequences per kind, resident in device memory, with a query batch of
    points within `radius` of the sensor for every frame."""

    def __init__(self, sets_by_kind: Dict[str, list], n_queries: int, radius: float = 2.0, seed: int = 9):
        import torch

        from . import scenes

        self.kinds = list(sets_by_kind)
        self.params = {k: dict(v[0].params) for k, v in sets_by_kind.items()}
        self.points, self.poses, self.queries = {}, {}, {}
        self.n_queries = n_queries
        for k, sets in sets_by_kind.items():
            self.points[k] = [[torch.from_numpy(p).cuda() for p in s.points] for s in sets]
            self.poses[k] = [[np.asarray(T, np.float32) for T in s.poses] for s in sets]
            self.queries[k] = [
                [
                    torch.from_numpy(scenes.random_queries(s, n_queries, radius=radius, seed=seed + 31 * j + f, scan_index=f)).cuda()
                    for f in range(len(s.points))
                ]
                for j, s in enumerate(sets)
            ]

    def frames(self, kind: str) -> int:
        return len(self.poses[kind][0])

    def frame(self, spec: SessionSpec, k: int):
        f = (spec.offset + k) % len(self.poses[spec.kind][spec.seq])
        return self.points[spec.kind][spec.seq][f], self.poses[spec.kind][spec.seq][f], self.queries[spec.kind][spec.seq][f]


def scratch_for_pool(pool: ScanPool, capacity: Dict[str, int], margin: float = 1.1) -> Dict[str, int]:
    """Scratch blocks per scan kind: the most blocks any scan of the pool enters, times
    `margin`. The rays of a scan enter the same blocks whatever the map already holds (every
    block a ray crosses is allocated), so one pass over the pool's scans measures it."""
    out = {}
    for kind in pool.kinds:
        p = pool.params[kind]
        pts = max(int(t.shape[0]) for seq in pool.points[kind] for t in seq)
        need = 0
        for seq, poses in zip(pool.points[kind], pool.poses[kind]):
            m = vbx.Map.from_scene_params(p, block_capacity=capacity.get(kind, 0), max_points=pts)
            for x, T in zip(seq, poses):
                m.integrate_scan(x, T)
                need = max(need, int(m.stats()["touched_blocks"]))
            m.close()
        out[kind] = int(need * margin) + 1
    return out


@dataclasses.dataclass
class _Active:
    spec: SessionSpec
    m: vbx.Map
    arrivals: np.ndarray
    next: int = 0


class MapServer:
    def __init__(
        self,
        pool: ScanPool,
        slots: int = 128,
        hbm_budget: float = 120e9,
        capacity: Optional[Dict[str, int]] = None,
        use_graph: bool = True,
        scratch: Optional[Dict[str, int]] = None,
        prealloc=None,
    ):
        import torch

        self.pool = pool
        self.slots = slots
        self.budget = float(hbm_budget)
        self.capacity = capacity or {}
        # blocks one scan of a kind may enter (its per-voxel sums live there); 0: the pool size
        self.scratch = scratch or {}
        self.use_graph = use_graph
        self.used = 0
        self.peak = 0
        self.free: Dict[str, List[vbx.Map]] = collections.defaultdict(list)
        # idle placeholder maps keep unbound slots valid (a slot always holds a map)
        self.idle = [vbx.Map(0.5, 4, 0.5, 1.0, block_capacity=8, max_points=1024) for _ in range(slots)]
        self.batch = vbx.MapBatch(self.idle, max_queries=pool.n_queries)
        # warm pool: maps created before the run (creation allocates and synchronises the
        # device, which would stall the step loop); they count against the budget.
        # prealloc = {kind: count}, or "fill": an equal share of the budget per kind, at most
        # one map per slot
        if prealloc == "fill":
            share = self.budget / max(len(pool.kinds), 1)
            prealloc = {k: min(slots, int(share // self.map_bytes(k))) for k in pool.kinds}
        for kind, n in (prealloc or {}).items():
            for _ in range(n):
                need = self.map_bytes(kind)
                if self.used + need > self.budget:
                    break
                try:
                    m = self._new_map(kind)
                except vbx.VbxError as e:  # the device has less free memory than the budget
                    if e.status != 2:
                        raise
                    break
                self.used += m.device_bytes()
                self.peak = max(self.peak, self.used)
                self.free[kind].append(m)
        # the batch's ESDF work lists are sized by the maps bound to it: bind the warm maps (the
        # largest first) to the slots once now, so that admissions during the run do not have to
        # grow them (growing them synchronises the device)
        spare = sorted((m for ms in self.free.values() for m in ms), key=lambda m: -m.device_bytes())[:slots]
        for slot, m in enumerate(spare):
            self.batch.bind(slot, m)
        for slot in range(len(spare)):
            self.batch.bind(slot, self.idle[slot])
        q = pool.n_queries
        self.out = [
            (
                torch.empty(q, dtype=torch.float32, device="cuda"),
                torch.empty((q, 3), dtype=torch.float32, device="cuda"),
                torch.empty(q, dtype=torch.uint8, device="cuda"),
            )
            for _ in range(slots)
        ]

    # ----------------------------------------------------------------------- memory
    def _new_map(self, kind: str) -> vbx.Map:
        p = self.pool.params[kind]
        pts = max(int(t.shape[0]) for seq in self.pool.points[kind] for t in seq)
        return vbx.Map.from_scene_params(
            p, block_capacity=self.capacity.get(kind, 0), max_points=pts, scratch_blocks=self.scratch.get(kind, 0)
        )

    def map_bytes(self, kind: str) -> int:
        p = self.pool.params[kind]
        pts = max(int(t.shape[0]) for seq in self.pool.points[kind] for t in seq)
        return vbx.map_bytes(int(p["voxels_per_block"]), self.capacity.get(kind, 0), pts, self.scratch.get(kind, 0))

    def _acquire(self, kind: str) -> Optional[vbx.Map]:
        if self.free[kind]:
            m = self.free[kind].pop()
            m.reset()
            return m
        need = self.map_bytes(kind)
        for other in list(self.free):
            while other != kind and self.free[other] and self.used + need > self.budget:
                m = self.free[other].pop()
                self.used -= m.device_bytes()
                m.close()
        if self.used + need > self.budget:
            return None
        try:
            m = self._new_map(kind)
        except vbx.VbxError as e:  # out of device memory below the budget: the session waits
            if e.status != 2:
                raise
            return None
        self.used += m.device_bytes()
        self.peak = max(self.peak, self.used)
        return m

    def close(self) -> None:
        self.batch.close()
        for ms in self.free.values():
            for m in ms:
                m.close()
        self.free.clear()

    # -------------------------------------------------------------------------- run
    def run(self, sessions: List[SessionSpec], **kw) -> Dict[str, object]:
        """Serves `sessions` (see _serve for the keyword arguments). Python's cyclic garbage
        collector is paused meanwhile: its collections stall the host loop for milliseconds,
        which scans waiting for their step would see as latency."""
        import gc

        enabled = gc.isenabled()
        gc.disable()
        try:
            return self._serve(sessions, **kw)
        finally:
            if enabled:
                gc.enable()

    def _serve(
        self,
        sessions: List[SessionSpec],
        seed: int = 7,
        on_finish: Optional[Callable[[SessionSpec, vbx.Map, tuple], None]] = None,
        time_limit: float = 600.0,
        max_in_flight: int = 2,
        profile_steps: bool = False,
    ) -> Dict[str, object]:
        """Serves `sessions` to completion. Steps are issued without waiting for the previous
        ones: up to `max_in_flight` server steps (each a map step and a query step, on one
        stream, so a session's consecutive scans stay in order) are on the GPU while the host
        admits sessions and forms the next batch. A step's completion is seen by polling its
        events; a scan's latency runs from its arrival to the host time at which the end of its
        step's map part was first seen, a query's to the end of the query part.
        profile_steps: a diagnostic pass instead, with direct (non-graph) launches and per-kernel
        device times of every step (one step at a time)."""
        import torch

        if profile_steps:
            max_in_flight = 1
        rng = np.random.default_rng(seed)
        waiting = collections.deque(sorted(sessions, key=lambda s: s.start))
        active: Dict[int, _Active] = {}
        free_slots = list(range(self.slots))[::-1]
        graph = 0 if (profile_steps or not self.use_graph) else vbx.STEP_GRAPH
        flags_map = vbx.STEP_INTEGRATE | vbx.STEP_ESDF | graph
        flags_q = vbx.STEP_QUERY | graph
        lat_scan, lat_query, batch_sizes = [], [], []
        # per scan: its kind, the wait from arrival to the issue of its step, and the time from
        # that issue to the end of the step's map part; they show where the latency tail comes from
        scan_kind, scan_wait, scan_step, scan_first, scan_gpu = [], [], [], [], []
        step_kernels = []  # profile_steps: per step, {kernel: ms} and its map-part device time
        if profile_steps:
            self.batch.set_profiling(True)
            prev_kt = self.batch.kernel_times()
        admitted = 0
        max_active = 0
        in_flight = collections.deque()
        pool_events = []

        def event():
            return pool_events.pop() if pool_events else torch.cuda.Event(enable_timing=True)

        gpu_ms = 0.0
        overlap_issues = 0  # steps issued while an earlier one was still on the GPU
        host = dict(issue=0.0, wait=0.0, admit=0.0, loops=0)  # host seconds by activity
        done_times = []  # host time at which each scan's step finished
        sat = [None, None]  # first and last time a session that had arrived waited for admission
        t0 = time.perf_counter()

        def retire(block: bool):
            nonlocal gpu_ms
            while in_flight:
                now = time.perf_counter() - t0
                for f in in_flight:
                    if f["t_scan"] is None and f["e1"].query():
                        f["t_scan"] = now
                f = in_flight[0]
                if block:
                    tw = time.perf_counter()
                    if f["t_scan"] is None:
                        f["e1"].synchronize()
                        f["t_scan"] = time.perf_counter() - t0
                    f["e2"].synchronize()
                    now = time.perf_counter() - t0
                    host["wait"] += time.perf_counter() - tw
                elif not f["e2"].query():
                    return
                if f["t_scan"] is None:
                    f["t_scan"] = now
                in_flight.popleft()
                t_done = now
                gpu_ms += f["e0"].elapsed_time(f["e2"])
                f["map_ms"] = f["e0"].elapsed_time(f["e1"])
                scan_gpu_s = f["map_ms"] * 1e-3
                for arrival, kind, first in f["scans"]:
                    done_times.append(t_done)
                    lat_query.append(t_done - arrival)
                    lat_scan.append(f["t_scan"] - arrival)
                    scan_kind.append(kind)
                    scan_first.append(first)
                    scan_gpu.append(scan_gpu_s)
                    scan_wait.append(max(f["t_issue"] - arrival, 0.0))
                    scan_step.append(f["t_scan"] - f["t_issue"])
                pool_events.extend((f["e0"], f["e1"], f["e2"]))
                block = False

        while waiting or active or in_flight:
            now = time.perf_counter() - t0
            if now > time_limit:
                raise RuntimeError("serving run exceeded its time limit")
            retire(False)
            host["loops"] += 1
            ta = time.perf_counter()
            # admission: arrival order, a free slot and room in the memory budget
            while waiting and waiting[0].start <= now and free_slots:
                spec = waiting[0]
                m = self._acquire(spec.kind)
                if m is None:
                    break
                waiting.popleft()
                slot = free_slots.pop()
                self.batch.bind(slot, m)
                gaps = rng.exponential(1.0 / spec.rate_hz, size=spec.n_scans)
                arrivals = max(spec.start, now) + np.cumsum(gaps) - gaps[0]
                active[slot] = _Active(spec, m, arrivals)
                admitted += 1
            max_active = max(max_active, len(active))
            if waiting and waiting[0].start <= now:  # saturated: an arrived session waits for a slot or memory
                sat[0] = now if sat[0] is None else sat[0]
                sat[1] = now
            ready = [s for s, a in active.items() if a.arrivals[a.next] <= now]
            host["admit"] += time.perf_counter() - ta
            if not ready or len(in_flight) >= max_in_flight:
                if not ready and not in_flight:
                    nxt = [a.arrivals[a.next] for a in active.values()]
                    if waiting and free_slots:
                        nxt.append(waiting[0].start)
                    wait = (min(nxt) - now) if nxt else 0.001
                    time.sleep(min(max(wait, 0.0), 0.002))
                elif len(in_flight) >= max_in_flight:
                    retire(True)
                else:
                    time.sleep(5e-5)
                continue
            points, poses, queries, scans = [], [], [], []
            for s in ready:
                a = active[s]
                p, T, q = self.pool.frame(a.spec, a.next)
                points.append(p)
                poses.append(T)
                queries.append((q,) + self.out[s])
                scans.append((float(a.arrivals[a.next]), a.spec.kind, a.next == 0))
            if in_flight:
                overlap_issues += 1
            f = dict(e0=event(), e1=event(), e2=event(), scans=scans, t_scan=None, t_issue=time.perf_counter() - t0)
            ti = time.perf_counter()
            f["e0"].record()
            self.batch.step(points, poses, flags=flags_map, slots=ready)
            f["e1"].record()
            self.batch.step(queries=queries, flags=flags_q, slots=ready)
            f["e2"].record()
            host["issue"] += time.perf_counter() - ti
            in_flight.append(f)
            batch_sizes.append(len(ready))
            if profile_steps:
                retire(True)
                kt = self.batch.kernel_times()
                step_kernels.append((f["map_ms"], {k: v["ms"] - prev_kt.get(k, {"ms": 0.0})["ms"] for k, v in kt.items()}))
                prev_kt = kt
            for s in ready:
                a = active[s]
                a.next += 1
                if a.next == a.spec.n_scans:
                    # the session's last scan is issued; work enqueued from here on (the callback's
                    # copies, a reset for the next session) runs after it on the same stream
                    if on_finish is not None:
                        on_finish(a.spec, a.m, tuple(t.clone() for t in self.out[s]))
                    self.batch.bind(s, self.idle[s])
                    self.free[a.spec.kind].append(a.m)
                    del active[s]
                    free_slots.append(s)
        if profile_steps:
            self.batch.set_profiling(False)
        self.batch.sync()
        wall = time.perf_counter() - t0
        n = len(lat_scan)
        ls = np.asarray(lat_scan) * 1e3
        lq = np.asarray(lat_query) * 1e3
        kinds = np.asarray(scan_kind)
        pct = lambda x: dict(p50=float(np.percentile(x, 50)), p99=float(np.percentile(x, 99))) if len(x) else None
        by_kind = {
            k: dict(
                scans=int((kinds == k).sum()),
                latency_ms=pct(ls[kinds == k]),
                wait_ms=pct(np.asarray(scan_wait)[kinds == k] * 1e3),
                step_ms=pct(np.asarray(scan_step)[kinds == k] * 1e3),
                step_gpu_ms=pct(np.asarray(scan_gpu)[kinds == k] * 1e3),
            )
            for k in sorted(set(scan_kind))
        }
        # a session's first scan starts from an empty map (all blocks new, the ESDF from scratch)
        first = np.asarray(scan_first, bool)
        by_kind.update(
            {
                f"{k}_first_scan": dict(scans=int(((kinds == k) & first).sum()), latency_ms=pct(ls[(kinds == k) & first]))
                for k in sorted(set(scan_kind))
            }
        )
        by_kind.update(
            {
                f"{k}_later_scans": dict(scans=int(((kinds == k) & ~first).sum()), latency_ms=pct(ls[(kinds == k) & ~first]))
                for k in sorted(set(scan_kind))
            }
        )
        return dict(
            sessions=admitted,
            scans=n,
            wall_s=wall,
            scans_per_s=n / wall,
            saturated_window_s=(sat[1] - sat[0]) if sat[0] is not None else 0.0,
            saturated_scans_per_s=(
                sum(1 for t in done_times if sat[0] <= t <= sat[1]) / (sat[1] - sat[0])
                if sat[0] is not None and sat[1] - sat[0] > 0.5
                else None
            ),
            gpu_busy_frac=gpu_ms / 1e3 / wall,
            scans_per_gpu_s=n / (gpu_ms / 1e3),
            steps=len(batch_sizes),
            mean_batch=float(np.mean(batch_sizes)) if batch_sizes else 0.0,
            max_concurrent_sessions=max_active,
            scan_latency_ms=dict(p50=float(np.percentile(ls, 50)), p99=float(np.percentile(ls, 99))),
            scan_latency_by_kind=by_kind,
            query_latency_ms=dict(p50=float(np.percentile(lq, 50)), p99=float(np.percentile(lq, 99))),
            peak_map_bytes=self.peak,
            budget_bytes=self.budget,
            steps_issued_while_gpu_busy=overlap_issues,
            host_ms_per_step={k: 1e3 * host[k] / max(len(batch_sizes), 1) for k in ("issue", "wait", "admit")},
            loop_iterations=host["loops"],
            max_in_flight=max_in_flight,
            slow_step_kernels=_slow_step_kernels(step_kernels) if profile_steps else None,
        )


def _slow_step_kernels(step_kernels, q: float = 99.0):
    """Mean per-kernel device time of the steps whose map part is at or above the q-th
    percentile of map-part device time, beside the same for the median half of the steps."""
    if not step_kernels:
        return None
    t = np.asarray([x[0] for x in step_kernels])
    hi = t >= np.percentile(t, q)
    mid = (t >= np.percentile(t, 25)) & (t <= np.percentile(t, 75))

    def mean(mask):
        ks = sorted({k for x in step_kernels for k in x[1]})
        n = max(int(mask.sum()), 1)
        return {k: sum(x[1].get(k, 0.0) for x, m in zip(step_kernels, mask) if m) / n for k in ks}

    return dict(
        steps=len(step_kernels),
        slow_steps=int(hi.sum()),
        slow_step_map_ms=float(t[hi].mean()),
        median_step_map_ms=float(np.median(t)),
        slow_step_kernel_ms=mean(hi),
        median_steps_kernel_ms=mean(mid),
    )

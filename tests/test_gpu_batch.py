"""Batched form: several maps of different scenes and parameters advanced by the same
launches (direct and CUDA-graph replay) give exactly the maps each would reach alone, and
every batched map matches the float64 oracle run on the same scans."""
import numpy as np
import pytest

import oracle
from paper_1611_03631_gb300 import scenes
from parity_util import compare_with_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vbx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03631_gb300 import vbx as v

    v.load_library()
    return v


def _scenes():
    return [
        scenes.plane_sphere(frames=3),
        scenes.room(frames=3, width=160, height=120, fx=131.25, fy=131.25),
        scenes.lidar_terrain(scans=3, beams=16, columns=512, n_buildings=60, n_trees=100),
        scenes.plane_sphere(frames=3, width=32, height=24, fx=25.0, fy=25.0, cx=16.0, cy=12.0, seed=7),
        scenes.room(frames=3, width=80, height=60, fx=65.6, fy=65.6, seed=11, voxel_size=0.1),
    ]


def _maps(vbx, ss):
    out = []
    for s in ss:
        kw = dict(block_capacity=1 << 16) if s.name == "lidar_terrain" else {}
        out.append(vbx.Map.from_scene_params(s.params, **kw))
    return out


def _same(a, b):
    ea, eb = a.export(), b.export()
    assert np.array_equal(ea["keys"], eb["keys"])
    assert np.array_equal(ea["flags"], eb["flags"])
    for k in ("D", "W", "d"):
        assert np.array_equal(ea[k], eb[k]), k


@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_maps_updated_alone(vbx, graph):
    ss = _scenes()
    alone = _maps(vbx, ss)
    mixed = _maps(vbx, ss)
    batch = vbx.MapBatch(mixed, max_queries=2048)
    orc = [oracle.OracleMap.from_scene_params(s.params) for s in ss]
    flags = vbx.STEP_INTEGRATE | vbx.STEP_ESDF | (vbx.STEP_GRAPH if graph else 0)
    for f in range(3):
        pts = [torch.from_numpy(s.points[f]).cuda() for s in ss]
        for m, s, p in zip(alone, ss, pts):
            m.integrate_scan(p, s.poses[f])
            m.update_esdf()
        batch.step(pts, [s.poses[f] for s in ss], flags=flags)
        batch.sync()
        for a, b in zip(alone, mixed):
            _same(a, b)
        for o, s, b in zip(orc, ss, mixed):
            o.integrate(s.points[f], s.poses[f])
            o.update_esdf()
            compare_with_oracle(b.export(), o.export(), s.params)
    # queries through the batch equal the single-map queries
    qs = [torch.from_numpy(scenes.random_queries(s, 1500, radius=2.0, seed=3)).cuda() for s in ss]
    outs = [(q, torch.empty(q.shape[0], device="cuda"), torch.empty((q.shape[0], 3), device="cuda"),
             torch.empty(q.shape[0], dtype=torch.uint8, device="cuda")) for q in qs]
    batch.step(queries=outs, flags=vbx.STEP_QUERY | (vbx.STEP_GRAPH if graph else 0))
    batch.sync()
    for m, q, (qq, d, g, st) in zip(alone, qs, outs):
        d1, g1, s1 = m.query(q)
        assert torch.equal(s1, st)
        ok = s1 == 0
        assert torch.equal(d1[ok], d[ok]) and torch.equal(g1[ok], g[ok])


def test_batch_slots_without_scans_and_autotune(vbx):
    ss = _scenes()[:3]
    maps = _maps(vbx, ss)
    ref = _maps(vbx, ss)
    batch = vbx.MapBatch(maps)
    pts = [torch.from_numpy(s.points[0]).cuda() for s in ss]
    report = batch.autotune(pts, [s.poses[0] for s in ss])
    assert "esdf_ctas_per_sm" in report
    trials = int(report.split("trial_steps=")[1].split()[0])
    assert trials >= 2
    # autotuning integrated frame 0 once per candidate into `maps`; do the same to `ref`
    for _ in range(trials):
        for m, s, p in zip(ref, ss, pts):
            m.integrate_scan(p, s.poses[0])
            m.update_esdf()
    # slot 1 idle in this step
    p1 = [torch.from_numpy(s.points[1]).cuda() for s in ss]
    p1[1] = None
    batch.step(p1, [s.poses[1] for s in ss])
    batch.sync()
    for i, (m, s) in enumerate(zip(ref, ss)):
        if i != 1:
            m.integrate_scan(torch.from_numpy(s.points[1]).cuda(), s.poses[1])
        m.update_esdf()
    for a, b in zip(ref, maps):
        _same(a, b)


def test_many_maps_rounds_equal_single_map_queues(vbx):
    """More than 16 maps at work: the batched ESDF runs in global rounds, while each map alone
    runs its waves as work queues. Both schedules must reach the same maps, bit for bit."""
    ss = [
        scenes.plane_sphere(frames=3, width=32, height=24, fx=25.0, fy=25.0, cx=16.0, cy=12.0, seed=20 + k)
        for k in range(20)
    ]
    alone = _maps(vbx, ss)
    mixed = _maps(vbx, ss)
    batch = vbx.MapBatch(mixed)
    for f in range(3):
        pts = [torch.from_numpy(s.points[f]).cuda() for s in ss]
        for m, s, p in zip(alone, ss, pts):
            m.integrate_scan(p, s.poses[f])
            m.update_esdf()
        batch.step(pts, [s.poses[f] for s in ss])
        batch.sync()
        for a, b in zip(alone, mixed):
            _same(a, b)
    assert max(m.stats()["lower_rounds"] for m in mixed) > 1  # rounds, not the queue
    assert max(m.stats()["lower_rounds"] for m in alone) == 1  # one queue

"""Served form: sessions admitted under a memory budget and advanced by continuously
re-formed batches (several steps in flight) give the same map and query results as each
session run alone, and every session's map matches the float64 oracle on the same frames."""
import numpy as np
import pytest

import oracle
from paper_1611_03631_gb300 import scenes
from parity_util import compare_with_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03631_gb300 import serve, vbx

    vbx.load_library()
    return vbx, serve


def test_sessions_alone_equal_sessions_in_the_mix(mods):
    vbx, serve = mods
    sets = {
        "room": [scenes.room(frames=4, width=96, height=72, fx=78.75, fy=78.75, seed=s) for s in (21, 22)],
        "ps": [scenes.plane_sphere(frames=4, width=32, height=24, fx=25.0, fy=25.0, cx=16.0, cy=12.0, seed=s) for s in (31, 32)],
    }
    pool = serve.ScanPool(sets, n_queries=600)
    cap = {"room": 1024, "ps": 16384}
    # served maps hold scratch for the largest scan of their kind only; the maps run alone below
    # keep the default (whole-pool) scratch
    scratch = serve.scratch_for_pool(pool, cap, margin=1.0)
    assert all(0 < scratch[k] < cap[k] for k in sets)
    # a budget for about two maps at a time, three slots: sessions wait, batches change every step
    one = max(
        vbx.map_bytes(sets[k][0].params["voxels_per_block"], cap[k], max(p.shape[0] for p in sets[k][0].points), scratch[k])
        for k in sets
    )
    srv = serve.MapServer(pool, slots=3, hbm_budget=2.5 * one, capacity=cap, use_graph=True, scratch=scratch)
    # fast arrivals (the GPU outpaces 10-30 Hz robots) so that sessions share steps
    specs = serve.poisson_sessions(
        7, ["room", "ps"], {"room": 2, "ps": 2}, {"room": 4, "ps": 4}, 2000.0, 3, rate_range=(500.0, 1000.0), seed=3
    )
    got = {}

    def finish(spec, m, qout):
        got[spec.sid] = (m.export(), tuple(t.cpu().numpy() for t in qout))

    res = srv.run(specs, on_finish=finish)
    assert res["scans"] == 7 * 3 and res["sessions"] == 7
    assert res["mean_batch"] > 1.0  # sessions shared steps
    assert res["peak_map_bytes"] <= 2.5 * one
    for spec in specs:
        m = vbx.Map.from_scene_params(pool.params[spec.kind], block_capacity=cap[spec.kind])
        for k in range(spec.n_scans):
            p, T, q = pool.frame(spec, k)
            m.integrate_scan(p, T)
            m.update_esdf()
        d, g, st = m.query(q)
        ex, (d2, g2, st2) = got[spec.sid]
        o = oracle.OracleMap.from_scene_params(pool.params[spec.kind])
        for k in range(spec.n_scans):
            f = (spec.offset + k) % len(sets[spec.kind][spec.seq].points)
            o.integrate(sets[spec.kind][spec.seq].points[f], sets[spec.kind][spec.seq].poses[f])
            o.update_esdf()
        compare_with_oracle(ex, o.export(), pool.params[spec.kind])
        mine = m.export()
        assert np.array_equal(mine["keys"], ex["keys"])
        assert np.array_equal(mine["flags"], ex["flags"])
        for key in ("D", "W", "d"):
            assert np.array_equal(mine[key], ex[key]), (spec.sid, key)
        st = st.cpu().numpy()
        assert np.array_equal(st, st2)
        ok = st == 0
        assert np.array_equal(d.cpu().numpy()[ok], d2[ok]) and np.array_equal(g.cpu().numpy()[ok], g2[ok])
        m.close()
    srv.close()

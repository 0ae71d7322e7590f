"""GPU parity of the CUDA map update against the CPU oracle, through the C ABI.

Bar: allocated-block, updated-voxel, observed and seed sets bit-exact; |dD| <= 1e-5 m,
relative dW <= 1e-6, |d ESDF| <= 1e-4 m (bit-exact when both sides start from the same
float32 TSDF values)."""
import math

import numpy as np
import pytest

import oracle
from paper_1611_03631_gb300 import scenes
from parity_util import TOL_D, TOL_W_REL, check_parents, compare_tsdf, compare_with_oracle, sort_rows

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _run_tsdf(vbx, s, frames, check_each=True, **kw):
    g = vbx.Map.from_scene_params(s.params, **kw)
    o = oracle.OracleMap.from_scene_params(s.params, **{k: v for k, v in kw.items() if k in ("grouped",)})
    worst = dict(max_dD=0.0, max_rel_dW=0.0)
    for i in range(frames):
        g.integrate_scan(_dev(s.points[i]), s.poses[i])
        o.integrate(s.points[i], s.poses[i])
        if check_each or i == frames - 1:
            gu = sort_rows(g.last_updated())
            ou = o.last_updated()
            assert np.array_equal(gu, ou), f"frame {i}: updated voxel sets differ ({len(gu)} vs {len(ou)})"
            gs, os_ = g.stats(), o.stats()
            assert gs["points_valid"] == os_["points_valid"]
            assert gs["rays"] == os_["groups"]
            assert gs["records"] == os_["records"]
            assert gs["new_blocks"] == os_["new_blocks"]
            r = compare_tsdf(g.export(), o.export(), s.params["voxels_per_block"])
            worst["max_dD"] = max(worst["max_dD"], r["max_dD"])
            worst["max_rel_dW"] = max(worst["max_rel_dW"], r["max_rel_dW"])
            assert r["max_dD"] <= TOL_D, (i, r)
            assert r["max_rel_dW"] <= TOL_W_REL, (i, r)
    return g, o, worst


# ------------------------------------------------------------------------------ TSDF


def test_tsdf_parity_plane_sphere_all_frames(vbx):
    s = scenes.plane_sphere()
    g, o, worst = _run_tsdf(vbx, s, len(s))
    print("plane_sphere TSDF max |dD| %.3g m, max rel dW %.3g" % (worst["max_dD"], worst["max_rel_dW"]))


def test_tsdf_parity_room_quadratic_weight(vbx):
    # room scene at reduced resolution (several tiles, ragged tail: 160*120 = 19200 points)
    s = scenes.room(frames=4, width=160, height=120, fx=131.25, fy=131.25)
    _run_tsdf(vbx, s, len(s))


def test_tsdf_parity_lidar_constant_weight(vbx):
    s = scenes.lidar_terrain(scans=2, beams=16, columns=512, n_buildings=60, n_trees=100)
    _run_tsdf(vbx, s, len(s), block_capacity=1 << 17)


def test_tsdf_parity_per_point_raycasting(vbx):
    s = scenes.plane_sphere(frames=2, width=32, height=24, fx=25.0, fy=25.0, cx=16.0, cy=12.0)
    _run_tsdf(vbx, s, len(s), grouped=False)


def test_integration_is_deterministic(vbx):
    s = scenes.room(frames=2, width=160, height=120, fx=131.25, fy=131.25)
    exports = []
    for _ in range(2):
        g = vbx.Map.from_scene_params(s.params)
        for i in range(len(s)):
            g.integrate_scan(_dev(s.points[i]), s.poses[i])
        g.update_esdf()
        exports.append(g.export())
    for k in ("keys", "D", "W", "d", "flags"):
        assert np.array_equal(exports[0][k], exports[1][k]), k


# ------------------------------------------------------------------------------ ESDF


def _esdf_same_input(vbx, s, frames, **esdf_opts):
    """GPU and oracle (float32 ESDF mode) run the ESDF update on identical float32 TSDF
    values taken from a reference oracle integration: ESDF values must agree bit-exactly.
    esdf_opts (fixed_band, esdf_mode) go to both sides."""
    ref = oracle.OracleMap.from_scene_params(s.params)
    o32 = oracle.OracleMap.from_scene_params(s.params, esdf_fp32=1, **esdf_opts)
    g = vbx.Map.from_scene_params(s.params, **esdf_opts)
    B = s.params["voxels_per_block"]
    v = np.float32(s.params["voxel_size"])
    L = (0.0, v, np.float32(v * np.float32(1.41421356237309515)), np.float32(v * np.float32(1.73205080756887719)))
    for i in range(frames):
        ref.integrate(s.points[i], s.poses[i])
        ex = ref.export()
        upd = ref.last_updated()
        idx = {tuple(k): j for j, k in enumerate(ex["keys"])}
        bj = np.array([idx[(x // B, y // B, z // B)] for x, y, z in upd], dtype=np.int64)
        loc = ((upd[:, 2] % B) * B + (upd[:, 1] % B)) * B + (upd[:, 0] % B)
        D32 = ex["D"][bj, loc].astype(np.float32)
        W32 = ex["W"][bj, loc].astype(np.float32)
        o32.set_tsdf(upd, D32.astype(np.float64), W32.astype(np.float64))
        g.import_tsdf(upd, D32, W32)
        o32.update_esdf()
        g.update_esdf()
        gex, oex = g.export(), o32.export()
        assert np.array_equal(gex["keys"], oex["keys"])
        assert np.array_equal(gex["flags"], oex["flags"]), f"frame {i}: observed/fixed flags differ"
        obs = (oex["flags"] & 1) > 0
        assert np.array_equal(gex["d"][obs], oex["d"][obs].astype(np.float32)), f"frame {i}: ESDF values differ"
        gs, os_ = g.stats(), o32.stats()
        assert gs["seeds"] == os_["seeds"]
        bad, checked = check_parents(gex, B, L)
        assert bad == 0 and (checked > 0 or not obs.any())
    return g, o32


def test_esdf_parity_same_tsdf_plane_sphere(vbx):
    s = scenes.plane_sphere(frames=6)
    _esdf_same_input(vbx, s, len(s))


def test_esdf_parity_same_tsdf_room(vbx):
    s = scenes.room(frames=3, width=160, height=120, fx=131.25, fy=131.25)
    _esdf_same_input(vbx, s, len(s))


def test_esdf_parity_same_tsdf_occupancy_mode(vbx):
    """The occupancy ESDF of Sec. VI-B (negative TSDF voxels occupied at distance 0)."""
    s = scenes.room(frames=3, width=160, height=120, fx=131.25, fy=131.25)
    g, _ = _esdf_same_input(vbx, s, len(s), esdf_mode=1)
    ex = g.export()
    obs = (ex["flags"] & 1) > 0
    assert (ex["d"][obs] >= 0).all()


def test_esdf_parity_same_tsdf_half_truncation_band(vbx):
    """The half-truncation fixed band of Sec. VI-B, |D| < delta / 2."""
    s = scenes.plane_sphere(frames=4)
    _esdf_same_input(vbx, s, len(s), fixed_band=0.5 * s.params["truncation"])


@pytest.mark.parametrize("method", ["occupancy", "half_band", "one_voxel_band"])
def test_esdf_parity_same_tsdf_benchmark_scene(vbx, method):
    """The three ESDF methods of Sec. VI-B on the simulated benchmark scene."""
    from paper_1611_03631_gb300 import esdf_methods

    s = scenes.esdf_benchmark(poses=5, width=80, height=60, fx=65.625, voxel_size=0.2)
    _esdf_same_input(vbx, s, len(s), **esdf_methods.method_options(method, s.params))


def test_esdf_methods_evaluation_runs(vbx):
    from paper_1611_03631_gb300 import esdf_methods

    s = scenes.esdf_benchmark(poses=5, width=80, height=60, fx=65.625, voxel_size=0.2)
    for method in esdf_methods.METHODS:
        r = esdf_methods.run(s, method)
        assert r["esdf_voxels_scored"] > 1000
        assert np.isfinite(r["esdf_mean_abs_err_m"]) and r["esdf_mean_abs_err_m"] < 1.0
    g = esdf_methods.run(s, "one_voxel_band", grouped=False)
    assert np.isfinite(g["tsdf_mean_abs_err_m"])


def _end_to_end(vbx, s, frames, label, **map_kw):
    """GPU integrate + ESDF against the float64 oracle after every frame: TSDF sets and counts
    bit-exact, then compare_with_oracle (TSDF tolerances, ESDF with the guard-band rule)."""
    p = s.params
    g = vbx.Map.from_scene_params(p, **map_kw)
    o = oracle.OracleMap.from_scene_params(p)
    worst = dict(max_dD=0.0, max_rel_dW=0.0, max_dd=0.0, excluded_seeds=0)
    for i in range(frames):
        g.integrate_scan(_dev(s.points[i]), s.poses[i])
        o.integrate(s.points[i], s.poses[i])
        gu = sort_rows(g.last_updated())
        assert np.array_equal(gu, o.last_updated()), f"{label} frame {i}: updated voxel sets differ"
        gs, os_ = g.stats(), o.stats()
        for a, b in (("points_valid", "points_valid"), ("rays", "groups"), ("records", "records"), ("new_blocks", "new_blocks")):
            assert gs[a] == os_[b], (label, i, a, gs[a], os_[b])
        g.update_esdf()
        o.update_esdf()
        r = compare_with_oracle(g.export(), o.export(), p)
        for k in ("max_dD", "max_rel_dW", "max_dd"):
            worst[k] = max(worst[k], r[k])
        worst["excluded_seeds"] += r["excluded_seeds"]
    print(
        "%s end to end: max |dD| %.3g m, max rel dW %.3g, max |dd| %.3g m, %d guard-band seeds excluded, %d blocks"
        % (label, worst["max_dD"], worst["max_rel_dW"], worst["max_dd"], worst["excluded_seeds"], g.num_blocks())
    )
    return g, o, worst


def test_esdf_end_to_end_plane_sphere(vbx):
    s = scenes.plane_sphere()
    _end_to_end(vbx, s, len(s), "plane_sphere")


def test_end_to_end_full_size_room_frames(vbx):
    """Two full 640x480 frames of the room sequence, TSDF and ESDF against the float64 oracle."""
    s = scenes.room(frames=2)
    _end_to_end(vbx, s, len(s), "room 640x480")


def test_end_to_end_full_size_lidar_scans(vbx):
    """The first three scans of the outdoor LiDAR growth sequence at its full size (64 x 2048
    rays, 60 m range, the 100-scan path over the 200 m terrain): TSDF and ESDF against the
    float64 oracle after every scan. These scans allocate about 24k blocks, traverse long
    block segments and run raise waves."""
    s = scenes.lidar_terrain(generate=3, workers=8)
    _, _, worst = _end_to_end(vbx, s, len(s), "lidar 64x2048", block_capacity=1 << 17)


# ----------------------------------------------------------------------------- query


def test_query_parity(vbx):
    s = scenes.plane_sphere(frames=4)
    g, o32 = _esdf_same_input(vbx, s, len(s))
    rng = np.random.default_rng(9)
    d = rng.normal(size=(4099, 3))
    q = (np.array([0.0, 0.0, 0.6]) + 2.2 * d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(0, 1, (4099, 1)) ** (1 / 3))
    q = np.concatenate([q.astype(np.float32), np.array([[0.05, 0.05, 0.05], [100.0, 0.0, 0.0]], np.float32)])
    dist, grad, status = g.query(_dev(q))
    dist, grad, status = dist.cpu().numpy(), grad.cpu().numpy(), status.cpu().numpy()
    od, og, os_ = o32.query(q)
    assert np.array_equal(status, os_), "query status (known/unknown) differs"
    ok = status == 0
    assert ok.sum() > 500 and (~ok).sum() > 0
    assert np.all(np.isnan(dist[~ok]))
    assert np.max(np.abs(dist[ok] - od[ok])) <= 1e-5
    # the gradient of the trilinear interpolant is a sum of about 8 corner values times float32
    # weights, divided by v: with identical corner values its float32 rounding error is at most
    # about 8 ulp(d_max) / v = 8 * 2.4e-7 / 0.1 m, about 2e-5
    v, dmax = s.params["voxel_size"], s.params["max_esdf_dist"]
    assert np.max(np.abs(grad[ok] - og[ok])) <= 8 * np.spacing(np.float32(dmax)) / v


# ------------------------------------------------------------------------ edge cases


def test_edge_cases_empty_nan_and_single_point(vbx):
    g = vbx.Map(0.1, 8, 0.3, 2.0)
    T = np.eye(4, dtype=np.float32)
    g.integrate_scan(torch.zeros((0, 3), dtype=torch.float32, device="cuda"), T)
    g.update_esdf()
    assert g.num_blocks() == 0
    g.integrate_scan(_dev(np.full((37, 3), np.nan)), T)
    assert g.stats()["points_valid"] == 0 and g.num_blocks() == 0
    o = oracle.OracleMap(0.1, 8, 0.3, 2.0)
    pt = np.array([[0.33, -0.21, 1.7]], np.float32)
    g.integrate_scan(_dev(pt), T)
    o.integrate(pt, T)
    compare_tsdf(g.export(), o.export(), 8)
    assert np.array_equal(sort_rows(g.last_updated()), o.last_updated())
    g.update_esdf()
    g.sync()


def test_max_range_filter_and_ragged_sizes(vbx):
    rng = np.random.default_rng(4)
    for n in (1, 31, 33, 255, 257, 1000):
        pts = rng.uniform(-3, 3, (n, 3)).astype(np.float32)
        pts[::7] = np.nan
        T = np.eye(4, dtype=np.float32)
        T[:3, 3] = [0.01, 0.02, 0.03]
        g = vbx.Map(0.1, 8, 0.3, 2.0, max_range=2.5)
        o = oracle.OracleMap(0.1, 8, 0.3, 2.0, max_range=2.5)
        g.integrate_scan(_dev(pts), T)
        o.integrate(pts, T)
        assert g.stats()["points_valid"] == o.stats()["points_valid"]
        r = compare_tsdf(g.export(), o.export(), 8)
        assert r["max_dD"] <= TOL_D


def test_pool_exhaustion_reports_out_of_memory(vbx):
    s = scenes.plane_sphere(frames=1)
    g = vbx.Map.from_scene_params(s.params, block_capacity=64)
    g.integrate_scan(_dev(s.points[0]), s.poses[0])
    with pytest.raises(vbx.VbxError) as ei:
        g.sync()
    assert ei.value.status == 2
    # the map stays usable
    g.update_esdf()
    g.sync()
    assert g.num_blocks() == 64


def test_scratch_overflow_rejects_the_whole_scan(vbx):
    """A scan whose rays enter more blocks than scratch_blocks is not integrated at all: the
    call reports out-of-memory and no voxel is observed (its blocks stay allocated, empty)."""
    s = scenes.plane_sphere(frames=1)
    g = vbx.Map.from_scene_params(s.params, scratch_blocks=64)
    g.integrate_scan(_dev(s.points[0]), s.poses[0])
    with pytest.raises(vbx.VbxError) as ei:
        g.sync()
    assert ei.value.status == 2
    st = g.stats()
    assert st["touched_blocks"] > 64 and st["updated"] == 0 and st["records"] == 0
    ex = g.export()
    assert not (ex["W"] > 0).any()
    g.update_esdf()
    g.sync()
    assert g.stats()["esdf_in"] == 0


def test_tight_scratch_equals_default(vbx):
    """Scratch sized exactly to the largest scan's touched blocks gives bit-identical maps."""
    s = scenes.room(frames=3, width=160, height=120, fx=131.25, fy=131.25)
    a = vbx.Map.from_scene_params(s.params)
    need = 0
    for i in range(len(s)):
        a.integrate_scan(_dev(s.points[i]), s.poses[i])
        a.update_esdf()
        need = max(need, a.stats()["touched_blocks"])
    b = vbx.Map.from_scene_params(s.params, scratch_blocks=need)
    for i in range(len(s)):
        b.integrate_scan(_dev(s.points[i]), s.poses[i])
        b.update_esdf()
    b.sync()
    ea, eb = a.export(), b.export()
    for k in ("keys", "D", "W", "d", "flags"):
        assert np.array_equal(ea[k], eb[k]), k
    assert vbx.map_bytes(16, 4096, 1 << 16, scratch_blocks=need) < vbx.map_bytes(16, 4096, 1 << 16)


def test_reset_map_equals_fresh_map(vbx):
    """A reset map (device-side, stream-ordered) integrates a new sequence exactly like a new map."""
    a_seq = scenes.room(frames=3, width=160, height=120, fx=131.25, fy=131.25, seed=11)
    b_seq = scenes.room(frames=3, width=160, height=120, fx=131.25, fy=131.25, seed=12)
    m = vbx.Map.from_scene_params(a_seq.params, block_capacity=4096)
    for i in range(len(a_seq)):
        m.integrate_scan(_dev(a_seq.points[i]), a_seq.poses[i])
        m.update_esdf()
    m.reset()
    fresh = vbx.Map.from_scene_params(b_seq.params, block_capacity=4096)
    for g in (m, fresh):
        for i in range(len(b_seq)):
            g.integrate_scan(_dev(b_seq.points[i]), b_seq.poses[i])
            g.update_esdf()
        g.sync()
    ea, eb = m.export(), fresh.export()
    for k in ("keys", "D", "W", "d", "flags"):
        assert np.array_equal(ea[k], eb[k]), k
    assert m.stats()["blocks"] == fresh.stats()["blocks"]


def test_invalid_arguments(vbx):
    with pytest.raises(vbx.VbxError):
        vbx.Map(0.1, 7, 0.3, 2.0)
    with pytest.raises(vbx.VbxError):
        vbx.Map(-0.1, 8, 0.3, 2.0)
    with pytest.raises(vbx.VbxError):
        vbx.Map(0.1, 8, 0.05, 2.0)

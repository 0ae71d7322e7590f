"""Pins of the oracle's TSDF half (Sec. IV, Eq. 1-4) against values fixed by hand,
brute force and invariants -- never against the oracle itself."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1611_03631_gb300 import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden", "eq1_eq4_cases.json")


def _gold():
    with open(GOLD) as f:
        return json.load(f)


# ----------------------------------------------------------------------------- Eq. (1)


def test_eq1_projective_distance_hand_cases():
    for c in _gold()["eq1"]:
        d = oracle.projective_distance(c["pbar"], c["s"], c["c"], c["v"], c["delta"])
        assert d == pytest.approx(c["d"], abs=2e-6), c["why"]


# ------------------------------------------------------------------------- Eq. (2), (4)


def test_eq4_quadratic_weight_hand_cases():
    g = _gold()["eq4"]
    p = oracle.make_params(0.1, 8, g["delta"], 2.0, weighting=1, eps=g["eps"])
    for c in g["cases"]:
        w = oracle.record_weight(p, g["Wg"], c["d"])
        assert w == pytest.approx(c["w"], abs=1e-6), c["why"]


def test_eq4_continuity_at_breakpoints():
    p = oracle.make_params(0.1, 8, 0.4, 2.0, weighting=1, eps=0.1)
    tiny = 1e-6
    assert oracle.record_weight(p, 3.0, -0.1 - tiny) == pytest.approx(3.0, abs=1e-4)
    assert oracle.record_weight(p, 3.0, -0.1 + tiny) == pytest.approx(3.0, abs=1e-4)
    assert oracle.record_weight(p, 3.0, -0.4 + tiny) == pytest.approx(0.0, abs=1e-4)


def test_eq2_constant_weight():
    g = _gold()["eq2"]
    p = oracle.make_params(0.1, 8, 0.3, 2.0, weighting=0)
    for c in g["cases"]:
        assert oracle.record_weight(p, g["Wg"], c["d"]) == c["w"]


# ------------------------------------------------------- single rays: Eq. (1)+(3), Sec. IV-B

# Sensor at (0.05, 0.05, 0.05) looking along world +x (sensor z -> world x); a point 1 m
# ahead lands at x = 1.05, the centre plane of voxel row 10 (v = 0.1). The voxel centres of
# row i are at x = 0.1 i + 0.05, so Eq. (1) gives d_i = 1.0 - 0.1 i, truncated at delta.
_R_FWD_X = np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], dtype=np.float64)


def _pose_fwd_x():
    T = np.eye(4)
    T[:3, :3] = _R_FWD_X
    T[:3, 3] = [0.05, 0.05, 0.05]
    return T.astype(np.float32)


def _row_values(m):
    ex = m.export()
    out = {}
    for b, k in enumerate(ex["keys"]):
        for l in range(8 ** 3):
            lx, ly, lz = l % 8, (l // 8) % 8, l // 64
            if ex["W"][b, l] > 0:
                out[(k[0] * 8 + lx, k[1] * 8 + ly, k[2] * 8 + lz)] = (ex["D"][b, l], ex["W"][b, l])
    return out, ex


def test_single_ray_constant_weight_two_scans():
    m = oracle.OracleMap(0.1, 8, 0.27, 2.0, weighting=0)
    T = _pose_fwd_x()
    m.integrate(np.array([[0.0, 0.0, 1.0]], np.float32), T)
    vals, ex = _row_values(m)
    # hand values: d_i = 1.0 - 0.1 i truncated at +-0.27; the ray ends at x = 1.32 (row 13)
    exp1 = [0.27] * 8 + [0.2, 0.1, 0.0, -0.1, -0.2, -0.27]
    assert sorted(vals) == [(i, 0, 0) for i in range(14)]
    for i, e in enumerate(exp1):
        assert vals[(i, 0, 0)][0] == pytest.approx(e, abs=2e-6)
        assert vals[(i, 0, 0)][1] == 1.0
    # rows 0..7 lie in block (0,0,0), rows 8..13 in block (1,0,0)
    assert sorted(map(tuple, ex["keys"])) == [(0, 0, 0), (1, 0, 0)]
    # second scan 0.1 m further: d'_i = 1.1 - 0.1 i; Eq. (3) with unit weights averages
    m.integrate(np.array([[0.0, 0.0, 1.1]], np.float32), T)
    vals, _ = _row_values(m)
    exp2 = [0.27] * 8 + [0.235, 0.15, 0.05, -0.05, -0.15, -0.235, -0.27]
    wexp = [2.0] * 14 + [1.0]
    assert sorted(vals) == [(i, 0, 0) for i in range(15)]
    for i, (e, w) in enumerate(zip(exp2, wexp)):
        assert vals[(i, 0, 0)][0] == pytest.approx(e, abs=2e-6), i
        assert vals[(i, 0, 0)][1] == w


def test_single_ray_weight_cap_of_eq3():
    """Eq. (3) with W_max = 2 (w_max option): four scans of the same ray at depths 1.0, 1.1,
    1.0, 1.1 (unit weights). Voxel row 10 (centre x = 1.05) sees d = 0.0, 0.1, 0.0, 0.1:
      D1 = 0, W1 = 1;  D2 = 0.05, W2 = 2;  D3 = (2 * 0.05 + 0) / 3, W3 = min(3, 2) = 2;
      D4 = (2 * D3 + 0.1) / 3 with the cap, against (3 * D3 + 0.1) / 4 = 0.05 without it."""
    T = _pose_fwd_x()
    depths = (1.0, 1.1, 1.0, 1.1)
    m = oracle.OracleMap(0.1, 8, 0.27, 2.0, weighting=0, w_max=2.0)
    for depth in depths:
        m.integrate(np.array([[0.0, 0.0, depth]], np.float32), T)
    vals, _ = _row_values(m)
    D3 = (2 * 0.05 + 0.0) / 3
    D, W = vals[(10, 0, 0)]
    assert W == 2.0
    assert D == pytest.approx((2 * D3 + 0.1) / 3, abs=2e-6)
    m2 = oracle.OracleMap(0.1, 8, 0.27, 2.0, weighting=0)
    for depth in depths:
        m2.integrate(np.array([[0.0, 0.0, depth]], np.float32), T)
    vals2, _ = _row_values(m2)
    D2u, W2u = vals2[(10, 0, 0)]
    assert W2u == 4.0
    assert D2u == pytest.approx((3 * D3 + 0.1) / 4, abs=2e-6)
    assert abs(D - D2u) > 1e-3  # the cap changes D from the fourth scan on


def test_single_ray_quadratic_weight_dropoff():
    # Eq. (4) with delta = 0.27, eps = 0.1; the point is at depth z = 1 so 1/z^2 = 1.
    m = oracle.OracleMap(0.1, 8, 0.27, 2.0, weighting=1, eps=0.1)
    m.integrate(np.array([[0.0, 0.0, 1.0]], np.float32), _pose_fwd_x())
    vals, _ = _row_values(m)
    # row 13 has d = -0.27 = -delta: weight 0, so it is traversed but not updated
    assert sorted(vals) == [(i, 0, 0) for i in range(13)]
    assert vals[(11, 0, 0)][1] == pytest.approx(1.0, abs=1e-6)  # d = -eps
    assert vals[(12, 0, 0)][1] == pytest.approx(0.07 / 0.17, abs=1e-6)  # ramp
    assert vals[(5, 0, 0)][1] == pytest.approx(1.0, abs=0)
    # a point at depth 2 weighs 1/4 in front of the surface
    m2 = oracle.OracleMap(0.1, 8, 0.27, 2.0, weighting=1, eps=0.1)
    m2.integrate(np.array([[0.0, 0.0, 2.0]], np.float32), _pose_fwd_x())
    vals2, _ = _row_values(m2)
    assert vals2[(3, 0, 0)][1] == pytest.approx(0.25, abs=1e-7)


def test_filter_drops_invalid_points():
    m = oracle.OracleMap(0.1, 8, 0.3, 2.0, max_range=1.5)
    pts = np.array(
        [[np.nan, 0, 1], [0, 0, 0], [0, 0, 2.0], [0, 0, np.inf], [0, 0, 1.0]], np.float32
    )
    m.integrate(pts, _pose_fwd_x())
    st = m.stats()
    assert st["points_in"] == 5 and st["points_valid"] == 1


def test_filter_bounds_of_reading_r1():
    """Reading R1 bounds the integer ranges: a point 2^14 voxels or more from the sensor is
    dropped (v = 1 m: 16,000 m kept, 16,500 m dropped), and under Eq. (4) so is a point whose
    1/z^2 weight exceeds 1024 (z = 0.03 m dropped, z = 0.032 m kept) or whose depth is not
    positive."""
    m = oracle.OracleMap(1.0, 8, 2.0, 5.0)
    m.integrate(np.array([[0, 0, 16000.0], [0, 0, 16500.0]], np.float32), _pose_fwd_x())
    assert m.stats()["points_valid"] == 1
    q = oracle.OracleMap(0.1, 8, 0.3, 2.0, weighting=1, eps=0.1)
    q.integrate(np.array([[0, 0, 0.03], [0, 0, 0.032], [0, 0, -1.0]], np.float32), _pose_fwd_x())
    assert q.stats()["points_valid"] == 1


# ------------------------------------------------------------------ grouping, Sec. IV-B


def test_grouping_single_point_groups_and_means():
    rng = np.random.default_rng(0)
    pts = rng.uniform(-3, 3, size=(400, 3)).astype(np.float32)
    T = np.eye(4, dtype=np.float32)
    p = oracle.make_params(0.1, 8, 0.3, 2.0)
    keys, pbar, Wg, cnt = oracle.group(p, pts, T)
    assert cnt.sum() == 400
    assert np.all(Wg == cnt)  # constant weight: group weight = point count
    # every mean lies in (or on the + face of) its voxel
    lo = keys * 0.1
    assert np.all(pbar >= lo - 1e-6) and np.all(pbar <= lo + 0.1 + 1e-6)
    # single-point groups reproduce their point to the 1/65536-voxel quantum
    fk = np.floor(pts / np.float32(0.1)).astype(np.int32)
    single = {tuple(k): i for i, k in enumerate(keys) if cnt[i] == 1}
    hits = 0
    for j in range(400):
        i = single.get(tuple(fk[j]))
        if i is not None:
            hits += 1
            assert np.max(np.abs(pbar[i] - pts[j])) <= 0.1 / 65536 + 4e-7
    assert hits > 300


def test_grouping_two_points_weighted_mean():
    T = np.eye(4, dtype=np.float32)
    # two points in voxel (10,0,0): the mean is their midpoint
    pts = np.array([[1.01, 0.02, 0.03], [1.07, 0.06, 0.05]], np.float32)
    keys, pbar, Wg, cnt = oracle.group(oracle.make_params(0.1, 8, 0.3, 2.0), pts, T)
    assert keys.tolist() == [[10, 0, 0]] and cnt.tolist() == [2] and Wg.tolist() == [2.0]
    assert np.allclose(pbar[0], [1.04, 0.04, 0.04], atol=3e-6)
    # quadratic weight: points at depth z weigh 1/z^2 -> mean pulled to the nearer point
    Tq = np.eye(4, dtype=np.float32)
    pq = np.array([[0.01, 0.01, 1.0], [0.03, 0.01, 2.0 ** 0.5 * 0 + 1.0]], np.float32)
    pq[1, 2] = 1.0  # same depth: equal weights
    keys, pbar, Wg, cnt = oracle.group(oracle.make_params(0.1, 8, 0.3, 2.0, weighting=1), pq, Tq)
    assert np.allclose(pbar[0], [0.02, 0.01, 1.0], atol=3e-6) and Wg[0] == pytest.approx(2.0, rel=1e-6)
    # depth 1 and depth 1.05 in one voxel: weights 1 and 1/1.1025
    pq2 = np.array([[0.01, 0.01, 1.01], [0.05, 0.01, 1.05]], np.float32)
    keys, pbar, Wg, cnt = oracle.group(oracle.make_params(0.1, 8, 0.3, 2.0, weighting=1), pq2, Tq)
    w1, w2 = 1 / 1.01 ** 2, 1 / 1.05 ** 2
    assert Wg[0] == pytest.approx(w1 + w2, rel=1e-6)
    assert pbar[0, 0] == pytest.approx((0.01 * w1 + 0.05 * w2) / (w1 + w2), abs=3e-6)


def test_grouped_equals_per_point_when_one_point_per_voxel():
    """With one point per voxel, grouped raycasting reduces to plain raycasting (up to the
    1/65536-voxel quantisation of the mean)."""
    rng = np.random.default_rng(3)
    # points on a sparse 3-D lattice, 0.4 m apart, so no two share a voxel
    g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(3), indexing="ij"), -1).reshape(-1, 3)
    pts = (g * 0.4 + np.array([1.0, -0.6, -0.4]) + rng.uniform(0.0, 0.08, g.shape)).astype(np.float32)
    T = np.eye(4, dtype=np.float32)
    T[:3, 3] = [0.013, 0.021, 0.017]
    a = oracle.OracleMap(0.1, 8, 0.3, 2.0, grouped=1)
    b = oracle.OracleMap(0.1, 8, 0.3, 2.0, grouped=0)
    a.integrate(pts, T)
    b.integrate(pts, T)
    ea, eb = a.export(), b.export()
    assert np.array_equal(ea["keys"], eb["keys"])
    obs = ea["W"] > 0
    # the traversed/updated sets can differ only where a quantised endpoint crosses a face
    agree = obs == (eb["W"] > 0)
    assert agree.mean() > 0.999
    both = obs & (eb["W"] > 0)
    assert np.max(np.abs(ea["D"][both] - eb["D"][both])) < 1e-4


# ---------------------------------------------------------------- DDA (R3), brute force


def _events(S, E):
    """All face crossings of S->E as (t, axis, step), sorted by t then axis (x, y, z)."""
    F = 65536
    ev = []
    for a in range(3):
        D = E[a] - S[a]
        if D > 0:
            for k in range(S[a] // F + 1, E[a] // F + 1):
                ev.append((Fraction(k * F - S[a], D), a, 1))
        elif D < 0:
            for k in range(S[a] // F, E[a] // F, -1):
                ev.append((Fraction(S[a] - k * F, -D), a, -1))
    ev.sort(key=lambda e: (e[0], e[1]))
    return ev


def _brute_voxels(S, E):
    F = 65536
    c = [S[0] // F, S[1] // F, S[2] // F]
    out = [tuple(c)]
    for t, a, st in _events(S, E):
        c[a] += st
        out.append(tuple(c))
    return out


def _closed_box_touches(S, E, c):
    F = 65536
    lo, hi = Fraction(0), Fraction(1)
    for a in range(3):
        D = E[a] - S[a]
        b0, b1 = c[a] * F, (c[a] + 1) * F
        if D == 0:
            if not (b0 <= S[a] <= b1):
                return False
            continue
        t0, t1 = Fraction(b0 - S[a], D), Fraction(b1 - S[a], D)
        if t0 > t1:
            t0, t1 = t1, t0
        lo, hi = max(lo, t0), min(hi, t1)
    return lo <= hi


def _random_segments(rng, n):
    F = 65536
    segs = []
    for i in range(n):
        mode = i % 4
        if mode == 0:  # generic
            S = rng.integers(-5 * F, 5 * F, 3)
            E = S + rng.integers(-6 * F, 6 * F, 3)
        elif mode == 1:  # endpoints on grid faces / corners
            S = rng.integers(-4, 4, 3) * F
            E = rng.integers(-4, 4, 3) * F + rng.integers(0, 2, 3) * F // 2
        elif mode == 2:  # exact diagonals through voxel corners
            S = rng.integers(-4, 4, 3) * F
            k = int(rng.integers(1, 5))
            E = S + np.array([1, -1, 1]) * rng.permutation([k, k, k]) * F
        else:  # axis-aligned and planar
            S = rng.integers(-5 * F, 5 * F, 3)
            E = S.copy()
            E[int(rng.integers(0, 3))] += int(rng.integers(-5 * F, 5 * F))
        segs.append(([int(x) for x in S], [int(x) for x in E]))
    return segs


def test_dda_matches_exact_event_sort_and_geometry():
    rng = np.random.default_rng(11)
    F = 65536
    for S, E in _random_segments(rng, 400):
        got = [tuple(int(y) for y in x) for x in oracle.traverse(S, E)]
        assert got == _brute_voxels(S, E), (S, E)
        # 6-connected, from floor(S) to floor(E), |dx|+|dy|+|dz|+1 voxels
        assert got[0] == tuple(s // F for s in S) and got[-1] == tuple(e // F for e in E)
        assert len(got) == sum(abs(e // F - s // F) for s, e in zip(S, E)) + 1
        for a, b in zip(got, got[1:]):
            assert sum(abs(x - y) for x, y in zip(a, b)) == 1
        # every visited voxel's closed box touches the segment
        for c in got:
            assert _closed_box_touches(S, E, c), (S, E, c)
        # every voxel the open segment passes through is visited
        ts = sorted({Fraction(0), Fraction(1)} | {e[0] for e in _events(S, E)})
        vs = set(got)
        for t0, t1 in zip(ts, ts[1:]):
            tm = (t0 + t1) / 2
            c = tuple(int((S[a] + tm * (E[a] - S[a])) // F) for a in range(3))
            assert c in vs, (S, E, c)


def test_dda_tie_break_order_x_then_y_then_z():
    F = 65536
    # from the centre of voxel 0 through the corner shared with voxel (1,1,1)
    got = [tuple(x) for x in oracle.traverse([F // 2] * 3, [3 * F // 2] * 3)]
    assert got == [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1)]
    got = [tuple(x) for x in oracle.traverse([F // 2] * 3, [-F // 2, -F // 2, F // 2])]
    assert got == [(0, 0, 0), (-1, 0, 0), (-1, -1, 0)]


# --------------------------------------------------------- scene-level TSDF invariants


@pytest.fixture(scope="module")
def plane_sphere_oracle():
    s = scenes.plane_sphere(frames=4)
    m = oracle.OracleMap.from_scene_params(s.params)
    Ws = []
    for i in range(len(s)):
        m.integrate(s.points[i], s.poses[i])
        ex = m.export()
        Ws.append((ex["keys"].copy(), ex["W"].copy(), ex["D"].copy()))
    return s, m, Ws


def test_tsdf_invariants_plane_sphere(plane_sphere_oracle):
    s, m, Ws = plane_sphere_oracle
    delta = float(np.float32(s.params["truncation"]))  # the map holds delta as float32
    prev = None
    for keys, W, D in Ws:
        assert np.all(np.abs(D) <= delta + 1e-9)
        assert np.all(W <= 1e4)
        cur = {tuple(k): W[i] for i, k in enumerate(keys)}
        if prev is not None:
            for k, w in prev.items():  # weights never decrease, blocks never vanish
                assert np.all(cur[k] >= w)
        prev = cur


def test_tsdf_near_surface_matches_true_sdf(plane_sphere_oracle):
    """Inside the fixed band the fused distance is within one voxel of the analytic signed
    distance of the plane + sphere scene (spec pin for the TSDF)."""
    s, m, Ws = plane_sphere_oracle
    keys, W, D = Ws[-1]
    v = s.params["voxel_size"]
    B = 8
    l = np.arange(B ** 3)
    loc = np.stack([l % B, (l // B) % B, l // (B * B)], -1)
    ctr = ((keys[:, None, :] * B + loc[None]) + 0.5) * v
    sdf = scenes.plane_sphere_sdf(ctr)
    sel = (W >= 3) & (np.abs(D) < v)
    assert sel.sum() > 500
    err = np.abs(D[sel] - sdf[sel])
    assert err.max() < v
    # and the sign agrees wherever the true surface is more than a voxel away
    far = (W > 0) & (np.abs(sdf) > 2 * v) & (np.abs(sdf) < 2.5 * v)
    assert np.mean(np.sign(D[far]) == np.sign(sdf[far])) > 0.99


# ----------------------------------------- grouping through integrate(), worked by hand

GROUP3 = os.path.join(os.path.dirname(__file__), "golden", "grouped_ray_three_points.json")


@pytest.mark.parametrize("mode", ["constant", "quadratic"])
def test_grouped_ray_of_three_points_through_integrate(mode):
    """Three points in voxel (0,0,4) become one ray at their R1 weighted mean (half-weight
    rounding term, integer point weights, a round-half-even tie under Eq. 4); the map that
    integrate() builds carries the hand-worked D and W at two voxels of that ray. The D
    values move by about 3e-6 m if the mean's rounding term or its weights are wrong."""
    with open(GROUP3) as f:
        g = json.load(f)
    su, c = g["setup"], g[mode]
    m = oracle.OracleMap(su["voxel_size"], su["voxels_per_block"], su["truncation"], su["max_esdf_dist"],
                         weighting=c["weighting"], eps=su["eps"])
    pts = np.array(su["points"], np.float32)
    m.integrate(pts, np.eye(4, dtype=np.float32))
    st = m.stats()
    assert st["points_valid"] == 3 and st["groups"] == 1
    ex = m.export()
    idx = {tuple(k): i for i, k in enumerate(ex["keys"])}
    B = su["voxels_per_block"]
    for vc in c["voxels"]:
        x, y, z = vc["voxel"]
        b = idx[(x // B, y // B, z // B)]
        l = ((z % B) * B + (y % B)) * B + (x % B)
        assert ex["W"][b, l] == vc["W"], vc["working"]
        assert abs(ex["D"][b, l] - vc["D"]) <= 1e-7, vc["working"]
    # the grouping entry point returns the same group (it casts from the same function)
    keys, pbar, Wg, cnt = oracle.group(
        oracle.make_params(su["voxel_size"], B, su["truncation"], su["max_esdf_dist"], weighting=c["weighting"], eps=su["eps"]),
        pts, np.eye(4, dtype=np.float32),
    )
    assert keys.tolist() == [[0, 0, 4]] and cnt.tolist() == [3]
    assert pbar[0].astype(np.float64).tolist() == c["pbar"] and float(Wg[0]) == c["W_g"]

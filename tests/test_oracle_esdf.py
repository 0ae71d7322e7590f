"""Pins of the oracle's ESDF half (Sec. V-A, Algorithm 1) and of the trilinear query,
against brute force, closed forms and invariants -- never against the oracle itself."""
import math

import numpy as np
import pytest

import oracle
from paper_1611_03631_gb300 import scenes

SQ2 = math.sqrt(2.0)
SQ3 = math.sqrt(3.0)


def _offsets():
    return [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1) if (dx, dy, dz) != (0, 0, 0)]


def brute_esdf(D, W, v, gamma, dmax, fp32=False, occupancy=False):
    """26-connected quasi-Euclidean distance by plain Bellman-Ford sweeps to a fixpoint.

    Sources: observed voxels with |D| < gamma (value |D|); with occupancy=True, observed voxels
    with D < 0 (value 0, every observed voxel positive). Relaxation runs only into observed,
    non-fixed voxels of the same sign. Values are capped at dmax. Unobserved -> NaN."""
    dt = np.float32 if fp32 else np.float64
    Df = D.astype(np.float32)
    obs = W > 0
    if occupancy:
        sign = np.ones(D.shape)
        fixed = obs & (Df < 0)
        seed = np.zeros(D.shape)
    else:
        sign = np.where(Df >= 0, 1.0, -1.0)
        fixed = obs & (np.abs(Df) < np.float32(gamma))
        seed = np.where(Df == 0, 0.0, np.abs(Df).astype(np.float64) if fp32 else np.abs(D))
    dist = np.full(D.shape, dt(np.float32(dmax)), dtype=dt)  # the map holds d_max as float32
    dist[fixed] = seed[fixed].astype(dt)
    if fp32:
        v32 = np.float32(v)
        L = {1: v32, 2: v32 * np.float32(1.41421356237309515), 3: v32 * np.float32(1.73205080756887719)}
    else:
        v64 = float(np.float32(v))  # the map stores the voxel size as float32
        L = {1: v64, 2: v64 * SQ2, 3: v64 * SQ3}
    G = D.shape
    pad = lambda a, fill: np.pad(a, 1, constant_values=fill)
    while True:
        dp = pad(dist, dt(np.inf))
        op = pad(obs, False)
        sp = pad(sign, 0.0)
        new = dist.copy()
        for dx, dy, dz in _offsets():
            sl = (slice(1 + dx, 1 + dx + G[0]), slice(1 + dy, 1 + dy + G[1]), slice(1 + dz, 1 + dz + G[2]))
            cand = (dp[sl] + L[abs(dx) + abs(dy) + abs(dz)]).astype(dt)
            ok = obs & ~fixed & op[sl] & (sp[sl] == sign) & (cand < new)
            new = np.where(ok, cand, new)
        if np.array_equal(new, dist):
            break
        dist = new
    out = np.where(obs, sign * dist.astype(np.float64), np.nan)
    return out


def grid_to_map(m, D, W, origin=(0, 0, 0), mask=None):
    G = D.shape
    idx = np.stack(np.meshgrid(*[np.arange(g) for g in G], indexing="ij"), -1).reshape(-1, 3)
    sel = np.ones(len(idx), bool) if mask is None else mask.reshape(-1)
    vox = idx[sel] + np.array(origin)
    m.set_tsdf(vox, D.reshape(-1)[sel], W.reshape(-1)[sel])


def map_to_grid(m, G, origin=(0, 0, 0)):
    ex = m.export()
    B = m.B
    out = np.full(G, np.nan)
    for b, k in enumerate(ex["keys"]):
        for l in range(B ** 3):
            c = np.array([k[0] * B + l % B, k[1] * B + (l // B) % B, k[2] * B + l // (B * B)]) - np.array(origin)
            if np.all(c >= 0) and np.all(c < np.array(G)) and ex["flags"][b, l] & 1:
                out[tuple(c)] = ex["d"][b, l]
    return out, ex


def _spheres_tsdf(G, v, delta, centers, radii, inside_neg=True):
    idx = np.stack(np.meshgrid(*[np.arange(g) for g in G], indexing="ij"), -1).astype(np.float64)
    x = (idx + 0.5) * v
    sdf = np.full(G, np.inf)
    for c, r in zip(centers, radii):
        sdf = np.minimum(sdf, np.linalg.norm(x - np.array(c) * v, axis=-1) - r * v)
    return np.clip(sdf, -delta, delta)


# ------------------------------------------------------------------ closed forms


def test_single_seed_gives_exact_chamfer_ball():
    v, G = 0.1, (16, 16, 16)
    D = np.full(G, 0.5)
    D[8, 8, 8] = 0.0
    W = np.ones(G)
    m = oracle.OracleMap(v, 16, 0.5, 10.0, fixed_band=v)
    grid_to_map(m, D, W)
    m.update_esdf()
    got, _ = map_to_grid(m, G)
    v32 = float(np.float32(v))  # the map stores the voxel size as float32
    for i in range(16):
        for j in range(16):
            for k in range(16):
                a, b, c = sorted([abs(i - 8), abs(j - 8), abs(k - 8)], reverse=True)
                exp = v32 * (c * SQ3 + (b - c) * SQ2 + (a - b))
                assert got[i, j, k] == pytest.approx(exp, abs=1e-12)
                # a grid path is never shorter than the straight line between centres
                assert got[i, j, k] >= v * math.sqrt(a * a + b * b + c * c) - 1e-12


def test_axis_aligned_plane_is_exact():
    v, G = 0.1, (8, 8, 16)
    z0 = 4.3 * v
    k = np.arange(16)
    zc = (k + 0.5) * v - z0
    D = np.broadcast_to(np.clip(zc, -0.3, 0.3), G).copy()
    W = np.ones(G)
    m = oracle.OracleMap(v, 8, 0.3, 2.0, fixed_band=v)
    grid_to_map(m, D, W)
    m.update_esdf()
    got, _ = map_to_grid(m, G)
    exp = np.broadcast_to(zc, G)
    # exact up to the float32 voxel size used for the step length (<= 12 steps)
    assert np.max(np.abs(got - exp)) < 1e-7


def test_raise_removing_the_only_seed_returns_to_dmax():
    v, G = 0.1, (16, 16, 16)
    D = np.full(G, 0.5)
    D[3, 4, 5] = 0.02
    W = np.ones(G)
    m = oracle.OracleMap(v, 8, 0.5, 1.0, fixed_band=v)
    grid_to_map(m, D, W)
    m.update_esdf()
    got, _ = map_to_grid(m, G)
    assert got[3, 4, 6] == pytest.approx(0.02 + v, abs=1e-7)
    # the seed leaves the band: its whole subtree is raised back to d_max
    m.set_tsdf(np.array([[3, 4, 5]]), np.array([0.5]), np.array([1.0]))
    m.update_esdf()
    got, _ = map_to_grid(m, G)
    assert np.all(got == 1.0)
    assert m.stats()["raise_pops"] > 100


# ---------------------------------------------------------------- brute force


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("B", [8, 16])
def test_incremental_matches_bellman_ford_over_updates(fp32, B):
    rng = np.random.default_rng(7 + B + 10 * fp32)
    v, G, delta, gamma, dmax = 0.1, (16, 16, 16), 0.3, 0.1, 1.2
    W = (rng.uniform(size=G) > 0.08).astype(np.float64)
    cs = [rng.uniform(2, 14, 3) for _ in range(3)]
    rs = list(rng.uniform(1.5, 4.0, 3))
    D = _spheres_tsdf(G, v, delta, cs, rs) + rng.normal(0, 0.01, G)
    pq = oracle.OracleMap(v, B, delta, dmax, fixed_band=gamma, esdf_fp32=int(fp32))
    ff = oracle.OracleMap(v, B, delta, dmax, fixed_band=gamma, esdf_fp32=int(fp32))
    grid_to_map(pq, D, W, mask=W > 0)
    grid_to_map(ff, D, W, mask=W > 0)
    for step in range(6):
        pq.update_esdf(fifo=False)
        ff.update_esdf(fifo=True)
        exp = brute_esdf(D, W, v, gamma, dmax, fp32=fp32)
        g1, ex1 = map_to_grid(pq, G)
        g2, _ = map_to_grid(ff, G)
        both = ~np.isnan(exp)
        assert np.array_equal(np.isnan(g1), np.isnan(exp))
        tol = 0.0 if fp32 else 1e-12
        assert np.max(np.abs(g1[both] - exp[both])) <= tol, step
        assert np.max(np.abs(g2[both] - exp[both])) <= tol, step
        # the batch recompute agrees too
        full = pq.full_esdf()
        obs = (ex1["flags"] & 1) > 0
        assert np.max(np.abs(full[obs] - ex1["d"][obs])) <= tol
        # next update: move a sphere, reveal new voxels, perturb values
        cs[step % 3] = cs[step % 3] + rng.normal(0, 1.5, 3)
        newW = np.maximum(W, (rng.uniform(size=G) > 0.5).astype(np.float64))
        D2 = _spheres_tsdf(G, v, delta, cs, rs) + rng.normal(0, 0.01, G)
        changed = (newW > 0) & ((W == 0) | (rng.uniform(size=G) < 0.6))
        D = np.where(changed, D2, D)
        W = newW
        grid_to_map(pq, D, W, mask=changed)
        grid_to_map(ff, D, W, mask=changed)


@pytest.mark.parametrize("fp32", [False, True])
def test_occupancy_mode_matches_bellman_ford_over_updates(fp32):
    """Occupancy ESDF (negative TSDF voxels occupied at distance 0, Sec. VI-B): incremental
    updates with moved spheres and new voxels equal Bellman-Ford from the occupied voxels."""
    rng = np.random.default_rng(31 + fp32)
    v, G, delta, dmax = 0.1, (16, 16, 16), 0.3, 1.2
    W = (rng.uniform(size=G) > 0.08).astype(np.float64)
    cs = [rng.uniform(2, 14, 3) for _ in range(3)]
    rs = list(rng.uniform(1.5, 4.0, 3))
    D = _spheres_tsdf(G, v, delta, cs, rs) + rng.normal(0, 0.01, G)
    m = oracle.OracleMap(v, 8, delta, dmax, esdf_fp32=int(fp32), esdf_mode=1)
    grid_to_map(m, D, W, mask=W > 0)
    for step in range(5):
        m.update_esdf()
        exp = brute_esdf(D, W, v, 0.0, dmax, fp32=fp32, occupancy=True)
        got, ex = map_to_grid(m, G)
        both = ~np.isnan(exp)
        assert np.array_equal(np.isnan(got), np.isnan(exp))
        assert np.max(np.abs(got[both] - exp[both])) <= (0.0 if fp32 else 1e-12), step
        assert (got[both] >= 0).all()  # unsigned
        occ = both & (D.astype(np.float32) < 0)
        assert (got[occ] == 0).all()
        full = m.full_esdf()
        obs = (ex["flags"] & 1) > 0
        assert np.max(np.abs(full[obs] - ex["d"][obs])) <= (0.0 if fp32 else 1e-12)
        cs[step % 3] = cs[step % 3] + rng.normal(0, 1.5, 3)
        newW = np.maximum(W, (rng.uniform(size=G) > 0.5).astype(np.float64))
        D2 = _spheres_tsdf(G, v, delta, cs, rs) + rng.normal(0, 0.01, G)
        changed = (newW > 0) & ((W == 0) | (rng.uniform(size=G) < 0.6))
        D = np.where(changed, D2, D)
        W = newW
        grid_to_map(m, D, W, mask=changed)


def test_occupancy_single_occupied_voxel_gives_chamfer_ball_from_zero():
    v, G = 0.1, (16, 16, 16)
    D = np.full(G, 0.5)
    D[8, 8, 8] = -0.05  # the one occupied voxel
    W = np.ones(G)
    m = oracle.OracleMap(v, 16, 0.5, 10.0, esdf_mode=1)
    grid_to_map(m, D, W)
    m.update_esdf()
    got, _ = map_to_grid(m, G)
    v32 = float(np.float32(v))
    for i in range(16):
        for j in range(16):
            for k in range(16):
                a, b, c = sorted([abs(i - 8), abs(j - 8), abs(k - 8)], reverse=True)
                assert got[i, j, k] == pytest.approx(v32 * (c * SQ3 + (b - c) * SQ2 + (a - b)), abs=1e-12)


def test_parent_directions_are_valid():
    """Every non-fixed voxel below d_max has a parent whose value plus the step gives it."""
    rng = np.random.default_rng(5)
    v, G = 0.1, (16, 16, 16)
    D = _spheres_tsdf(G, v, 0.3, [rng.uniform(3, 13, 3)], [3.0])
    m = oracle.OracleMap(v, 16, 0.3, 1.0, fixed_band=v)
    grid_to_map(m, D, np.ones(G))
    m.update_esdf()
    ex = m.export()
    d, par, fl = ex["d"][0], ex["parent"][0], ex["flags"][0]
    checked = 0
    for l in range(16 ** 3):
        if (fl[l] & 2) or abs(d[l]) >= 1.0:
            continue
        x, y, z = l % 16, (l // 16) % 16, l // 256
        k = int(par[l])
        assert k != 255 and k != 13
        dx, dy, dz = k // 9 - 1, (k // 3) % 3 - 1, k % 3 - 1
        pl = (z + dz) * 256 + (y + dy) * 16 + (x + dx)
        L = float(np.float32(v)) * [0, 1, SQ2, SQ3][abs(dx) + abs(dy) + abs(dz)]
        assert abs(d[l]) == pytest.approx(abs(d[pl]) + L, abs=1e-12)
        checked += 1
    assert checked > 1000


# -------------------------------------------------------- scene: incremental == batch


def test_incremental_equals_batch_on_plane_sphere_frames():
    s = scenes.plane_sphere(frames=3, width=32, height=24, fx=25.0, fy=25.0, cx=16.0, cy=12.0)
    for fifo in (False, True):
        m = oracle.OracleMap.from_scene_params(s.params)
        for i in range(len(s)):
            m.integrate(s.points[i], s.poses[i])
            m.update_esdf(fifo=fifo)
            ex = m.export()
            obs = (ex["flags"] & 1) > 0
            assert np.array_equal(obs, ex["W"] > 0)  # observed flags follow the TSDF
            full = m.full_esdf()
            assert np.max(np.abs(full[obs] - ex["d"][obs])) == 0.0
            assert np.all(np.abs(ex["d"][obs]) <= 2.0)


# ----------------------------------------------------------------- trilinear query


def test_query_reproduces_linear_field_and_gradient():
    v = 0.1
    a, b, c, e = 0.3, -0.7, 0.45, 0.2
    idx = np.stack(np.meshgrid(np.arange(-3, 5), np.arange(2, 9), np.arange(-6, 0), indexing="ij"), -1).reshape(-1, 3)
    ctr = (idx + 0.5) * v
    dv = a * ctr[:, 0] + b * ctr[:, 1] + c * ctr[:, 2] + e
    m = oracle.OracleMap(v, 8, 0.3, 2.0)
    m.set_esdf(idx, dv, np.ones(len(idx), np.uint8))
    rng = np.random.default_rng(1)
    lo = (np.array([-3, 2, -6]) + 0.5) * v + 1e-4
    hi = (np.array([4, 8, -1]) + 0.5) * v - 1e-4
    q = rng.uniform(lo, hi, size=(500, 3)).astype(np.float32)
    dist, grad, status = m.query(q)
    assert np.all(status == 0)
    q64 = q.astype(np.float64)
    exp = a * q64[:, 0] + b * q64[:, 1] + c * q64[:, 2] + e
    assert np.max(np.abs(dist - exp)) < 2e-6
    assert np.allclose(grad, [a, b, c], atol=1e-9)
    # outside the patch one corner is unknown
    qo = np.array([[(-3 + 0.5) * v - 0.01, 0.3, -0.3], [0.0, (8 + 0.5) * v + 0.01, -0.3]], np.float32)
    d2, g2, s2 = m.query(qo)
    assert np.all(s2 == 1) and np.all(np.isnan(d2))


def test_query_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    v = 0.2
    idx = np.stack(np.meshgrid(np.arange(0, 6), np.arange(0, 6), np.arange(0, 6), indexing="ij"), -1).reshape(-1, 3)
    dv = rng.uniform(-1, 1, len(idx))
    m = oracle.OracleMap(v, 8, 0.6, 5.0)
    m.set_esdf(idx, dv, np.ones(len(idx), np.uint8))
    # points well inside cells so that +-h stays in the same cell
    cell = rng.integers(0, 5, size=(200, 3))
    f = rng.uniform(0.2, 0.8, size=(200, 3))
    q = ((cell + 0.5 + f) * v).astype(np.float32)
    h = 1e-3
    d0, g0, s0 = m.query(q)
    assert np.all(s0 == 0)
    for ax in range(3):
        qp = q.astype(np.float64).copy()
        qm = q.astype(np.float64).copy()
        qp[:, ax] += h
        qm[:, ax] -= h
        dp, _, _ = m.query(qp.astype(np.float32))
        dm, _, _ = m.query(qm.astype(np.float32))
        step = qp[:, ax].astype(np.float32).astype(np.float64) - qm[:, ax].astype(np.float32).astype(np.float64)
        fd = (dp - dm) / step
        assert np.max(np.abs(fd - g0[:, ax])) < 2e-3


# ----------------------------------------------------- error-analysis constants (Sec. V-B)


def test_error_analysis_constants():
    """The closed forms of Sec. V-B, by numerical quadrature (sanity check of the readings
    of the fixed band and quasi-Euclidean steps; no oracle involved)."""
    th = np.linspace(math.pi / 20, math.pi / 2, 200001)
    Erp = np.trapezoid(20 / (9 * math.pi) * (np.sin(th) - 1.0), th)
    assert Erp == pytest.approx(-0.3014, abs=1e-4)
    rq = lambda phi: 1.0 - np.sin(5 * math.pi / 8 - phi) / math.sin(3 * math.pi / 8)
    assert rq(math.pi / 8) == pytest.approx(-0.0824, abs=1e-4)
    ph = np.linspace(0, math.pi / 4, 200001)
    assert np.trapezoid(4 / math.pi * rq(ph), ph) == pytest.approx(-0.0548, abs=1e-4)

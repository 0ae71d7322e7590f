"""Pins of the oracle's full-Euclidean ESDF variant (Sec. V-A: the parent holds the full offset
to the site; reading R13), against closed forms, brute force and order-free invariants.

Nearest-site propagation through neighbours depends on the processing order, so the variant
has no single result to compare with; every result must instead satisfy, on each observed
non-fixed voxel n:
  * consistency: n's value is exactly the distance its stored site offers it,
    |d_s| + v * ||n - s||, and the site is an observed fixed voxel of n's sign;
  * local optimality: no observed same-sign neighbour's site offers n a smaller distance;
  * bounds: the brute-force minimum over all same-sign fixed voxels of their offer (capped at
    d_max) <= n's value <= the quasi-Euclidean value of the same map (Bellman-Ford).
A stale site after a raise breaks consistency, a missed relaxation breaks local optimality."""
import math

import numpy as np
import pytest

import oracle
from paper_1611_03631_gb300 import scenes
from test_oracle_esdf import _spheres_tsdf, brute_esdf, grid_to_map


def _offer(dsite, s, n, v, fp32):
    """Distance a site s (value dsite) offers voxel n."""
    q = float(np.sum((np.asarray(n, np.int64) - np.asarray(s, np.int64)) ** 2))
    if fp32:
        return float(np.float32(abs(np.float32(dsite))) + np.float32(np.float32(v) * np.sqrt(np.float32(q))))
    return abs(dsite) + float(np.float32(v)) * math.sqrt(q)


def _grid_state(m, G):
    """Per grid voxel: value (NaN unobserved), fixed flag, site (or None)."""
    ex = m.export()
    off, has = m.export_sites()
    B = m.B
    val = np.full(G, np.nan)
    fixed = np.zeros(G, bool)
    site = {}
    for b, k in enumerate(ex["keys"]):
        for l in range(B ** 3):
            c = (k[0] * B + l % B, k[1] * B + (l // B) % B, k[2] * B + l // (B * B))
            if not all(0 <= c[i] < G[i] for i in range(3)) or not (ex["flags"][b, l] & 1):
                continue
            val[c] = ex["d"][b, l]
            fixed[c] = bool(ex["flags"][b, l] & 2)
            if has[b, l]:
                site[c] = tuple(int(c[i] + off[b, l, i]) for i in range(3))
    return val, fixed, site


def check_invariants(m, D, W, v, gamma, dmax, fp32, G):
    val, fixed, site = _grid_state(m, G)
    obs = ~np.isnan(val)
    assert np.array_equal(obs, W > 0)
    dmax32 = float(np.float32(dmax))
    quasi = brute_esdf(D, W, v, gamma, dmax, fp32=fp32)
    seeds = [tuple(c) for c in np.argwhere(fixed)]
    sv = np.array([val[s] for s in seeds])
    sp = np.array(seeds, np.int64).reshape(-1, 3)
    stats = dict(voxels=0, exact=0, max_excess=0.0)
    for n in map(tuple, np.argwhere(obs & ~fixed)):
        d = val[n]
        s = site.get(n)
        if s is None:
            assert abs(d) == dmax32, (n, d)
        else:
            assert all(0 <= s[i] < G[i] for i in range(3)) and fixed[s], (n, s)
            assert (val[s] >= 0) == (d >= 0), (n, s)
            assert abs(d) == _offer(val[s], s, n, v, fp32), (n, s, d)
        # local optimality against every observed same-sign neighbour's site
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    p = (n[0] + dx, n[1] + dy, n[2] + dz)
                    if p == n or not all(0 <= p[i] < G[i] for i in range(3)) or not obs[p]:
                        continue
                    if (val[p] >= 0) != (d >= 0):
                        continue
                    ps = p if fixed[p] else site.get(p)
                    if ps is None:
                        continue
                    assert abs(d) <= _offer(val[ps], ps, n, v, fp32), (n, p, ps)
        # bounds: brute force over all same-sign seeds, and the quasi-Euclidean value
        same = (sv >= 0) == (d >= 0)
        if fp32:
            q = np.sum((sp[same] - np.array(n)) ** 2, axis=1).astype(np.float32)
            offers = np.abs(sv[same]).astype(np.float32) + np.float32(v) * np.sqrt(q)
        else:
            q = np.sum((sp[same] - np.array(n)) ** 2, axis=1).astype(np.float64)
            offers = np.abs(sv[same]) + float(np.float32(v)) * np.sqrt(q)
        lo = min(float(offers.min()) if offers.size else np.inf, dmax32)
        assert abs(d) >= lo, (n, d, lo)
        assert abs(d) <= abs(quasi[n]) + 1e-6, (n, d, quasi[n])
        stats["voxels"] += 1
        stats["exact"] += int(abs(d) == lo)
        stats["max_excess"] = max(stats["max_excess"], abs(d) - lo)
    return stats


def test_single_seed_gives_the_euclidean_distance_to_it():
    v, G, dmax = 0.1, (16, 16, 16), 10.0
    D = np.full(G, 0.5)
    D[8, 7, 9] = 0.0
    W = np.ones(G)
    m = oracle.OracleMap(v, 8, 0.5, dmax, fixed_band=v, euclidean=1)
    grid_to_map(m, D, W)
    m.update_esdf()
    val, fixed, site = _grid_state(m, G)
    v64 = float(np.float32(v))
    for n in map(tuple, np.argwhere(~fixed)):
        assert site[n] == (8, 7, 9)
        exp = v64 * math.sqrt((n[0] - 8) ** 2 + (n[1] - 7) ** 2 + (n[2] - 9) ** 2)
        assert val[n] == pytest.approx(exp, abs=1e-12), n


def test_axis_aligned_plane_is_exact():
    """Seeds on a plane of voxels: every voxel's nearest seed is straight below or above it."""
    v, G, delta, dmax = 0.1, (8, 8, 16), 0.3, 10.0
    z0 = 4.3 * v
    zc = (np.arange(16) + 0.5) * v - z0
    D = np.broadcast_to(np.clip(zc, -delta, delta), G).copy()
    W = np.ones(G)
    m = oracle.OracleMap(v, 8, delta, dmax, fixed_band=v, euclidean=1)
    grid_to_map(m, D, W)
    m.update_esdf()
    val, fixed, _ = _grid_state(m, G)
    v64 = float(np.float32(v))
    for n in map(tuple, np.argwhere(~fixed)):
        k = n[2]
        ks = 4 if k >= 4 else 3  # the seed layer on n's side of the plane (|zc| < v at k = 3, 4)
        assert fixed[n[0], n[1], ks]
        exp = abs(D[n[0], n[1], ks]) + v64 * abs(k - ks)
        assert abs(val[n]) == pytest.approx(exp, abs=1e-12), n


@pytest.mark.parametrize("fp32", [False, True])
def test_invariants_and_bounds_over_incremental_updates(fp32):
    """Spheres that move, voxels revealed, values perturbed, seeds leaving and entering the band:
    after every update the result is consistent, locally optimal and within its bounds."""
    rng = np.random.default_rng(11 + fp32)
    v, G, delta, gamma, dmax = 0.1, (16, 16, 16), 0.3, 0.1, 1.2
    W = (rng.uniform(size=G) > 0.08).astype(np.float64)
    cs = [rng.uniform(2, 14, 3) for _ in range(3)]
    rs = list(rng.uniform(1.5, 4.0, 3))
    D = _spheres_tsdf(G, v, delta, cs, rs) + rng.normal(0, 0.01, G)
    maps = [oracle.OracleMap(v, 8, delta, dmax, fixed_band=gamma, esdf_fp32=int(fp32), euclidean=1) for _ in range(2)]
    for m in maps:
        grid_to_map(m, D, W, mask=W > 0)
    total = dict(voxels=0, exact=0, raised=0)
    for step in range(6):
        for fifo, m in enumerate(maps):
            m.update_esdf(fifo=bool(fifo))
            st = check_invariants(m, D, W, v, gamma, dmax, fp32, G)
            total["voxels"] += st["voxels"]
            total["exact"] += st["exact"]
            total["raised"] += m.stats()["raise_pops"]
            assert st["max_excess"] <= 0.5 * v
        cs[step % 3] = cs[step % 3] + rng.normal(0, 1.5, 3)
        newW = np.maximum(W, (rng.uniform(size=G) > 0.5).astype(np.float64))
        D2 = _spheres_tsdf(G, v, delta, cs, rs) + rng.normal(0, 0.01, G)
        changed = (newW > 0) & ((W == 0) | (rng.uniform(size=G) < 0.6))
        D = np.where(changed, D2, D)
        W = newW
        for m in maps:
            grid_to_map(m, D, W, mask=changed)
    assert total["raised"] > 0
    # nearest-site propagation finds the exact nearest seed almost everywhere
    assert total["exact"] >= 0.95 * total["voxels"]


def test_raise_drops_every_voxel_measured_to_a_removed_seed():
    """Two seeds; the one most voxels are measured to leaves the band: no voxel keeps it."""
    v, G, delta, dmax = 0.1, (16, 16, 16), 0.5, 10.0
    D = np.full(G, 0.45)
    D[4, 4, 4] = 0.0
    D[12, 12, 12] = 0.05
    W = np.ones(G)
    m = oracle.OracleMap(v, 8, delta, dmax, fixed_band=v, euclidean=1)
    grid_to_map(m, D, W)
    m.update_esdf()
    _, _, site = _grid_state(m, G)
    assert sum(s == (4, 4, 4) for s in site.values()) > 1000
    D[4, 4, 4] = 0.45
    grid_to_map(m, D, W, mask=np.arange(D.size).reshape(G) == np.ravel_multi_index((4, 4, 4), G))
    m.update_esdf()
    val, fixed, site = _grid_state(m, G)
    assert not fixed[4, 4, 4]
    assert set(site.values()) == {(12, 12, 12)}
    v64 = float(np.float32(v))
    for n, s in site.items():
        exp = 0.05 + v64 * math.sqrt(sum((n[i] - 12) ** 2 for i in range(3)))
        assert val[n] == pytest.approx(exp, abs=1e-9), n


def test_euclidean_is_not_above_quasi_and_closer_to_the_true_distance_on_the_scene():
    """Plane + sphere frames fused once, ESDF by both variants from the same TSDF: the Euclidean
    value never exceeds the quasi-Euclidean one, and its error against the analytic distance
    (free voxels near the surfaces) is smaller on average."""
    s = scenes.plane_sphere(frames=3)
    q = oracle.OracleMap.from_scene_params(s.params)
    e = oracle.OracleMap.from_scene_params(s.params, euclidean=1)
    for i in range(len(s)):
        for m in (q, e):
            m.integrate(s.points[i], s.poses[i])
            m.update_esdf()
    eq, ee = q.export(), e.export()
    assert np.array_equal(eq["keys"], ee["keys"]) and np.array_equal(eq["flags"], ee["flags"])
    obs = (eq["flags"] & 1) > 0
    assert np.all(np.abs(ee["d"][obs]) <= np.abs(eq["d"][obs]) + 1e-9)
    B, v = q.B, s.params["voxel_size"]
    l = np.arange(B ** 3)
    loc = np.stack([l % B, (l // B) % B, l // (B * B)], -1)
    x = ((eq["keys"][:, None, :] * B + loc[None]) + 0.5) * v
    sdf = scenes.plane_sphere_sdf(x)
    free = obs & (eq["d"] > 0) & (sdf > 0.3) & (sdf < 1.5) & ((eq["flags"] & 2) == 0)
    err_q = np.mean(np.abs(eq["d"][free] - sdf[free]))
    err_e = np.mean(np.abs(ee["d"][free] - sdf[free]))
    assert free.sum() > 1000 and err_e < err_q

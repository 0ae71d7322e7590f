"""Comparison helpers shared by the GPU parity tests (no compute of the method here)."""
from __future__ import annotations

import math

import numpy as np

# Tolerances of the map update (float32 GPU path against the float64-accumulated oracle).
TOL_D = 1e-5  # |delta TSDF distance| in metres
TOL_W_REL = 1e-6  # relative TSDF weight error
TOL_ESDF = 1e-4  # |delta ESDF distance| in metres


def sort_rows(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a)
    if len(a) == 0:
        return a.reshape(0, 3)
    return a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]


def compare_tsdf(gex: dict, oex: dict, B: int) -> dict:
    """Block sets, observed flags (bit-exact), D and W errors on observed voxels."""
    assert np.array_equal(gex["keys"], oex["keys"]), "allocated block sets differ"
    gobs = gex["W"] > 0
    oobs = oex["W"] > 0
    assert np.array_equal(gobs, oobs), f"observed sets differ in {int(np.sum(gobs != oobs))} voxels"
    dD = np.abs(gex["D"][gobs].astype(np.float64) - oex["D"][oobs])
    rW = np.abs(gex["W"][gobs].astype(np.float64) - oex["W"][oobs]) / oex["W"][oobs]
    return dict(
        blocks=len(gex["keys"]),
        observed=int(gobs.sum()),
        max_dD=float(dD.max()) if dD.size else 0.0,
        max_rel_dW=float(rW.max()) if rW.size else 0.0,
    )


def voxel_coords(keys: np.ndarray, B: int) -> np.ndarray:
    l = np.arange(B ** 3)
    loc = np.stack([l % B, (l // B) % B, l // (B * B)], -1)
    return keys[:, None, :] * B + loc[None]


def check_parents(ex: dict, B: int, L: tuple) -> int:
    """Every non-fixed observed voxel below d_max with a parent gets exactly |d_parent| + L_k
    from it (the parent tree is valid even where equal candidates make it non-unique)."""
    keys = ex["keys"]
    idx = {tuple(k): i for i, k in enumerate(keys)}
    d, par, fl = ex["d"], ex["parent"], ex["flags"]
    bad = 0
    checked = 0
    nb = len(keys)
    for b in range(nb):
        for l in np.nonzero(((fl[b] & 3) == 1) & (par[b] != 255))[0]:
            k = int(par[b, l])
            dx, dy, dz = k // 9 - 1, (k // 3) % 3 - 1, k % 3 - 1
            x = keys[b, 0] * B + l % B + dx
            y = keys[b, 1] * B + (l // B) % B + dy
            z = keys[b, 2] * B + l // (B * B) + dz
            j = idx.get((x // B, y // B, z // B))
            if j is None:
                bad += 1
                continue
            pl = ((z % B) * B + (y % B)) * B + (x % B)
            step = L[abs(dx) + abs(dy) + abs(dz)]
            exp = np.float32(np.float32(abs(d[j, pl])) + np.float32(step))
            if np.float32(abs(d[b, l])) != exp:
                bad += 1
            checked += 1
    return bad, checked


def compare_with_oracle(gex: dict, oex: dict, params: dict) -> dict:
    """A GPU map export against the float64 oracle's after the same scans and ESDF updates:
    block sets and observed flags bit-exact, |dD| <= 1e-5 m, relative dW <= 1e-6, then the ESDF.
    Seeds whose oracle TSDF value lies within 1e-5 m of the band edge or of zero may
    legitimately differ (float32 against float64 accumulation) and are excluded together with
    their d_max neighbourhood; every other seed must match, and |dd| <= 1e-4 m."""
    B = int(params["voxels_per_block"])
    r = compare_tsdf(gex, oex, B)
    assert r["max_dD"] <= TOL_D and r["max_rel_dW"] <= TOL_W_REL, r
    gobs, oobs = (gex["flags"] & 1) > 0, (oex["flags"] & 1) > 0
    assert np.array_equal(gobs, oobs), "ESDF observed flags differ"
    gfix, ofix = (gex["flags"] & 2) > 0, (oex["flags"] & 2) > 0
    Do = oex["D"].astype(np.float32)
    gamma = np.float32(params["fixed_band"])
    ambiguous = (np.abs(np.abs(Do) - gamma) < 1e-5) | (np.abs(Do) < 1e-5)
    diff = ((gfix != ofix) | (np.sign(gex["D"]) != np.sign(Do))) & oobs
    assert not np.any(diff & ~ambiguous), "seed sets differ outside the guard band"
    mask = oobs.copy()
    if np.any(diff):
        vc = voxel_coords(gex["keys"], B)
        rad = int(math.ceil(params["max_esdf_dist"] / params["voxel_size"])) + 1
        for c in vc[diff]:
            mask &= ~(np.max(np.abs(vc - c), axis=-1) <= rad)
    err = np.abs(gex["d"][mask].astype(np.float64) - oex["d"][mask])
    r["max_dd"] = float(err.max()) if err.size else 0.0
    r["excluded_seeds"] = int(diff.sum())
    assert r["max_dd"] <= TOL_ESDF, r
    return r


def _block_codes(keys: np.ndarray) -> np.ndarray:
    k = keys.astype(np.int64) + (1 << 20)
    return (k[..., 0] << 42) | (k[..., 1] << 21) | k[..., 2]


def euclid_invariants(ex: dict, off: np.ndarray, has: np.ndarray, v: float, dmax: float, quasi_d=None) -> dict:
    """Order-free checks of a full-Euclidean ESDF export (blocks sorted by key; off/has from
    export_sites in the same order), on every observed non-fixed voxel n:
      * its site (n + offset) is an observed fixed voxel of n's sign, and n's value is exactly the
        float32 offer of that site, |d_s| + v * sqrt(q); a voxel without a site sits at d_max;
      * no observed same-sign neighbour's site (the neighbour itself if fixed) offers n less;
      * |d| <= the quasi-Euclidean value of the same map (quasi_d, same block order), if given.
    Returns counts; raises AssertionError with the first violation."""
    keys, d, fl = ex["keys"], ex["d"].astype(np.float32), ex["flags"]
    nb, B3 = d.shape
    B = round(B3 ** (1 / 3))
    codes = _block_codes(keys)
    order = np.argsort(codes)
    sc = codes[order]
    l = np.arange(B3)
    loc = np.stack([l % B, (l // B) % B, l // (B * B)], -1)
    coords = keys[:, None, :].astype(np.int64) * B + loc[None]  # (nb, B3, 3)
    obs, fixed = (fl & 1) > 0, (fl & 2) > 0
    v32 = np.float32(v)

    def lookup(c):
        """(found, block, local) of voxel coordinates c (..., 3)."""
        bk = np.floor_divide(c, B)
        code = _block_codes(bk)
        pos = np.clip(np.searchsorted(sc, code), 0, len(sc) - 1)
        found = sc[pos] == code
        blk = order[pos]
        lc = c - bk * B
        return found, blk, (lc[..., 2] * B + lc[..., 1]) * B + lc[..., 0]

    def offer(ds, q):
        return np.float32(np.abs(ds).astype(np.float32) + np.float32(v32 * np.sqrt(q.astype(np.float32))))

    sel = obs & ~fixed
    nsel = int(sel.sum())
    # sites and consistency
    hs = sel & has
    c = coords[hs]
    s = c + off[hs].astype(np.int64)
    f, sb, sl = lookup(s)
    assert f.all(), "a site lies in an absent block"
    assert (fixed[sb, sl] & obs[sb, sl]).all(), "a site is not an observed fixed voxel"
    ds = d[sb, sl]
    dn = d[hs]
    assert np.array_equal(ds >= 0, dn >= 0), "a site of the other sign"
    q = np.sum((s - c) ** 2, axis=1)
    assert np.array_equal(np.abs(dn), offer(ds, q)), "a value differs from its site's offer"
    nos = sel & ~has
    assert np.all(np.abs(d[nos]) == np.float32(dmax)), "a voxel without a site below d_max"
    # local optimality: each neighbour's site offers n no less than n holds
    cn = coords[sel]
    dsel = d[sel]
    worse = 0
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                if dx == dy == dz == 0:
                    continue
                p = cn + np.array([dx, dy, dz])
                f, pb, pl = lookup(p)
                f &= obs[pb, pl] & ((d[pb, pl] >= 0) == (dsel >= 0))
                pf = fixed[pb, pl]
                ph = has[pb, pl]
                ok = f & (pf | ph)
                site = np.where(pf[:, None], p, p + off[pb, pl].astype(np.int64))
                sf, sb2, sl2 = lookup(site)
                ok &= sf
                o = offer(d[sb2, sl2], np.sum((site - cn) ** 2, axis=1))
                worse += int(np.sum(ok & (o < np.abs(dsel))))
    assert worse == 0, f"{worse} voxels are offered less by a neighbour's site"
    res = dict(checked=nsel, with_site=int(hs.sum()))
    if quasi_d is not None:
        qd = quasi_d.astype(np.float32)
        excess = np.abs(d[sel]) - np.abs(qd[sel])
        res["max_above_quasi"] = float(excess.max()) if excess.size else 0.0
        assert res["max_above_quasi"] <= 1e-6, res
        res["mean_below_quasi"] = float(-excess.mean()) if excess.size else 0.0
    return res

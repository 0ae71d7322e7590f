"""Comparison helpers shared by the GPU parity tests (no compute of the method here)."""
from __future__ import annotations

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

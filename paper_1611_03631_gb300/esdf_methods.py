"""ESDF construction methods compared on the simulated benchmark of Sec. VI-B.

Each method runs the GPU map update (TSDF integration, then the incremental ESDF after every
scan) on the same scans; the final ESDF is scored against the analytic distance of the scene
at the voxel centres, the evaluation the paper plots in Fig. 7:

  * occupancy      -- negative TSDF voxels are occupied at distance 0 (the occupancy ESDF)
  * half_band      -- fixed band |D| < delta / 2
  * one_voxel_band -- fixed band |D| < v (the method the paper recommends)
  * half_band_euclidean, one_voxel_band_euclidean -- the same bands with full Euclidean
    distances (each voxel keeps the offset to its site) instead of quasi-Euclidean ones; the
    paper reports the error reduction and the time increase of this choice for the half band

Errors are taken over observed free-space voxels whose true distance lies in (0, 1.5] m (below
the ESDF's 2 m cap). Times are GPU times (CUDA events) summed over the scans.
"""
from __future__ import annotations

from typing import Dict

import numpy as np

from . import scenes, vbx

METHODS = ("occupancy", "half_band", "half_band_euclidean", "one_voxel_band", "one_voxel_band_euclidean")
EVAL_MAX_DIST = 1.5


def method_options(method: str, params: Dict[str, float]) -> Dict[str, object]:
    if method == "occupancy":
        return dict(esdf_mode=1)
    if method.endswith("_euclidean"):
        return dict(method_options(method[: -len("_euclidean")], params), euclidean=True)
    if method == "half_band":
        return dict(fixed_band=0.5 * float(params["truncation"]))
    if method == "one_voxel_band":
        return dict(fixed_band=float(params["voxel_size"]))
    raise ValueError(f"unknown ESDF method {method!r}")


def voxel_centres(export: Dict[str, np.ndarray], B: int, v: float) -> np.ndarray:
    """World coordinates (nb, B^3, 3) of the voxel centres of an export."""
    l = np.arange(B ** 3)
    local = np.stack([l % B, (l // B) % B, l // (B * B)], -1)
    idx = export["keys"][:, None, :].astype(np.int64) * B + local[None]
    return (idx + 0.5) * v


def run(scans: scenes.ScanSet, method: str, grouped: bool = True, block_capacity: int = 0) -> Dict[str, float]:
    import torch

    p = scans.params
    m = vbx.Map.from_scene_params(
        p, grouped=grouped, block_capacity=block_capacity, max_points=max(x.shape[0] for x in scans.points), **method_options(method, p)
    )
    pts = [torch.from_numpy(x).cuda() for x in scans.points]
    tsdf_ms = esdf_ms = 0.0
    for x, T in zip(pts, scans.poses):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        m.integrate_scan(x, T)
        e1.record()
        m.update_esdf()
        e2.record()
        e2.synchronize()
        tsdf_ms += e0.elapsed_time(e1)
        esdf_ms += e1.elapsed_time(e2)
    m.sync()
    ex = m.export()
    m.close()
    v = float(np.float32(p["voxel_size"]))
    x = voxel_centres(ex, int(p["voxels_per_block"]), v)
    gt = scenes.esdf_benchmark_sdf(x)
    obs = (ex["flags"] & 1) > 0
    sel = obs & (gt > 0) & (gt <= EVAL_MAX_DIST)
    err = ex["d"][sel].astype(np.float64) - gt[sel]
    # TSDF error near the surface (the TSDF itself does not depend on the ESDF method)
    W = ex["W"]
    near = (W > 0) & (np.abs(gt) < 0.5 * float(p["truncation"]))
    terr = ex["D"][near].astype(np.float64) - gt[near]
    n = len(scans)
    return dict(
        method=method,
        grouped=bool(grouped),
        voxel_size=float(p["voxel_size"]),
        scans=n,
        esdf_voxels_scored=int(sel.sum()),
        esdf_mean_abs_err_m=float(np.mean(np.abs(err))) if err.size else float("nan"),
        esdf_rms_err_m=float(np.sqrt(np.mean(err * err))) if err.size else float("nan"),
        esdf_max_abs_err_m=float(np.max(np.abs(err))) if err.size else float("nan"),
        tsdf_mean_abs_err_m=float(np.mean(np.abs(terr))) if terr.size else float("nan"),
        tsdf_ms_per_scan=tsdf_ms / n,
        esdf_ms_per_scan=esdf_ms / n,
    )


def compare(scans: scenes.ScanSet, voxel_sizes=(0.05, 0.10, 0.20)) -> Dict[str, object]:
    """All methods at each voxel size, plus per-point raycasting against grouped raycasting
    (Sec. IV-B) for the recommended method."""
    out = []
    for v in voxel_sizes:
        s = scenes.ScanSet(scans.name, scans.points, scans.poses, dict(scans.params), dict(scans.meta))
        s.params.update(voxel_size=v, truncation=4.0 * v, eps=v, fixed_band=v)
        for meth in METHODS:
            out.append(run(s, meth))
        out.append(run(s, "one_voxel_band", grouped=False))
    # full Euclidean against quasi-Euclidean distances, per band and voxel size: the ESDF error
    # reduction and the ESDF time increase (Sec. VI-B reports both for the half band)
    by = {(r["method"], r["voxel_size"], r["grouped"]): r for r in out}
    euclid = []
    for v in voxel_sizes:
        vv = float(v)
        for band in ("half_band", "one_voxel_band"):
            q = by.get((band, vv, True))
            e = by.get((band + "_euclidean", vv, True))
            if q is None or e is None:
                continue
            euclid.append(
                dict(
                    band=band,
                    voxel_size=vv,
                    error_reduction_pct=100.0 * (q["esdf_mean_abs_err_m"] - e["esdf_mean_abs_err_m"]) / q["esdf_mean_abs_err_m"],
                    esdf_time_increase_pct=100.0 * (e["esdf_ms_per_scan"] - q["esdf_ms_per_scan"]) / q["esdf_ms_per_scan"],
                )
            )
    return dict(results=out, euclidean_vs_quasi=euclid)

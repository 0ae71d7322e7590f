"""Python handle on the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use this
package. It loads ``libvbx_oracle.so`` (built from ``vbx_oracle.cpp`` by :func:`build`)
through ctypes and exposes the oracle's map, its primitives and its exports as numpy
arrays. It never imports the CUDA library or the product package's compute code.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vbx_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libvbx_oracle.so")

_lib = None


class orc_params(ctypes.Structure):
    _fields_ = [
        ("voxel_size", ctypes.c_float),
        ("voxels_per_block", ctypes.c_int),
        ("truncation", ctypes.c_float),
        ("max_esdf_dist", ctypes.c_float),
        ("weighting", ctypes.c_int),
        ("eps", ctypes.c_float),
        ("fixed_band", ctypes.c_float),
        ("w_max", ctypes.c_float),
        ("max_range", ctypes.c_float),
        ("grouped", ctypes.c_int),
        ("esdf_fp32", ctypes.c_int),
        ("esdf_mode", ctypes.c_int),
        ("euclidean", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (single-threaded, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = [
            "g++",
            "-std=c++17",
            "-O2",
            "-ffp-contract=off",
            "-fno-fast-math",
            "-shared",
            "-fPIC",
            "-o",
            tmp,
            _SRC,
        ]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64
    P = ctypes.POINTER
    lib.orc_create.restype = vp
    lib.orc_create.argtypes = [P(orc_params)]
    lib.orc_destroy.argtypes = [vp]
    lib.orc_integrate.argtypes = [vp, vp, i64, vp]
    lib.orc_update_esdf.argtypes = [vp, ctypes.c_int]
    lib.orc_stats.argtypes = [vp, vp]
    lib.orc_num_blocks.restype = i64
    lib.orc_num_blocks.argtypes = [vp]
    lib.orc_export.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.orc_num_last_updated.restype = i64
    lib.orc_num_last_updated.argtypes = [vp]
    lib.orc_last_updated.argtypes = [vp, vp]
    lib.orc_full_esdf.argtypes = [vp, vp]
    lib.orc_query.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.orc_set_tsdf.argtypes = [vp, vp, vp, vp, i64]
    lib.orc_set_esdf.argtypes = [vp, vp, vp, vp, i64]
    lib.orc_traverse.restype = i64
    lib.orc_traverse.argtypes = [vp, vp, vp, i64]
    lib.orc_projective_distance.restype = ctypes.c_float
    lib.orc_projective_distance.argtypes = [vp, vp, vp, ctypes.c_float, ctypes.c_float]
    lib.orc_record_weight.restype = ctypes.c_float
    lib.orc_record_weight.argtypes = [P(orc_params), ctypes.c_float, ctypes.c_float]
    lib.orc_group.restype = i64
    lib.orc_group.argtypes = [P(orc_params), vp, i64, vp, vp, vp, vp, vp, i64]
    lib.orc_extract_mesh.restype = i64
    lib.orc_extract_mesh.argtypes = [vp, vp, vp, i64]
    lib.orc_export_sites.argtypes = [vp, vp, vp]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_params(
    voxel_size: float,
    voxels_per_block: int,
    truncation: float,
    max_esdf_dist: float,
    weighting: int = 0,
    eps: Optional[float] = None,
    fixed_band: Optional[float] = None,
    w_max: float = 1e4,
    max_range: float = math.inf,
    grouped: int = 1,
    esdf_fp32: int = 0,
    esdf_mode: int = 0,
    euclidean: int = 0,
) -> orc_params:
    return orc_params(
        voxel_size,
        voxels_per_block,
        truncation,
        max_esdf_dist,
        weighting,
        voxel_size if eps is None else eps,
        voxel_size if fixed_band is None else fixed_band,
        w_max,
        max_range,
        grouped,
        esdf_fp32,
        esdf_mode,
        euclidean,
    )


STAT_NAMES = (
    "points_in",
    "points_valid",
    "groups",
    "records",
    "updated",
    "new_blocks",
    "esdf_updated_in",
    "seeds",
    "raise_pops",
    "lower_pops",
    "lower_improve",
)


class OracleMap:
    """One oracle map (std::unordered_map of blocks)."""

    def __init__(self, voxel_size, voxels_per_block, truncation, max_esdf_dist, **kw):
        self._lib = _load()
        self.params = make_params(voxel_size, voxels_per_block, truncation, max_esdf_dist, **kw)
        self.B = voxels_per_block
        self.voxel_size = voxel_size
        self._h = self._lib.orc_create(ctypes.byref(self.params))

    @classmethod
    def from_scene_params(cls, params: Dict[str, float], **kw) -> "OracleMap":
        args = dict(
            weighting=int(params.get("weighting", 0)),
            eps=params.get("eps"),
            fixed_band=params.get("fixed_band"),
            max_range=params.get("max_range", math.inf),
        )
        args.update(kw)
        return cls(params["voxel_size"], params["voxels_per_block"], params["truncation"], params["max_esdf_dist"], **args)

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, points: np.ndarray, T: np.ndarray) -> None:
        p = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
        T = np.ascontiguousarray(T, dtype=np.float32).reshape(16)
        self._lib.orc_integrate(self._h, _ptr(p), p.shape[0], _ptr(T))

    def update_esdf(self, fifo: bool = False) -> None:
        self._lib.orc_update_esdf(self._h, 1 if fifo else 0)

    def stats(self) -> Dict[str, int]:
        out = np.zeros(11, dtype=np.int64)
        self._lib.orc_stats(self._h, _ptr(out))
        return dict(zip(STAT_NAMES, (int(x) for x in out)))

    def num_blocks(self) -> int:
        return int(self._lib.orc_num_blocks(self._h))

    def export(self) -> Dict[str, np.ndarray]:
        nb = self.num_blocks()
        B3 = self.B ** 3
        keys = np.zeros((nb, 3), dtype=np.int32)
        D = np.zeros(nb * B3, dtype=np.float64)
        W = np.zeros(nb * B3, dtype=np.float64)
        d = np.zeros(nb * B3, dtype=np.float64)
        parent = np.zeros(nb * B3, dtype=np.uint8)
        flags = np.zeros(nb * B3, dtype=np.uint8)
        self._lib.orc_export(self._h, _ptr(keys), _ptr(D), _ptr(W), _ptr(d), _ptr(parent), _ptr(flags))
        return dict(
            keys=keys,
            D=D.reshape(nb, B3),
            W=W.reshape(nb, B3),
            d=d.reshape(nb, B3),
            parent=parent.reshape(nb, B3),
            flags=flags.reshape(nb, B3),
        )

    def export_sites(self):
        """Euclidean variant: (offsets, has_site) in the block order of export(); offsets are
        site - voxel as (nb, B^3, 3) int32, has_site (nb, B^3) bool."""
        nb = self.num_blocks()
        B3 = self.B ** 3
        off = np.zeros(nb * B3 * 3, dtype=np.int32)
        has = np.zeros(nb * B3, dtype=np.uint8)
        self._lib.orc_export_sites(self._h, _ptr(off), _ptr(has))
        return off.reshape(nb, B3, 3), has.reshape(nb, B3).astype(bool)

    def last_updated(self) -> np.ndarray:
        n = int(self._lib.orc_num_last_updated(self._h))
        out = np.zeros((n, 3), dtype=np.int32)
        if n:
            self._lib.orc_last_updated(self._h, _ptr(out))
        return out

    def full_esdf(self) -> np.ndarray:
        nb = self.num_blocks()
        out = np.zeros(nb * self.B ** 3, dtype=np.float64)
        self._lib.orc_full_esdf(self._h, _ptr(out))
        return out.reshape(nb, self.B ** 3)

    def query(self, q: np.ndarray):
        q = np.ascontiguousarray(q, dtype=np.float32).reshape(-1, 3)
        n = q.shape[0]
        dist = np.zeros(n, dtype=np.float64)
        grad = np.zeros((n, 3), dtype=np.float64)
        status = np.zeros(n, dtype=np.uint8)
        self._lib.orc_query(self._h, _ptr(q), n, _ptr(dist), _ptr(grad), _ptr(status))
        return dist, grad, status

    def extract_mesh(self):
        """Triangles of the TSDF iso-surface (reading R12), sorted by (cell, index in cell):
        cells (n, 4) int32 = cell min-corner voxel and index, verts (n, 3, 3) float32."""
        n = int(self._lib.orc_extract_mesh(self._h, None, None, 0))
        cells = np.zeros((max(n, 1), 4), np.int32)
        verts = np.zeros((max(n, 1), 3, 3), np.float32)
        self._lib.orc_extract_mesh(self._h, _ptr(cells), _ptr(verts), n)
        return cells[:n], verts[:n]

    def set_tsdf(self, vox: np.ndarray, D: np.ndarray, W: np.ndarray) -> None:
        vox = np.ascontiguousarray(vox, dtype=np.int32).reshape(-1, 3)
        D = np.ascontiguousarray(D, dtype=np.float64).reshape(-1)
        W = np.ascontiguousarray(W, dtype=np.float64).reshape(-1)
        self._lib.orc_set_tsdf(self._h, _ptr(vox), _ptr(D), _ptr(W), vox.shape[0])

    def set_esdf(self, vox: np.ndarray, d: np.ndarray, observed: np.ndarray) -> None:
        vox = np.ascontiguousarray(vox, dtype=np.int32).reshape(-1, 3)
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1)
        observed = np.ascontiguousarray(observed, dtype=np.uint8).reshape(-1)
        self._lib.orc_set_esdf(self._h, _ptr(vox), _ptr(d), _ptr(observed), vox.shape[0])


# ------------------------------------------------------------------------------------------
# primitives


def traverse(S, E) -> np.ndarray:
    """Voxels visited by the integer DDA from fixed-point S to E (65536 units per voxel)."""
    lib = _load()
    S = np.ascontiguousarray(S, dtype=np.int64)
    E = np.ascontiguousarray(E, dtype=np.int64)
    cap = int(np.sum(np.abs((E >> 16) - (S >> 16)))) + 1
    out = np.zeros((cap, 3), dtype=np.int32)
    n = lib.orc_traverse(_ptr(S), _ptr(E), _ptr(out), cap)
    assert n == cap
    return out


def projective_distance(pbar, s, c, v, delta) -> float:
    lib = _load()
    pbar = np.ascontiguousarray(pbar, dtype=np.float32)
    s = np.ascontiguousarray(s, dtype=np.float32)
    c = np.ascontiguousarray(c, dtype=np.int32)
    return float(lib.orc_projective_distance(_ptr(pbar), _ptr(s), _ptr(c), v, delta))


def record_weight(params: orc_params, Wg: float, d: float) -> float:
    return float(_load().orc_record_weight(ctypes.byref(params), Wg, d))


def group(params: orc_params, points: np.ndarray, T: np.ndarray):
    """Grouped-raycasting bins: (keys int32 (G,3), pbar float32 (G,3), W_g (G,), count (G,))."""
    lib = _load()
    p = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
    T = np.ascontiguousarray(T, dtype=np.float32).reshape(16)
    cap = p.shape[0]
    keys = np.zeros((cap, 3), dtype=np.int32)
    pbar = np.zeros((cap, 3), dtype=np.float32)
    Wg = np.zeros(cap, dtype=np.float32)
    count = np.zeros(cap, dtype=np.int64)
    n = lib.orc_group(ctypes.byref(params), _ptr(p), cap, _ptr(T), _ptr(keys), _ptr(pbar), _ptr(Wg), _ptr(count), cap)
    return keys[:n], pbar[:n], Wg[:n], count[:n]

"""Thin Python binding of the C ABI in ``include/vbx.h`` (argument marshalling only).

Every step of the map update runs in the CUDA library ``_build/libvbx.so``; this module
only converts arguments (torch device tensors for device memory, numpy arrays for host
data) and checks statuses. There is no CPU fallback: without the library or a CUDA device
every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvbx.so")

VBX_OK = 0
STATUS_NAMES = {
    0: "VBX_OK",
    1: "VBX_ERR_INVALID_ARG",
    2: "VBX_ERR_OUT_OF_MEMORY",
    3: "VBX_ERR_HASH_FULL",
    4: "VBX_ERR_TIMEOUT",
    5: "VBX_ERR_CUDA",
    6: "VBX_ERR_CAPACITY",
}
VBX_ERR_CAPACITY = 6

# vbx_mesh_block
MESH_BLOCK_DTYPE = np.dtype([("key", "<i4", (3,)), ("num_triangles", "<u4"), ("first_triangle", "<i8")])


class VbxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class vbx_map_options(ctypes.Structure):
    _fields_ = [
        ("weighting", ctypes.c_int),
        ("eps", ctypes.c_float),
        ("fixed_band", ctypes.c_float),
        ("w_max", ctypes.c_float),
        ("max_range", ctypes.c_float),
        ("grouped", ctypes.c_int),
        ("block_capacity", ctypes.c_int64),
        ("max_points", ctypes.c_int64),
        ("scratch_blocks", ctypes.c_int64),
        ("esdf_mode", ctypes.c_int),
        ("euclidean", ctypes.c_int),
    ]


class vbx_stats(ctypes.Structure):
    _fields_ = [
        (n, ctypes.c_int64)
        for n in (
            "points_in",
            "points_valid",
            "rays",
            "records",
            "updated",
            "new_blocks",
            "blocks",
            "esdf_in",
            "seeds",
            "raise_pops",
            "lower_pops",
            "raise_rounds",
            "lower_rounds",
            "launches",
            "esdf_block_visits",
            "esdf_local_iters",
            "esdf_classify_ns",
            "esdf_raise_ns",
            "esdf_lower_ns",
            "touched_blocks",
        )
    ]


class vbx_scan_in(ctypes.Structure):
    _fields_ = [("points_dev", ctypes.c_void_p), ("n", ctypes.c_int64), ("T_world_sensor", ctypes.c_float * 16)]


class vbx_query_io(ctypes.Structure):
    _fields_ = [
        ("q_dev", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("dist_dev", ctypes.c_void_p),
        ("grad_dev", ctypes.c_void_p),
        ("status_dev", ctypes.c_void_p),
    ]


STEP_INTEGRATE, STEP_ESDF, STEP_QUERY, STEP_GRAPH = 1, 2, 4, 8

# numpy records with the layouts of vbx_scan_in and vbx_query_io
SCAN_IN_DTYPE = np.dtype([("points_dev", "<u8"), ("n", "<i8"), ("T", "<f4", (16,))])
QUERY_IO_DTYPE = np.dtype([("q_dev", "<u8"), ("n", "<i8"), ("dist_dev", "<u8"), ("grad_dev", "<u8"), ("status_dev", "<u8")])
assert SCAN_IN_DTYPE.itemsize == ctypes.sizeof(vbx_scan_in) and QUERY_IO_DTYPE.itemsize == ctypes.sizeof(vbx_query_io)

_lib = None

# exported symbols and their (restype, argtypes)
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_SIGS = {
    "vbx_default_options": (ctypes.c_int, [ctypes.POINTER(vbx_map_options)]),
    "vbx_create_map": (
        ctypes.c_int,
        [ctypes.c_float, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.POINTER(vbx_map_options), ctypes.POINTER(_vp)],
    ),
    "vbx_destroy_map": (ctypes.c_int, [_vp]),
    "vbx_integrate_scan": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "vbx_integrate_scan_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "vbx_update_esdf": (ctypes.c_int, [_vp, _vp]),
    "vbx_query_distance_gradient": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "vbx_sync": (ctypes.c_int, [_vp, _vp]),
    "vbx_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(vbx_stats), _vp]),
    "vbx_num_blocks": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), _vp]),
    "vbx_export_blocks": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp]),
    "vbx_export_updated": (ctypes.c_int, [_vp, _vp, _i64, ctypes.POINTER(_i64), _vp]),
    "vbx_export_sites": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp]),
    "vbx_import_tsdf": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp]),
    "vbx_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
    "vbx_get_kernel_times": (
        ctypes.c_int,
        [_vp, ctypes.POINTER(ctypes.c_char_p), _vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp],
    ),
    "vbx_reset_kernel_times": (ctypes.c_int, [_vp]),
    "vbx_total_launches": (_i64, []),
    "vbx_map_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vbx_map_options), ctypes.POINTER(_i64)]),
    "vbx_map_device_bytes": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "vbx_reset_map": (ctypes.c_int, [_vp, _vp]),
    "vbx_extract_mesh": (
        ctypes.c_int,
        [_vp, ctypes.c_int, _vp, _vp, _i64, _vp, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64), _vp],
    ),
    "vbx_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i64, ctypes.POINTER(_vp)]),
    "vbx_batch_bind": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "vbx_batch_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "vbx_batch_autotune": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_char_p, ctypes.c_int]),
    "vbx_batch_sync": (ctypes.c_int, [_vp, _vp]),
    "vbx_batch_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
    "vbx_batch_kernel_times": (
        ctypes.c_int,
        [_vp, ctypes.POINTER(ctypes.c_char_p), _vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp],
    ),
    "vbx_batch_destroy": (ctypes.c_int, [_vp]),
    "vbx_last_error": (ctypes.c_char_p, []),
}


def exported_symbols():
    return list(_SIGS)


def load_library(path: str = LIB_PATH):
    """Loads libvbx.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st: int):
    if st != VBX_OK:
        raise VbxError(st, _lib.vbx_last_error().decode())


def _stream_ptr(stream) -> Optional[int]:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev_f32(t, cols: Optional[int] = None):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 tensor")
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"expected shape (N, {cols})")
    return t


def total_launches() -> int:
    return int(load_library().vbx_total_launches())


class Map:
    """A TSDF + ESDF map on the current CUDA device (see include/vbx.h)."""

    def __init__(
        self,
        voxel_size: float,
        voxels_per_block: int,
        truncation: float,
        max_esdf_dist: float,
        weighting: int = 0,
        eps: Optional[float] = None,
        fixed_band: Optional[float] = None,
        w_max: float = 1e4,
        max_range: float = math.inf,
        grouped: bool = True,
        block_capacity: int = 0,
        max_points: int = 0,
        scratch_blocks: int = 0,
        esdf_mode: int = 0,
        euclidean: bool = False,
    ):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("vbx.Map needs a CUDA device")
        self._lib = load_library()
        o = vbx_map_options()
        _check(self._lib.vbx_default_options(ctypes.byref(o)))
        o.weighting = int(weighting)
        o.eps = 0.0 if eps is None else float(eps)
        o.fixed_band = 0.0 if fixed_band is None else float(fixed_band)
        o.w_max = float(w_max)
        o.max_range = float(max_range) if math.isfinite(max_range) else 0.0
        o.grouped = 1 if grouped else 0
        o.block_capacity = int(block_capacity)
        o.max_points = int(max_points)
        o.scratch_blocks = int(scratch_blocks)
        o.esdf_mode = int(esdf_mode)
        o.euclidean = 1 if euclidean else 0
        h = ctypes.c_void_p()
        _check(self._lib.vbx_create_map(voxel_size, voxels_per_block, truncation, max_esdf_dist, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.B = int(voxels_per_block)
        self.voxel_size = float(voxel_size)

    @classmethod
    def from_scene_params(cls, params: Dict[str, float], **kw) -> "Map":
        args = dict(
            weighting=int(params.get("weighting", 0)),
            eps=params.get("eps"),
            fixed_band=params.get("fixed_band"),
            max_range=params.get("max_range", math.inf),
        )
        args.update(kw)
        return cls(params["voxel_size"], params["voxels_per_block"], params["truncation"], params["max_esdf_dist"], **args)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.vbx_destroy_map(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h.value

    # -------------------------------------------------------------------- hot path
    def integrate_scan(self, points, T_world_sensor, stream=None) -> None:
        p = _dev_f32(points, 3)
        T = np.ascontiguousarray(np.asarray(T_world_sensor, dtype=np.float32).reshape(16))
        _check(self._lib.vbx_integrate_scan(self._h, p.data_ptr(), p.shape[0], T.ctypes.data, _stream_ptr(stream)))

    def integrate_scan_noalloc(self, points, T_world_sensor, stream=None) -> None:
        """vbx_integrate_scan_noalloc: same result, scratch in a static device array (n <= 65536)."""
        p = _dev_f32(points, 3)
        T = np.ascontiguousarray(np.asarray(T_world_sensor, dtype=np.float32).reshape(16))
        _check(self._lib.vbx_integrate_scan_noalloc(self._h, p.data_ptr(), p.shape[0], T.ctypes.data, _stream_ptr(stream)))

    def update_esdf(self, stream=None) -> None:
        _check(self._lib.vbx_update_esdf(self._h, _stream_ptr(stream)))

    def query(self, q, out=None, stream=None):
        import torch

        q = _dev_f32(q, 3)
        n = q.shape[0]
        if out is None:
            dist = torch.empty(n, dtype=torch.float32, device=q.device)
            grad = torch.empty((n, 3), dtype=torch.float32, device=q.device)
            status = torch.empty(n, dtype=torch.uint8, device=q.device)
        else:
            dist, grad, status = out
        _check(
            self._lib.vbx_query_distance_gradient(
                self._h, q.data_ptr(), n, dist.data_ptr(), grad.data_ptr(), status.data_ptr(), _stream_ptr(stream)
            )
        )
        return dist, grad, status

    # ------------------------------------------------------------------ inspection
    def sync(self, stream=None) -> None:
        _check(self._lib.vbx_sync(self._h, _stream_ptr(stream)))

    def stats(self, stream=None) -> Dict[str, int]:
        s = vbx_stats()
        _check(self._lib.vbx_get_stats(self._h, ctypes.byref(s), _stream_ptr(stream)))
        return {f: int(getattr(s, f)) for f, _ in vbx_stats._fields_}

    def num_blocks(self, stream=None) -> int:
        n = ctypes.c_int64()
        _check(self._lib.vbx_num_blocks(self._h, ctypes.byref(n), _stream_ptr(stream)))
        return int(n.value)

    def export(self, sort: bool = True, stream=None) -> Dict[str, np.ndarray]:
        """Map contents on the host; blocks sorted by key (x, y, z) when sort=True."""
        nb = self.num_blocks(stream)
        B3 = self.B ** 3
        keys = np.zeros((max(nb, 1), 3), np.int32)
        tsdf = np.zeros((max(nb, 1), B3, 2), np.float32)
        d = np.zeros((max(nb, 1), B3), np.float32)
        parent = np.zeros((max(nb, 1), B3), np.uint8)
        flags = np.zeros((max(nb, 1), B3), np.uint8)
        _check(
            self._lib.vbx_export_blocks(
                self._h, keys.ctypes.data, tsdf.ctypes.data, d.ctypes.data, parent.ctypes.data, flags.ctypes.data, max(nb, 1), _stream_ptr(stream)
            )
        )
        keys, tsdf, d, parent, flags = keys[:nb], tsdf[:nb], d[:nb], parent[:nb], flags[:nb]
        if sort and nb:
            order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
            keys, tsdf, d, parent, flags = keys[order], tsdf[order], d[order], parent[order], flags[order]
        return dict(keys=keys, D=tsdf[..., 0], W=tsdf[..., 1], d=d, parent=parent, flags=flags)

    def export_sites(self, sort: bool = True, stream=None):
        """Euclidean maps: (offsets (nb, B^3, 3) int8 site - voxel, has_site (nb, B^3) bool), in
        the block order of export(sort)."""
        nb = self.num_blocks(stream)
        B3 = self.B ** 3
        off = np.zeros((max(nb, 1), B3, 3), np.int8)
        has = np.zeros((max(nb, 1), B3), np.uint8)
        keys = np.zeros((max(nb, 1), 3), np.int32)
        _check(self._lib.vbx_export_sites(self._h, off.ctypes.data, has.ctypes.data, max(nb, 1), _stream_ptr(stream)))
        _check(self._lib.vbx_export_blocks(self._h, keys.ctypes.data, None, None, None, None, max(nb, 1), _stream_ptr(stream)))
        off, has, keys = off[:nb], has[:nb].astype(bool), keys[:nb]
        if sort and nb:
            order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
            off, has = off[order], has[order]
        return off, has

    def last_updated(self, stream=None) -> np.ndarray:
        n = ctypes.c_int64()
        _check(self._lib.vbx_export_updated(self._h, None, 0, ctypes.byref(n), _stream_ptr(stream)))
        out = np.zeros((max(int(n.value), 1), 3), np.int32)
        _check(self._lib.vbx_export_updated(self._h, out.ctypes.data, out.shape[0], ctypes.byref(n), _stream_ptr(stream)))
        return out[: int(n.value)]

    def import_tsdf(self, vox: np.ndarray, D: np.ndarray, W: np.ndarray, stream=None) -> None:
        vox = np.ascontiguousarray(vox, dtype=np.int32).reshape(-1, 3)
        D = np.ascontiguousarray(D, dtype=np.float32).reshape(-1)
        W = np.ascontiguousarray(W, dtype=np.float32).reshape(-1)
        if not (len(vox) == len(D) == len(W)):
            raise ValueError("vox, D and W must have the same length")
        _check(self._lib.vbx_import_tsdf(self._h, vox.ctypes.data, D.ctypes.data, W.ctypes.data, len(D), _stream_ptr(stream)))

    # -------------------------------------------------------------------- profiling
    def set_profiling(self, enable: bool) -> None:
        _check(self._lib.vbx_set_profiling(self._h, 1 if enable else 0))

    def kernel_times(self, stream=None) -> Dict[str, Dict[str, float]]:
        cap = 32
        names = (ctypes.c_char_p * cap)()
        ms = np.zeros(cap, np.float64)
        cnt = np.zeros(cap, np.int64)
        n = ctypes.c_int()
        _check(self._lib.vbx_get_kernel_times(self._h, names, ms.ctypes.data, cnt.ctypes.data, cap, ctypes.byref(n), _stream_ptr(stream)))
        return {names[i].decode(): dict(ms=float(ms[i]), launches=int(cnt[i])) for i in range(min(n.value, cap))}

    def reset_kernel_times(self) -> None:
        _check(self._lib.vbx_reset_kernel_times(self._h))

    def device_bytes(self) -> int:
        n = ctypes.c_int64()
        _check(self._lib.vbx_map_device_bytes(self._h, ctypes.byref(n)))
        return int(n.value)

    def reset(self, stream=None) -> None:
        _check(self._lib.vbx_reset_map(self._h, _stream_ptr(stream)))

    # -------------------------------------------------------------------- mesh
    def extract_mesh(self, updated_only: bool = False, stream=None):
        """Triangles of the TSDF iso-surface (vbx_extract_mesh): every block, or only the blocks
        whose mesh may have changed since the last call. Returns (cells, verts, blocks): cells an
        int32 (n, 4) CUDA tensor (cell minimum-corner voxel, index in the cell), verts a float32
        (n, 3, 3) CUDA tensor, blocks a host array of MESH_BLOCK_DTYPE. cells and verts are views
        of buffers that the next call on this map overwrites."""
        import torch

        bufs = getattr(self, "_mesh_bufs", None)
        tri_cap = bufs[0].shape[0] if bufs is not None else 1 << 16
        blk_cap = bufs[2].shape[0] if bufs is not None else 1 << 10
        n_tri, n_blk = ctypes.c_int64(), ctypes.c_int64()
        for _ in range(2):
            if bufs is None or bufs[0].shape[0] < tri_cap or bufs[2].shape[0] < blk_cap:
                dev = torch.device("cuda", torch.cuda.current_device())
                bufs = (
                    torch.empty((tri_cap, 4), dtype=torch.int32, device=dev),
                    torch.empty((tri_cap, 3, 3), dtype=torch.float32, device=dev),
                    torch.empty((blk_cap, 3), dtype=torch.int64, device=dev),
                )
                self._mesh_bufs = bufs
            st = self._lib.vbx_extract_mesh(
                self._h, 1 if updated_only else 0, bufs[0].data_ptr(), bufs[1].data_ptr(), bufs[0].shape[0],
                bufs[2].data_ptr(), bufs[2].shape[0], ctypes.byref(n_tri), ctypes.byref(n_blk), _stream_ptr(stream),
            )
            if st != VBX_ERR_CAPACITY:
                break
            tri_cap = max(tri_cap, int(n_tri.value + n_tri.value // 4 + 1024))
            blk_cap = max(blk_cap, int(n_blk.value + n_blk.value // 4 + 64))
        _check(st)
        n, m = int(n_tri.value), int(n_blk.value)
        blocks = np.frombuffer(bufs[2][:m].cpu().numpy().tobytes(), dtype=MESH_BLOCK_DTYPE) if m else np.zeros(0, MESH_BLOCK_DTYPE)
        return bufs[0][:n], bufs[1][:n], blocks


def map_bytes(voxels_per_block: int, block_capacity: int = 0, max_points: int = 0, scratch_blocks: int = 0) -> int:
    """Device bytes of a map with these sizes (vbx_map_bytes)."""
    lib = load_library()
    o = vbx_map_options()
    _check(lib.vbx_default_options(ctypes.byref(o)))
    o.block_capacity = int(block_capacity)
    o.max_points = int(max_points)
    o.scratch_blocks = int(scratch_blocks)
    n = ctypes.c_int64()
    _check(lib.vbx_map_bytes(int(voxels_per_block), ctypes.byref(o), ctypes.byref(n)))
    return int(n.value)


class MapBatch:
    """A fixed-slot batch of maps advanced by the same launches (vbx_batch_* in vbx.h)."""

    def __init__(self, maps, max_queries: int = 0):
        self._lib = load_library()
        self.maps = list(maps)
        arr = (ctypes.c_void_p * len(self.maps))(*[m.handle for m in self.maps])
        h = ctypes.c_void_p()
        _check(self._lib.vbx_batch_create(arr, len(self.maps), int(max_queries), ctypes.byref(h)))
        self._h = h
        self.count = len(self.maps)
        # descriptors as numpy records with the C layouts of vbx_scan_in / vbx_query_io
        self._scans = np.zeros(self.count, SCAN_IN_DTYPE)
        self._queries = np.zeros(self.count, QUERY_IO_DTYPE)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.vbx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bind(self, slot: int, m: "Map") -> None:
        _check(self._lib.vbx_batch_bind(self._h, int(slot), m.handle))
        self.maps[slot] = m

    def _fill(self, points, poses, queries, slots=None):
        """Descriptors of one step. Without `slots`, points / poses / queries have one entry per
        slot (None: nothing for that slot); with `slots`, they hold entries for those slots only
        and every other slot is idle."""
        sc, qd = self._scans, self._queries
        sc["points_dev"] = 0
        sc["n"] = 0
        qd[:] = 0
        idx = range(self.count) if slots is None else slots
        for j, i in enumerate(idx):
            k = i if slots is None else j
            p = points[k] if points is not None else None
            if p is not None and p.shape[0] > 0:
                _dev_f32(p, 3)
                sc["points_dev"][i] = p.data_ptr()
                sc["n"][i] = p.shape[0]
            if poses is not None and poses[k] is not None:
                sc["T"][i] = np.asarray(poses[k], dtype=np.float32).reshape(16)
            if queries is not None and queries[k] is not None:
                qq, dist, grad, status = queries[k]
                _dev_f32(qq, 3)
                qd[i] = (qq.data_ptr(), qq.shape[0], dist.data_ptr(), grad.data_ptr(), status.data_ptr())

    def step(self, points=None, poses=None, queries=None, flags: int = STEP_INTEGRATE | STEP_ESDF, stream=None, slots=None) -> None:
        """points[i]: (N,3) device tensor or None; poses[i]: 4x4; queries[i]: (q, dist, grad, status)
        or None; one entry per slot, or per listed slot when `slots` is given."""
        self._fill(points, poses, queries, slots)
        _check(self._lib.vbx_batch_step(self._h, self._scans.ctypes.data, self._queries.ctypes.data, int(flags), _stream_ptr(stream)))

    def autotune(self, points=None, poses=None, queries=None, flags: int = STEP_INTEGRATE | STEP_ESDF, stream=None) -> str:
        self._fill(points, poses, queries)
        buf = ctypes.create_string_buffer(256)
        _check(
            self._lib.vbx_batch_autotune(
                self._h, self._scans.ctypes.data, self._queries.ctypes.data, int(flags), _stream_ptr(stream), buf, 256
            )
        )
        return buf.value.decode()

    def sync(self, stream=None) -> None:
        _check(self._lib.vbx_batch_sync(self._h, _stream_ptr(stream)))

    def set_profiling(self, enable: bool) -> None:
        _check(self._lib.vbx_batch_set_profiling(self._h, 1 if enable else 0))

    def kernel_times(self, stream=None):
        cap = 32
        names = (ctypes.c_char_p * cap)()
        ms = np.zeros(cap, np.float64)
        cnt = np.zeros(cap, np.int64)
        n = ctypes.c_int()
        _check(self._lib.vbx_batch_kernel_times(self._h, names, ms.ctypes.data, cnt.ctypes.data, cap, ctypes.byref(n), _stream_ptr(stream)))
        return {names[i].decode(): dict(ms=float(ms[i]), launches=int(cnt[i])) for i in range(min(n.value, cap))}

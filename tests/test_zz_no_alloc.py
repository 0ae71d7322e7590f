"""vbx_integrate_scan_noalloc against vbx_integrate_scan, through the C ABI.

The allocation-free entry point serves callers that must not allocate device memory while
they run: a robot's real-time loop, where cudaMalloc/cudaFree synchronise the device and can
miss the loop's deadline, or a process whose device-memory budget is fixed at start-up. Its
per-scan scratch lives in a static device array of the library instead of map-owned buffers,
so it must give the same map, bit for bit, as the regular entry point, also for a scan larger
than the map's own point scratch (which the regular entry point grows). This file is collected
last so that a run that stops at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_1611_03631_gb300 import scenes
from parity_util import check_parents, sort_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NOALLOC_MAX_POINTS = 65536


@pytest.fixture(scope="module")
def vbx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03631_gb300 import vbx as v

    v.load_library()
    return v


def _same_maps(a, b, tag):
    ga, gb = a.stats(), b.stats()
    for k in ("points_valid", "rays", "records", "updated", "new_blocks", "blocks", "touched_blocks"):
        assert ga[k] == gb[k], (tag, k, ga[k], gb[k])
    assert np.array_equal(sort_rows(a.last_updated()), sort_rows(b.last_updated())), tag
    ea, eb = a.export(), b.export()
    for k in ("keys", "D", "W", "d", "flags"):
        assert np.array_equal(ea[k], eb[k]), (tag, k)
    # parent directions may differ where two neighbours offer the same value (the ESDF's work
    # order decides); each must still reproduce its voxel's value exactly
    v = np.float32(a.voxel_size)
    L = (0.0, v, np.float32(v * np.float32(1.41421356237309515)), np.float32(v * np.float32(1.73205080756887719)))
    for ex in (ea, eb):
        bad, _ = check_parents(ex, a.B, L)
        assert bad == 0, tag


def test_noalloc_entry_point_matches_regular_one_on_two_calls(vbx):
    s = scenes.room(frames=2, width=160, height=120, fx=131.25, fy=131.25)
    regular = vbx.Map.from_scene_params(s.params)
    noalloc = vbx.Map.from_scene_params(s.params)
    for i in range(2):  # two calls in a row: the shared static scratch is reused
        pts = torch.from_numpy(s.points[i]).cuda()
        regular.integrate_scan(pts, s.poses[i])
        noalloc.integrate_scan_noalloc(pts, s.poses[i])
        _same_maps(regular, noalloc, f"room scan {i}")
    regular.update_esdf()
    noalloc.update_esdf()
    _same_maps(regular, noalloc, "room ESDF")


def test_noalloc_scan_at_the_limit_on_a_map_with_small_point_scratch(vbx):
    """Two scans of exactly 65536 points (a 32 x 2048 LiDAR) on maps created for 1024 points:
    the regular entry point grows the map's point scratch, the allocation-free one leaves the
    map's device memory unchanged, and both give the same map."""
    s = scenes.lidar_terrain(scans=2, beams=32, columns=2048, n_buildings=80, n_trees=120, extent=120.0, path_length=30.0)
    assert all(p.shape[0] == NOALLOC_MAX_POINTS for p in s.points)
    regular = vbx.Map.from_scene_params(s.params, max_points=1024, block_capacity=1 << 16)
    noalloc = vbx.Map.from_scene_params(s.params, max_points=1024, block_capacity=1 << 16)
    bytes_regular, bytes_noalloc = regular.device_bytes(), noalloc.device_bytes()
    assert bytes_regular == bytes_noalloc
    for i in range(2):
        pts = torch.from_numpy(s.points[i]).cuda()
        regular.integrate_scan(pts, s.poses[i])
        noalloc.integrate_scan_noalloc(pts, s.poses[i])
        _same_maps(regular, noalloc, f"lidar scan {i}")
        assert noalloc.device_bytes() == bytes_noalloc
        assert regular.device_bytes() > bytes_regular
    regular.update_esdf()
    noalloc.update_esdf()
    _same_maps(regular, noalloc, "lidar ESDF")


def test_noalloc_entry_point_rejects_scans_above_its_limit(vbx):
    m = vbx.Map(0.1, 8, 0.3, 2.0)
    pts = torch.zeros((NOALLOC_MAX_POINTS + 1, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(vbx.VbxError) as ei:
        m.integrate_scan_noalloc(pts, np.eye(4, dtype=np.float32))
    assert ei.value.status == 1 and str(NOALLOC_MAX_POINTS) in str(ei.value)

"""Large single-map ESDF updates run on a kernel compiled for the map's block edge (work-queue
schedule only); the batch path runs the general kernel. Both must reach the same maps, bit for
bit, for every block edge, on LiDAR updates large enough to select the specialised kernel."""
import numpy as np
import pytest

from paper_1611_03631_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LARGE_UPDATE = 1 << 19  # dirty voxels from which the next single-map update takes the large shape


@pytest.fixture(scope="module")
def vbx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03631_gb300 import vbx as v

    v.load_library()
    return v


@pytest.fixture(scope="module")
def lidar():
    return scenes.lidar_terrain(scans=40, generate=3, workers=8)


def _same(a, b):
    ea, eb = a.export(), b.export()
    assert np.array_equal(ea["keys"], eb["keys"])
    assert np.array_equal(ea["flags"], eb["flags"])
    for k in ("D", "W", "d"):
        assert np.array_equal(ea[k], eb[k]), k


@pytest.mark.parametrize("B,capacity,scratch", [(4, 1 << 19, 1 << 18), (8, 1 << 17, 1 << 16), (16, 1 << 15, 1 << 13)])
def test_large_update_kernel_matches_general_kernel(vbx, lidar, B, capacity, scratch):
    params = dict(lidar.params, voxels_per_block=B)
    kw = dict(block_capacity=capacity, scratch_blocks=scratch, max_points=lidar.points[0].shape[0])
    alone = vbx.Map.from_scene_params(params, **kw)
    mixed = vbx.Map.from_scene_params(params, **kw)
    # a second, small map makes the batch launch the general kernel (two maps at work)
    other_scene = scenes.plane_sphere(frames=3, width=32, height=24, fx=25.0, fy=25.0, cx=16.0, cy=12.0, seed=5)
    other = vbx.Map.from_scene_params(other_scene.params)
    batch = vbx.MapBatch([mixed, other])
    large_updates = 0
    for f in range(3):
        pts = torch.from_numpy(lidar.points[f]).cuda()
        prev_in = alone.stats()["esdf_in"] if f else 0
        alone.integrate_scan(pts, lidar.poses[f])
        alone.update_esdf()
        large_updates += prev_in >= LARGE_UPDATE
        batch.step([pts, torch.from_numpy(other_scene.points[f]).cuda()], [lidar.poses[f], other_scene.poses[f]])
        batch.sync()
        _same(alone, mixed)
        assert alone.stats()["esdf_in"] == mixed.stats()["esdf_in"]
    assert large_updates >= 2  # scans 1 and 2 followed an update of at least 2^19 dirty voxels
    for m in (alone, mixed, other):
        m.close()

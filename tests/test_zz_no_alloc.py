"""vbx_integrate_scan_noalloc against vbx_integrate_scan, through the C ABI.

The allocation-free entry point serves callers that must not allocate device memory while
they run (a robot's real-time loop, where cudaMalloc/cudaFree synchronise the device and can
miss the loop's deadline, or a process with a device-memory budget fixed at start-up). It must
give the same map as the regular entry point. This file is collected last so that a run that
stops at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_1611_03631_gb300 import scenes
from parity_util import TOL_D, TOL_W_REL, compare_tsdf, sort_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vbx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03631_gb300 import vbx as v

    v.load_library()
    return v


def test_noalloc_entry_point_matches_regular_one_on_two_calls(vbx):
    s = scenes.room(frames=2, width=160, height=120, fx=131.25, fy=131.25)
    regular = vbx.Map.from_scene_params(s.params)
    noalloc = vbx.Map.from_scene_params(s.params)
    for i in range(2):  # two calls in a row: the shared static scratch is reused
        pts = torch.from_numpy(s.points[i]).cuda()
        regular.integrate_scan(pts, s.poses[i])
        noalloc.integrate_scan_noalloc(pts, s.poses[i])
        ga, gb = regular.stats(), noalloc.stats()
        for k in ("points_valid", "rays", "records", "updated", "new_blocks", "blocks"):
            assert ga[k] == gb[k], (i, k)
        assert np.array_equal(sort_rows(regular.last_updated()), sort_rows(noalloc.last_updated()))
        r = compare_tsdf(noalloc.export(), regular.export(), s.params["voxels_per_block"])
        assert r["max_dD"] <= TOL_D and r["max_rel_dW"] <= TOL_W_REL, (i, r)
    regular.update_esdf()
    noalloc.update_esdf()
    ea, eb = regular.export(), noalloc.export()
    obs = (ea["flags"] & 1) > 0
    assert np.array_equal(ea["flags"], eb["flags"])
    assert np.max(np.abs(ea["d"][obs] - eb["d"][obs])) <= 1e-4


def test_noalloc_entry_point_rejects_scans_above_its_limit(vbx):
    m = vbx.Map(0.1, 8, 0.3, 2.0)
    pts = torch.zeros((65537, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(vbx.VbxError) as ei:
        m.integrate_scan_noalloc(pts, np.eye(4, dtype=np.float32))
    assert ei.value.status == 1 and "65536" in str(ei.value)

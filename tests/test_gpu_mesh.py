"""Parity of the CUDA mesh extraction (vbx_extract_mesh) with the oracle's marching cells, and
the properties of its incremental form.

* Same seeded synthetic TSDF imported into both: identical triangles, bit for bit (cell key,
  index in cell, the 9 vertex coordinates), for block sizes 4, 8 and 16.
* Incremental extraction on maps fused from scans (the full-size room workload): after every
  scan, the per-block meshes kept from the incremental calls equal a full extraction; the
  surface has no edge traversed twice in one direction and every vertex lies on a lattice edge.
* Capacity errors report the sizes needed and keep the stale marks; reset clears them.
"""
import ctypes
from collections import Counter

import numpy as np
import pytest
import torch

import oracle
from paper_1611_03631_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vbx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03631_gb300 import vbx as v

    v.load_library()
    return v


def _sorted(cells, verts):
    cells = np.asarray(cells)
    verts = np.asarray(verts).reshape(-1, 9)
    order = np.lexsort(cells.T[::-1])
    return cells[order], verts[order]


def _gpu_mesh(m, updated_only=False):
    c, v, blocks = m.extract_mesh(updated_only=updated_only)
    torch.cuda.synchronize()
    return c.cpu().numpy(), v.cpu().numpy(), blocks


@pytest.mark.parametrize("B", [8, 16, 4])
def test_mesh_matches_oracle_on_imported_tsdf(vbx, B):
    v, delta = 0.1, 0.4
    vox, D, W = scenes.synthetic_tsdf(voxel_size=v, voxels_per_block=B, truncation=delta, seed=7 + B)
    g = vbx.Map(v, B, delta, 2.0, block_capacity=1 << 14)
    g.import_tsdf(vox, D, W)
    o = oracle.OracleMap(v, B, delta, 2.0)
    o.set_tsdf(vox, D.astype(np.float64), W.astype(np.float64))
    gc, gv, blocks = _gpu_mesh(g)
    oc, ov = o.extract_mesh()
    assert oc.shape[0] > 10000
    gc, gv = _sorted(gc, gv)
    assert np.array_equal(gc, oc), "cell keys or per-cell triangle counts differ"
    assert np.array_equal(gv.view(np.uint32), ov.reshape(-1, 9).view(np.uint32)), "vertex bits differ"
    # block records: every allocated block listed once, counts and ranges consistent
    assert blocks.shape[0] == g.num_blocks()
    assert len({tuple(k) for k in blocks["key"]}) == blocks.shape[0]
    assert int(blocks["num_triangles"].sum()) == gc.shape[0]
    g.close()


def test_mesh_block_ranges_hold_their_cells(vbx):
    B = 8
    vox, D, W = scenes.synthetic_tsdf(voxels_per_block=B, seed=3)
    g = vbx.Map(0.1, B, 0.4, 2.0, block_capacity=1 << 14)
    g.import_tsdf(vox, D, W)
    cells, _, blocks = _gpu_mesh(g)
    for b in blocks:
        f, n = int(b["first_triangle"]), int(b["num_triangles"])
        assert (np.floor_divide(cells[f : f + n, :3], B) == np.asarray(b["key"])[None]).all()
    ranges = sorted((int(b["first_triangle"]), int(b["num_triangles"])) for b in blocks)
    pos = 0
    for f, n in ranges:
        assert f == pos
        pos += n
    assert pos == cells.shape[0]
    g.close()


def _surface_properties(cells, verts, v):
    """The 2nd and 3rd vertex of every triangle lie on an edge of the voxel lattice (the 1st is
    a loop centroid in fans): two of their coordinates are voxel centres, ((float)i + 1/2) v in
    float32, and the third lies within one voxel of the cell's corner. Vertices are identified
    by their exact bits; distinct lattice edges can only meet at a lattice corner (a voxel with
    D exactly 0, or t rounding to 0 or 1), so triangles with a vertex exactly on a corner are
    left out of the edge counts: among the rest no directed edge appears twice (consistent
    orientation, no fold) and no undirected edge in more than two triangles."""
    v32 = np.float32(v)
    t = verts.reshape(-1, 3, 3).astype(np.float32)
    i = np.round(t.astype(np.float64) / float(v32) - 0.5)
    centre = ((i.astype(np.float32) + np.float32(0.5)) * v32).astype(np.float32)
    ncentre = (t == centre).sum(axis=-1)
    assert (ncentre[:, 1:] >= 2).all()
    lo = (cells[:, None, :3].astype(np.float64) + 0.5) * float(v32)
    assert ((t[:, 1:] >= lo - 1e-6) & (t[:, 1:] <= lo + float(v32) + 1e-6)).all()
    keep = (ncentre < 3).all(axis=1)
    assert keep.mean() > 0.5
    key = t[keep].view(np.uint32)
    directed = Counter()
    undirected = Counter()
    for tri in key:
        for k in range(3):
            a, b = tuple(tri[k]), tuple(tri[(k + 1) % 3])
            directed[(a, b)] += 1
            undirected[frozenset((a, b))] += 1
    assert max(directed.values()) == 1
    assert max(undirected.values()) <= 2


def test_incremental_mesh_equals_full_on_room_scans(vbx):
    """Room workload at full size (640x480 frames, v = 0.05 m, 16^3 blocks): after each scan the
    blocks returned by the incremental call replace the kept meshes, and the kept meshes equal
    a full extraction of the same map."""
    s = scenes.room()
    p = s.params
    g = vbx.Map.from_scene_params(p)
    kept = {}
    for i in range(8):
        g.integrate_scan(torch.from_numpy(s.points[i]).cuda(), s.poses[i])
        cells, verts, blocks = _gpu_mesh(g, updated_only=True)
        assert blocks.shape[0] > 0
        for b in blocks:
            f, n = int(b["first_triangle"]), int(b["num_triangles"])
            kept[tuple(int(x) for x in b["key"])] = (cells[f : f + n].copy(), verts[f : f + n].copy())
        fc, fv, fb = _gpu_mesh(g, updated_only=False)
        kc = np.concatenate([c for c, _ in kept.values()]) if kept else np.zeros((0, 4), np.int32)
        kv = np.concatenate([x for _, x in kept.values()]) if kept else np.zeros((0, 3, 3), np.float32)
        kc, kv = _sorted(kc, kv)
        fc, fv = _sorted(fc, fv)
        assert np.array_equal(kc, fc), f"scan {i}: kept meshes differ from the full mesh"
        assert np.array_equal(kv.view(np.uint32), fv.view(np.uint32))
        # nothing is stale right after a full extraction
        _, _, nb = _gpu_mesh(g, updated_only=True)
        assert nb.shape[0] == 0
    _surface_properties(fc, fv, float(p["voxel_size"]))
    assert fc.shape[0] > 50000
    g.close()


def test_mesh_capacity_error_keeps_marks_and_reset_clears(vbx):
    vox, D, W = scenes.synthetic_tsdf(seed=5)
    g = vbx.Map(0.1, 8, 0.4, 2.0, block_capacity=1 << 14)
    assert _gpu_mesh(g)[0].shape[0] == 0  # empty map
    g.import_tsdf(vox, D, W)
    lib = vbx.load_library()
    cells = torch.empty((16, 4), dtype=torch.int32, device="cuda")
    verts = torch.empty((16, 3, 3), dtype=torch.float32, device="cuda")
    blk = torch.empty((4, 3), dtype=torch.int64, device="cuda")
    nt, nb = ctypes.c_int64(), ctypes.c_int64()
    st = lib.vbx_extract_mesh(
        g.handle, 1, cells.data_ptr(), verts.data_ptr(), 16, blk.data_ptr(), 4, ctypes.byref(nt), ctypes.byref(nb),
        torch.cuda.current_stream().cuda_stream,
    )
    assert st == vbx.VBX_ERR_CAPACITY
    assert nt.value > 16 and nb.value == g.num_blocks()
    # marks kept: the incremental call lists every block again, with the same triangles as a
    # full extraction
    c1, v1, b1 = _gpu_mesh(g, updated_only=True)
    assert b1.shape[0] == nb.value and c1.shape[0] == nt.value
    c2, v2, _ = _gpu_mesh(g, updated_only=False)
    a, b = _sorted(c1, v1), _sorted(c2, v2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    # an import marks its blocks and their lower neighbours stale
    one = vox[:1]
    g.import_tsdf(one, D[:1], W[:1])
    _, _, b3 = _gpu_mesh(g, updated_only=True)
    keys = {tuple(int(x) for x in k) for k in b3["key"]}
    kb = tuple(int(x) for x in np.floor_divide(one[0], 8))
    assert kb in keys and len(keys) <= 8
    assert all(all(kb[a] - k[a] in (0, 1) for a in range(3)) for k in keys)
    g.import_tsdf(vox, D, W)
    g.reset()
    _, _, b4 = _gpu_mesh(g, updated_only=True)
    assert b4.shape[0] == 0
    g.close()

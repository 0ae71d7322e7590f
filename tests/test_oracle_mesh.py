"""Pins of the oracle's TSDF mesh (reading R12: marching cells with inside corners cut off on
ambiguous faces, loops fanned around their centroid): closed forms for a plane and a sphere,
and watertight, consistently oriented surfaces on random fields full of ambiguous faces."""
from collections import Counter

import numpy as np
import pytest

import oracle


def _grid_map(D, v=0.1, B=8):
    G = D.shape
    idx = np.stack(np.meshgrid(*[np.arange(g) for g in G], indexing="ij"), -1).reshape(-1, 3)
    m = oracle.OracleMap(v, B, 0.3, 2.0)
    m.set_tsdf(idx, D.reshape(-1), np.ones(idx.shape[0]))
    return m


def _edges(verts, tol):
    key = lambda p: tuple(np.round(p / tol).astype(np.int64))
    directed, undirected, vs = Counter(), Counter(), set()
    for t in verts:
        ks = [key(p) for p in t]
        vs.update(ks)
        for i in range(3):
            a, b = ks[i], ks[(i + 1) % 3]
            directed[(a, b)] += 1
            undirected[frozenset((a, b))] += 1
    return directed, undirected, vs


def test_plane_gives_a_flat_grid_at_the_zero_crossing():
    v, G, z0 = 0.1, (6, 5, 8), 0.437
    k = np.arange(G[2])
    D = np.broadcast_to(((k + 0.5) * v - z0).astype(np.float32), G).astype(np.float64)
    cells, verts = _grid_map(D, v).extract_mesh()
    # one crossing cell layer of (G0-1) x (G1-1) cells, a quad each: four triangles around
    # its centre
    assert len(cells) == 4 * (G[0] - 1) * (G[1] - 1)
    assert np.max(np.abs(verts[..., 2] - z0)) < 1e-6
    n = np.cross(verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0])
    assert (n[:, 2] > 0).all() and np.allclose(n[:, :2], 0, atol=1e-9)  # towards positive D


def test_sphere_is_closed_oriented_outwards_and_on_the_surface():
    v, G, c, r = 0.1, 24, np.array([1.2, 1.2, 1.2]), 0.8
    idx = np.stack(np.meshgrid(*[np.arange(G)] * 3, indexing="ij"), -1)
    D = np.linalg.norm((idx + 0.5) * v - c, axis=-1) - r
    cells, verts = _grid_map(D, v).extract_mesh()
    directed, undirected, vs = _edges(verts, 1e-4 * v)
    assert set(undirected.values()) == {2}  # watertight
    assert max(directed.values()) == 1  # consistently oriented
    assert len(vs) - len(undirected) + len(verts) == 2  # Euler characteristic of a sphere
    rad = np.linalg.norm(verts.reshape(-1, 3) - c, axis=1) - r
    assert np.max(np.abs(rad)) < 0.05 * v  # linear interpolation of a curved field
    n = np.cross(verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0])
    assert (np.einsum("ij,ij->i", n, verts.mean(1) - c) > 0).all()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_fields_give_watertight_oriented_surfaces(seed):
    """Random corner values inside a positive border: closed surfaces with many ambiguous
    faces, which neighbouring cells must cut the same way."""
    rng = np.random.default_rng(seed)
    D = np.ones((12, 12, 12))
    D[1:-1, 1:-1, 1:-1] = rng.uniform(-1.0, 1.0, (10, 10, 10))
    cells, verts = _grid_map(D, 0.1).extract_mesh()
    assert len(cells) > 500
    directed, undirected, _ = _edges(verts, 1e-5)
    assert set(undirected.values()) == {2}
    assert max(directed.values()) == 1
    # no triangle is degenerate
    n = np.cross(verts[:, 1] - verts[:, 0], verts[:, 2] - verts[:, 0])
    assert (np.linalg.norm(n, axis=1) > 0).all()
    # normals towards positive D: the closed surfaces enclose the negative regions, so the
    # signed volume they bound (divergence theorem) is positive
    vol = np.einsum("ij,ij->i", verts[:, 0].astype(np.float64), np.cross(verts[:, 1], verts[:, 2]).astype(np.float64)).sum() / 6
    assert vol > 0


def _one_cell(Dc, v=0.1):
    """A map holding one cell (corner c = x + 2y + 4z at voxel (x, y, z)), all observed."""
    D = np.zeros((2, 2, 2))
    for c in range(8):
        D[c & 1, (c >> 1) & 1, c >> 2] = Dc[c]
    return _grid_map(D, v).extract_mesh()


def test_single_inside_corner_is_one_triangle_cut_at_the_interpolated_points():
    """Worked example: corner 0 at D = -0.25, the others at +0.75. Each of its three edges
    crosses a quarter of the way from corner 0 (t = -0.25 / (-0.25 - 0.75)), so the triangle's
    vertices are the cell origin plus v/4 along x, y and z; its normal points away from the
    inside corner, towards positive D."""
    v = 0.1
    cells, verts = _one_cell([-0.25] + [0.75] * 7, v)
    assert cells.shape[0] == 1 and tuple(cells[0]) == (0, 0, 0, 0)
    o = np.float32(0.5) * np.float32(v)
    q = o + np.float32(0.25) * np.float32(v)
    expect = {(q, o, o), (o, q, o), (o, o, q)}
    got = {tuple(np.round(p, 7)) for p in verts[0].astype(np.float64)}
    assert got == {tuple(np.round(np.array(e, np.float64), 7)) for e in expect}
    n = np.cross(verts[0, 1] - verts[0, 0], verts[0, 2] - verts[0, 0])
    assert n @ np.ones(3) > 0


def test_complement_gives_the_same_triangle_reversed():
    a_cells, a = _one_cell([-0.25] + [0.75] * 7)
    b_cells, b = _one_cell([0.25] + [-0.75] * 7)
    assert a.shape[0] == b.shape[0] == 1
    assert {tuple(p) for p in a[0]} == {tuple(p) for p in b[0]}
    na = np.cross(a[0, 1] - a[0, 0], a[0, 2] - a[0, 0])
    nb = np.cross(b[0, 1] - b[0, 0], b[0, 2] - b[0, 0])
    assert na @ nb < 0


def test_diagonal_inside_corners_on_a_face_are_cut_off_separately():
    """Corners 0 and 3 inside (diagonal on the face z = 0), the rest outside: the ambiguous face
    is resolved by cutting each inside corner off alone, so the cell holds two separate
    triangles (six distinct vertices) rather than one band."""
    Dc = [0.5] * 8
    Dc[0] = Dc[3] = -0.5
    cells, verts = _one_cell(Dc)
    assert cells.shape[0] == 2
    assert len({tuple(p) for t in verts for p in t}) == 6


def test_a_zero_corner_counts_as_outside():
    """fl32(D) = 0 (either sign) is outside: with corner 0 at -0.5 and corner 1 at exactly 0,
    the x edge crosses at t = 1, i.e. exactly at corner 1."""
    v = 0.1
    for z in (0.0, -0.0):
        Dc = [-0.5, z, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5]
        cells, verts = _one_cell(Dc, v)
        assert cells.shape[0] == 1
        c1 = np.array([1.5, 0.5, 0.5], np.float32) * np.float32(v)
        assert any(np.array_equal(p, c1) for p in verts[0])

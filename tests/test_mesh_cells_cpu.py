"""Host check of the CUDA library's per-cell mesh code (mesh_cells.cuh, compiled with nvcc as
host code; no GPU needed) against the oracle's mesh: every one of the 256 inside/outside
patterns, with random corner values including +0 and -0, gives bit-identical triangles in the
same order within the cell."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cells(seed, draws):
    """Corner values (n, 8) float32, corner c = x + 2 y + 4 z; every pattern `draws` times."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(256):
        inside = np.array([(p >> c) & 1 for c in range(8)], bool)
        for _ in range(draws):
            mag = rng.uniform(0.0, 1.0, 8).astype(np.float32)
            D = np.where(inside, -np.maximum(mag, np.float32(1e-6)), mag).astype(np.float32)
            zero = (~inside) & (rng.random(8) < 0.15)
            D[zero] = np.where(rng.random(8) < 0.5, np.float32(0.0), np.float32(-0.0))[zero]
            out.append(D)
    return np.stack(out)


def _check_exe(d):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = os.path.join(d, "mesh_cells_check")
    src = os.path.join(ROOT, "tests", "mesh_cells_check.cu")
    inc = os.path.join(ROOT, "paper_1611_03631_gb300", "csrc")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off", "-I", inc, src, "-o", exe], check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("v", [0.1, 0.05])
def test_cell_code_matches_oracle_on_every_pattern(v):
    Dc = _cells(seed=11, draws=4)
    n = Dc.shape[0]
    # cells 3 voxels apart (unobserved voxels between them), some at negative coordinates
    k = np.arange(n)
    g = np.stack([3 * (k % 32), 3 * ((k // 32) % 32), 3 * (k // 1024)], 1) - np.array([40, 13, 2])
    v32 = np.float32(v)
    with tempfile.TemporaryDirectory() as d:
        exe = _check_exe(d)
        lines = [str(n)]
        vb = "%08x" % v32.view(np.uint32)
        for i in range(n):
            lines.append(" ".join([str(int(x)) for x in g[i]] + [vb] + ["%08x" % u for u in Dc[i].view(np.uint32)]))
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr
    rows = [ln.split() for ln in r.stdout.splitlines()]
    got_cell = np.array([[*g[int(x[0])], int(x[1])] for x in rows], np.int32).reshape(-1, 4)
    got_v = np.array([[int(h, 16) for h in x[2:]] for x in rows], np.uint32).reshape(-1, 9)

    # the oracle: one map holding all cells, every cell's 8 voxels observed with weight 1
    corner = np.array([[c & 1, (c >> 1) & 1, c >> 2] for c in range(8)])
    vox = (g[:, None, :] + corner[None]).reshape(-1, 3)
    m = oracle.OracleMap(float(v32), 8, 0.3, 2.0)
    m.set_tsdf(vox, Dc.reshape(-1).astype(np.float64), np.ones(vox.shape[0]))
    cells, verts = m.extract_mesh()
    assert cells.shape[0] > 0
    # the oracle meshes exactly the n cells (each 3 voxels from the next)
    assert len({tuple(c) for c in cells[:, :3]}) == len({tuple(c) for c in got_cell[:, :3]})

    order = np.lexsort(got_cell.T[::-1])
    got_cell, got_v = got_cell[order], got_v[order]
    assert np.array_equal(got_cell, cells), "cell keys or per-cell triangle counts differ"
    assert np.array_equal(got_v, verts.reshape(-1, 9).view(np.uint32)), "vertex bits differ"

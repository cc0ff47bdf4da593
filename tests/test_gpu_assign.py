"""Alg. 1 stage II on the GPU against the oracle: the network of every
occupied voxel is bit-identical (integer decisions), the boxes are the
networks' voxel bounding boxes, and a render with the assigned fields
matches the oracle like any other partition."""
import numpy as np
import pytest

import fixtures as F
import oracle as O
import oracle.parity as P
from gpu_parity import assert_render, records

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def roam():
    import paper_2208_02705_gb300 as roam
    from paper_2208_02705_gb300 import build
    build.build()
    return roam


def _occ_linear(scene):
    z, y, x = np.nonzero(scene.occ)
    gx, gy, _ = scene.dims
    return (z.astype(np.int64) * gy + y) * gx + x


@pytest.mark.parametrize("which,n", [("room32", 8), ("room32", 37), ("floor256", 512)])
def test_assign_fields_matches_oracle(roam, which, n):
    wl = F.room32() if which == "room32" else F.floor256(views="equirect")
    r = roam.Roam(0)
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    labels, boxes = r.assign_fields(n)
    torch.cuda.synchronize()
    got = labels.cpu().numpy().view(np.uint16).astype(np.int32)
    lin = _occ_linear(wl.scene)
    ref = O.assign_fields(wl.scene.dims, lin, n)
    assert np.array_equal(got, ref)
    gx, gy, _ = wl.scene.dims
    xyz = np.stack([lin % gx, (lin // gx) % gy, lin // (gx * gy)], axis=1)
    b = boxes.cpu().numpy()
    for k in range(n):
        sel = xyz[ref == k]
        assert np.array_equal(b[k, :3], sel.min(axis=0)) and np.array_equal(b[k, 3:], sel.max(axis=0) + 1)
    r.close()


def test_render_with_assigned_fields(roam, room32, room32_grid):
    r = roam.Roam(0)
    r.load_grid(room32.scene.bits, room32.scene.dims, room32.scene.origin, room32.scene.vox)
    n = 8
    labels, boxes = r.assign_fields(n)
    part = F.Partition(boxes.cpu().numpy().reshape(n, 2, 3).astype(np.int32),
                       labels.cpu().numpy().view(np.uint16).copy())
    aff = F.field_affine(room32.scene, part)
    r.load_fields(part.field_of_rank, aff)
    w = F.xavier_weights(1, F.ROLE_TEACHER, n, 32, 2)
    r.load_weights(w, 32, 2, room32.sigma_scale)
    opts = roam.render_opts(room32.delta, room32.n_max)
    rgb, _, _ = r.render(room32.cams, opts)
    torch.cuda.synchronize()
    grid = O.Grid(room32.scene, part)
    cnt, recs = records(r, room32.cams, opts)
    rep = P.check_render(grid, w, aff, 32, 2, room32.sigma_scale, F.camera_array(room32.cams), None, room32.delta,
                         room32.n_max, cnt, recs, rgb.cpu().numpy(), tol=1e-4)
    assert_render(rep)
    r.close()

"""Parity of the progressive occupancy update (Eq. 6) with the oracle, on
depth and opacity maps rendered by the library itself (both sides take the
same FP32 maps as input).

Integer decisions -- which voxels a ray crosses, which voxel it ends in,
hit over free -- are exact in both (FP64 traversals); a voxel may differ
only where the oracle reports a near-tie interval (a segment passing
within 1e-9 voxel of a voxel edge: at most two voxels per such interval),
with no allowance beyond that.  Log-odds: FP32 sums of the same
increments, within 1e-5.  Occupancy bits: identical except voxels whose
log-odds sit within 1e-4 of the threshold."""
import math

import numpy as np
import pytest

import fixtures as F
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def roam():
    import paper_2208_02705_gb300 as roam
    from paper_2208_02705_gb300 import build
    build.build()
    return roam


def _compare(L_gpu, L_ref, bits_gpu, bits_ref, ties):
    diff = np.abs(L_gpu.astype(np.float64) - L_ref)
    touched = np.count_nonzero(L_ref)
    bad = diff > 1e-5
    assert touched > 100
    assert bad.sum() <= 2 * max(ties, 0), (bad.sum(), ties, touched)
    thr = math.log(0.97 / 0.03)
    occ_g = np.unpackbits(bits_gpu.view(np.uint8), bitorder="little").astype(bool)
    occ_r = np.unpackbits(bits_ref.view(np.uint8), bitorder="little").astype(bool)
    far = np.abs(L_ref - thr) > 1e-4
    assert np.array_equal(occ_g[far & ~bad], occ_r[far & ~bad])


def _render_maps(roam, r, cams, wl, precision):
    opts = roam.render_opts(wl.delta, wl.n_max, precision=precision)
    _, depth, op = r.render(cams, opts)
    torch.cuda.synchronize()
    return depth, op


def test_occupancy_room32_three_scans(roam, room32):
    r = roam.Roam(0)
    r.load_workload(room32)
    cams = [room32.cams[0],
            F.Camera(F.EQUIRECT, 96, 48, 0.0, F.yaw_pitch(1.1, 0.05), room32.cams[0].o + np.array([0.3, 0.0, -0.2])),
            F.Camera(F.PERSPECTIVE, 80, 60, math.pi / 2, F.yaw_pitch(-0.7, 0.1), room32.cams[0].o)]
    depth, op = _render_maps(roam, r, cams, room32, roam.ROAM_F32)
    n_vox = 32 ** 3
    L = torch.zeros(n_vox, dtype=torch.float32, device="cuda")
    bits = torch.zeros(n_vox // 32, dtype=torch.int32, device="cuda")
    r.occupancy_update(cams, depth, op, L, bits)
    torch.cuda.synchronize()
    r.check()
    Lr = np.zeros(n_vox)
    bits_r, ties = O.occupancy_update(room32.scene.dims, room32.scene.origin, room32.scene.vox, Lr,
                                      F.camera_array(cams), depth.cpu().numpy(), op.cpu().numpy())
    _compare(L.cpu().numpy(), Lr, bits.cpu().numpy().view(np.uint32), bits_r, ties)
    # repeated scans of the same views saturate at the clamp, never past it
    for _ in range(6):
        r.occupancy_update(cams, depth, op, L, bits)
    torch.cuda.synchronize()
    Lg = L.cpu().numpy()
    assert Lg.min() >= -2.0 and Lg.max() <= 3.5
    assert np.isclose(Lg.max(), 3.5) and np.isclose(Lg.min(), -2.0)
    r.close()


def test_occupancy_floor256_scans_sampled_views(roam):
    """Four 256x128 equirect scans of the eight-room floor (BF16 render)."""
    wl = F.floor256(views="equirect")
    r = roam.Roam(0)
    r.load_workload(wl)
    cams = F.make_cameras(wl.scene, 6, [(F.EQUIRECT, 256, 128, 0.0)] * 4)
    depth, op = _render_maps(roam, r, cams, wl, roam.ROAM_BF16)
    n_vox = 256 ** 3
    L = torch.zeros(n_vox, dtype=torch.float32, device="cuda")
    bits = torch.zeros(n_vox // 32, dtype=torch.int32, device="cuda")
    r.occupancy_update(cams, depth, op, L, bits)
    torch.cuda.synchronize()
    r.check()
    Lr = np.zeros(n_vox)
    bits_r, ties = O.occupancy_update(wl.scene.dims, wl.scene.origin, wl.scene.vox, Lr, F.camera_array(cams),
                                      depth.cpu().numpy(), op.cpu().numpy())
    _compare(L.cpu().numpy(), Lr, bits.cpu().numpy().view(np.uint32), bits_r, ties)
    r.close()


def test_occupancy_transparent_maps_change_nothing(roam, room32):
    r = roam.Roam(0)
    r.load_workload(room32)
    n = room32.cams[0].n_pixels
    depth = torch.rand(n, device="cuda")
    op = torch.full((n,), 0.3, device="cuda")          # below the opacity floor
    L = torch.full((32 ** 3,), 0.25, dtype=torch.float32, device="cuda")
    bits = torch.zeros(32 ** 3 // 32, dtype=torch.int32, device="cuda")
    r.occupancy_update(room32.cams, depth, op, L, bits)
    torch.cuda.synchronize()
    assert torch.all(L == 0.25)
    assert int(bits.abs().sum()) == 0
    r.close()

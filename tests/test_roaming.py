"""Stereo eye placement of the roaming loop (CPU) and the loop itself on
the GPU: both eyes rendered in one graph-replayed call per frame give the
same bits as separate plain renders of each eye."""
import numpy as np
import pytest

import fixtures as F
from paper_2208_02705_gb300.roaming import roam_frames, stereo_pair


def test_stereo_pair_geometry():
    cam = F.Camera(F.PERSPECTIVE, 64, 32, 1.2, F.yaw_pitch(0.7, 0.2), np.array([1.0, 2.0, 3.0]))
    left, right = stereo_pair(cam, 0.064)
    assert np.allclose(right.o - left.o, 0.064 * np.asarray(cam.R)[:, 0])
    assert np.allclose(0.5 * (left.o + right.o), cam.o)
    assert np.array_equal(left.R, cam.R) and np.array_equal(right.R, cam.R)
    assert (left.width, left.height, left.fov_h) == (cam.width, cam.height, cam.fov_h)


def test_roaming_path_stays_in_free_space():
    wl = F.floor256(views="equirect")
    cams = F.roaming_path(wl.scene, 2, 50)
    for c in cams:
        v = np.floor(np.asarray(c.o) / wl.scene.vox).astype(int)
        assert not wl.scene.occ[v[2], v[1], v[0]]


@pytest.mark.gpu
def test_stereo_loop_graph_frames_match_plain_renders(room32):
    torch = pytest.importorskip("torch")
    import paper_2208_02705_gb300 as roam
    from paper_2208_02705_gb300 import build
    build.build()
    r = roam.Roam(0)
    r.load_workload(room32)
    poses = F.roaming_path(room32.scene, 1, 6, width=96, height=64)
    gopts = roam.render_opts(room32.delta, room32.n_max, precision=roam.ROAM_BF16, use_graph=True)
    times, (lt, rt) = roam_frames(r, poses, gopts)
    assert len(times) == 6 and all(t > 0 for t in times)
    opts = roam.render_opts(room32.delta, room32.n_max, precision=roam.ROAM_BF16)
    left, right = stereo_pair(poses[-1])
    l_ref = r.render([left], opts)[0]
    r_ref = r.render([right], opts)[0]
    torch.cuda.synchronize()
    assert torch.equal(lt, l_ref) and torch.equal(rt, r_ref)
    assert not torch.equal(lt, rt)
    r.close()


@pytest.mark.gpu
@pytest.mark.parametrize("which,prec", [("room32", "bf16"), ("room32", "f32"), ("floor256", "bf16")])
def test_stereo_frame_matches_oracle(room32, which, prec):
    """Both eyes of the last frame of a graph-replayed walk against the FP64
    oracle under the render parity rule (oracle.parity): the room's 96x64
    eye pair on every pixel, the eight-room floor's 1280x720 pair (the
    benchmark's eyes) on 3000 sampled pixels."""
    torch = pytest.importorskip("torch")
    import oracle as O
    import oracle.parity as P
    from gpu_parity import assert_render, records
    import paper_2208_02705_gb300 as roam
    from paper_2208_02705_gb300 import build
    build.build()
    wl = room32 if which == "room32" else F.floor256(views="equirect")
    size = (96, 64) if which == "room32" else (1280, 720)
    r = roam.Roam(0)
    r.load_workload(wl)
    poses = F.roaming_path(wl.scene, 1 if which == "room32" else 2, 4, width=size[0], height=size[1])
    p = roam.ROAM_BF16 if prec == "bf16" else roam.ROAM_F32
    opts = roam.render_opts(wl.delta, wl.n_max, precision=p)
    gopts = roam.render_opts(wl.delta, wl.n_max, precision=p, use_graph=True)
    _, (lt, rt) = roam_frames(r, poses, gopts)
    eyes = list(stereo_pair(poses[-1]))
    got_all = torch.cat([lt, rt]).cpu().numpy().astype(np.float64)
    n_eye = size[0] * size[1]
    if which == "room32":
        rays = None
        got = got_all
    else:
        rng = np.random.default_rng(720)
        view = rng.integers(0, 2, 3000)
        rays = np.stack([view, rng.integers(0, n_eye, 3000)], 1).astype(np.uint32)
        got = got_all[view * n_eye + rays[:, 1].astype(np.int64)]
    cnt, recs = records(r, eyes, opts, rays)
    g = O.Grid(wl.scene, wl.part)
    rep = P.check_render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, F.camera_array(eyes), rays, wl.delta,
                         wl.n_max, cnt, recs, got, tol=2e-2 if prec == "bf16" else 1e-4)
    assert_render(rep, psnr_min=40.0 if prec == "bf16" else None, got=got)
    r.close()

"""Parity of the CUDA render path (through the C ABI) with the FP64 oracle.

Integer work (sample indices, field ids, bucketing) is compared bit-exactly.
A ray whose kept-sample list differs from the oracle's must be certified by
the oracle (every differing sample within 1e-3 voxel of a face whose two
sides differ), and such rays stay below 0.1% of rays.  Colours are held to
their bar on EVERY ray: against the oracle's render where the lists agree,
against the oracle recomputed on the library's own list where they differ
(oracle.parity).  FP32 colours: <= 1e-4 max abs (plus t_stop where the
transmittance meets the stopping threshold within 1e-3 in log space).
BF16 colours: >= 40 dB PSNR and <= 2e-2 max abs."""
import math

import numpy as np
import pytest

import fixtures as F
import oracle as O
import oracle.parity as P
from gpu_parity import assert_march, assert_render, records

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def roam():
    import paper_2208_02705_gb300 as roam
    from paper_2208_02705_gb300 import build
    build.build()
    return roam


@pytest.fixture(scope="module")
def room(roam, room32):
    r = roam.Roam(0)
    r.load_workload(room32)
    yield r
    r.close()


@pytest.fixture(scope="module")
def floor():
    return F.floor256()


@pytest.fixture(scope="module")
def floor_grid(floor):
    return O.Grid(floor.scene, floor.part)


@pytest.fixture(scope="module")
def floor_ctx(roam, floor):
    r = roam.Roam(0)
    r.load_workload(floor)
    yield r
    r.close()


def test_march_room32_all_pixels(roam, room, room32, room32_grid):
    opts = roam.render_opts(room32.delta, room32.n_max)
    cnt, recs = records(room, room32.cams, opts)
    _, rep, _ = P.check_march(room32_grid, F.camera_array(room32.cams), None, room32.delta, room32.n_max, cnt, recs)
    assert_march(rep, rep.n)
    assert cnt.sum() > 0


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_march_ragged_ray_list_and_perspective(roam, room, room32, room32_grid, precision):
    cams = [room32.cams[0], F.Camera(F.PERSPECTIVE, 37, 23, 1.3, F.yaw_pitch(0.4, -0.2), room32.cams[0].o)]
    rng = np.random.default_rng(3)
    n = 1001
    view = rng.integers(0, 2, n)
    pix = np.where(view == 0, rng.integers(0, 128 * 64, n), rng.integers(0, 37 * 23, n))
    rays_np = np.stack([view, pix], 1).astype(np.uint32)
    prec = roam.ROAM_F32 if precision == "f32" else roam.ROAM_BF16
    opts = roam.render_opts(room32.delta, 17, precision=prec)
    cnt, recs = records(room, cams, opts, rays_np)
    (cnt_o, _, _), rep, _ = P.check_march(room32_grid, F.camera_array(cams), rays_np, room32.delta, 17, cnt, recs)
    assert_march(rep, n)
    assert (cnt_o == 17).any()       # the cap is exercised


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_march_floor256_sampled(roam, floor_ctx, floor, floor_grid, precision):
    rng = np.random.default_rng(5)
    n = 20000
    view = rng.integers(0, 2, n)
    sizes = [c.n_pixels for c in floor.cams]
    pix = np.array([rng.integers(0, sizes[v]) for v in view])
    rays_np = np.stack([view, pix], 1).astype(np.uint32)
    prec = roam.ROAM_F32 if precision == "f32" else roam.ROAM_BF16
    opts = roam.render_opts(floor.delta, floor.n_max, precision=prec)
    cnt, recs = records(floor_ctx, floor.cams, opts, rays_np)
    _, rep, _ = P.check_march(floor_grid, F.camera_array(floor.cams), rays_np, floor.delta, floor.n_max, cnt, recs)
    assert_march(rep, n)


@pytest.mark.parametrize("n,which,skew", [(0, "room", False), (1, "room", False), (4096, "room3", False),
                                          (100003, "floor", True), (5000, "floor", False)])
def test_bucket_groups_by_field(roam, room, floor_ctx, n, which, skew):
    ctx = floor_ctx if which == "floor" else room
    Fn = ctx.n_fields
    rng = np.random.default_rng(n + 1)
    if skew:
        keys = np.minimum(rng.zipf(1.2, n) - 1, Fn - 1)        # Zipf-skewed field sizes
    elif which == "room3":
        keys = rng.integers(0, 3, n)                           # empty fields at the end
    else:
        keys = rng.integers(0, Fn, n)
    keys_t = torch.from_numpy(keys.astype(np.int16)).cuda()
    perm, offsets = ctx.bucket(keys_t)
    torch.cuda.synchronize()
    ctx.check()
    perm = perm.cpu().numpy().astype(np.int64)
    offsets = offsets.cpu().numpy().astype(np.int64)
    expect_off = np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=Fn))])
    assert np.array_equal(offsets, expect_off)
    assert np.array_equal(np.sort(perm), np.arange(n))
    for f in range(Fn):
        seg = perm[offsets[f]:offsets[f + 1]]
        assert (keys[seg] == f).all()


def _points_in_fields(wl, n, rng):
    boxes = wl.part.boxes
    f = rng.integers(0, boxes.shape[0], n)
    lo = boxes[f, 0, :] * wl.scene.vox
    hi = boxes[f, 1, :] * wl.scene.vox
    p = lo + rng.uniform(0, 1, (n, 3)) * (hi - lo)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return p.astype(np.float32), d.astype(np.float32), f.astype(np.uint16)


def test_mlp_eval_f32_matches_oracle(roam, room32):
    W, H = room32.W, room32.H
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.3)
    r = roam.Roam(0)
    r.load_grid(room32.scene.bits, room32.scene.dims, room32.scene.origin, room32.scene.vox)
    r.load_fields(room32.part.field_of_rank, room32.affine)
    r.load_weights(w, W, H, room32.sigma_scale)
    rng = np.random.default_rng(9)
    n = 1531
    p, d, f = _points_in_fields(room32, n, rng)
    out = r.mlp_eval(torch.from_numpy(p).cuda(), torch.from_numpy(d).cuda(),
                     torch.from_numpy(f.astype(np.int16)).cuda(), roam.ROAM_F32)
    torch.cuda.synchronize()
    out = out.cpu().numpy().astype(np.float64)
    for i in range(n):
        ref = O.mlp(w[f[i]], W, H, room32.sigma_scale, room32.affine[f[i]], p[i].astype(np.float64),
                    d[i].astype(np.float64))
        # FP32 rounding of x_loc (6e-8) is amplified by the 2^9 pi encoding
        # frequency to ~1e-4 in the features; sigma carries sigma_scale on top
        assert abs(out[i, 0] - ref[0]) <= 1e-4 * max(1.0, ref[0]), (i, out[i], ref)
        assert np.all(np.abs(out[i, 1:] - ref[1:]) <= 2e-5), (i, out[i], ref)
    r.close()


def test_composite_matches_oracle(roam, room):
    rng = np.random.default_rng(4)
    n, n_max = 777, 40
    cnt = rng.integers(0, n_max + 1, n)
    sr = np.zeros((n, n_max, 4), np.float32)
    sr[..., 0] = rng.exponential(8.0, (n, n_max))
    sr[..., 1:] = rng.uniform(0, 1, (n, n_max, 3))
    t = np.cumsum(rng.uniform(0.01, 0.05, (n, n_max)), axis=1).astype(np.float32)
    delta, t_stop, bg = 0.025, 1e-4, (0.2, 0.3, 0.4)
    opts = roam.render_opts(delta, n_max, t_stop, bg)
    rgb, depth, op, used = room.composite(torch.from_numpy(cnt.astype(np.int32)).cuda(),
                                          torch.from_numpy(sr).cuda(), torch.from_numpy(t).cuda(), opts)
    torch.cuda.synchronize()
    rgb, depth, op, used = (x.cpu().numpy() for x in (rgb, depth, op, used))
    df = O.f32(delta)
    for r_ in range(n):
        c = int(cnt[r_])
        out, u, margin = O.composite(sr[r_, :c, 0], sr[r_, :c, 1:], t[r_, :c], df, O.f32(t_stop),
                                     [O.f32(b) for b in bg])
        # a transmittance within 1e-4 (log space) of t_stop may stop one
        # sample either side; that sample weighs at most t_stop
        extra = 0.0
        if u != used[r_]:
            assert margin < 1e-4 and abs(int(used[r_]) - u) == 1
            extra = O.f32(t_stop)
        assert np.abs(rgb[r_] - out[:3]).max() <= 2e-6 + extra
        assert abs(op[r_] - out[4]) <= 2e-6 + extra
        assert abs(depth[r_] - out[3]) <= 2e-6 * max(1.0, out[3]) + extra * float(t[r_, :c].max(initial=0.0))


def test_render_room32_f32(roam, room, room32, room32_grid):
    opts = roam.render_opts(room32.delta, room32.n_max)
    rgb, depth, op = room.render(room32.cams, opts)
    torch.cuda.synchronize()
    room.check()
    cnt, recs = records(room, room32.cams, opts)
    rep = P.check_render(room32_grid, room32.weights, room32.affine, room32.W, room32.H, room32.sigma_scale,
                         F.camera_array(room32.cams), None, room32.delta, room32.n_max, cnt, recs,
                         rgb.cpu().numpy(), depth.cpu().numpy(), op.cpu().numpy(), tol=1e-4)
    assert_render(rep, depth_tol=1e-4 * max(1.0, float(np.abs(depth.cpu().numpy()).max())), opacity_tol=1e-4)


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_render_round_schedule_is_invisible(roam, room, room32, precision):
    """Rounds (and a smaller first round) change the work done, never the
    result: bit-identical images and composited-sample counts."""
    prec = roam.ROAM_F32 if precision == "f32" else roam.ROAM_BF16
    outs = []
    for R, R0 in ((1, 0), (7, 0), (32, 0), (64, 0), (32, 4), (16, 5), (64, 8)):
        opts = roam.render_opts(room32.delta, room32.n_max, round_size=R, first_round_size=R0, precision=prec)
        rgb, depth, op = room.render(room32.cams, opts)
        torch.cuda.synchronize()
        outs.append((rgb.clone(), depth.clone(), op.clone(), room.get_stats().n_used))
    for o in outs[1:]:
        for a, b in zip(outs[0][:3], o[:3]):
            assert torch.equal(a, b)
        assert o[3] == outs[0][3]


def test_round_size_tuner_picks_a_valid_pair(roam, room, room32):
    base = roam.render_opts(room32.delta, room32.n_max, precision=roam.ROAM_BF16)
    R, R0, ms = room.tune_round_size(room32.cams, base)
    assert 4 <= R <= room32.n_max and 4 <= R0 <= R and ms > 0
    ref = [x.clone() for x in room.render(room32.cams, base)]
    tuned = room.render(room32.cams, roam.render_opts(room32.delta, room32.n_max, precision=roam.ROAM_BF16,
                                                      round_size=R, first_round_size=R0))
    torch.cuda.synchronize()
    for a, b in zip(ref, tuned):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_render_graph_replay_is_bit_identical(roam, room, room32, precision):
    """CUDA-graph replay (captured once per configuration) gives the same bits
    as plain launches; a new camera set of another size, new output buffers
    and host outputs each re-capture."""
    prec = roam.ROAM_F32 if precision == "f32" else roam.ROAM_BF16
    plain = roam.render_opts(room32.delta, room32.n_max, precision=prec)
    graph = roam.render_opts(room32.delta, room32.n_max, precision=prec, use_graph=True)
    persp = [F.Camera(F.PERSPECTIVE, 40, 24, math.pi / 2, F.yaw_pitch(0.3, 0.1), room32.cams[0].o)]
    for cams in (room32.cams, persp, room32.cams):
        ref = [t.clone() for t in room.render(cams, plain)]
        outs = [room.render(cams, graph) for _ in range(3)]        # capture, then two replays
        torch.cuda.synchronize()
        for o in outs:
            for a, b in zip(ref, o):
                assert torch.equal(a, b)
        n = ref[0].shape[0]
        rgb_h = np.zeros((n, 3), np.float32)
        room.render_host(cams, graph, rgb_h)
        assert np.array_equal(rgb_h, ref[0].cpu().numpy())
    st = room.get_stats()
    assert st.n_rays == 128 * 64


def test_render_host_outputs_match_device(roam, room, room32):
    opts = roam.render_opts(room32.delta, room32.n_max)
    rgb_d, depth_d, op_d = room.render(room32.cams, opts)
    n = 128 * 64
    rgb_h = np.zeros((n, 3), np.float32)
    depth_h = np.zeros(n, np.float32)
    op_h = np.zeros(n, np.float32)
    room.render_host(room32.cams, opts, rgb_h, depth_h, op_h)
    assert np.array_equal(rgb_h, rgb_d.cpu().numpy())
    assert np.array_equal(depth_h, depth_d.cpu().numpy())
    assert np.array_equal(op_h, op_d.cpu().numpy())


def test_render_edge_cases(roam, room32):
    r = roam.Roam(0)
    occ = np.zeros((32, 32, 32), dtype=bool)
    r.load_grid(F.pack_bits(occ), (32, 32, 32), (0, 0, 0), 0.1)
    aff = np.array([[1, 1, 1, 0, 0, 0]], dtype=np.float32)
    r.load_fields(np.zeros(0, np.uint16), aff)
    r.load_weights(np.zeros((1, F.n_params(32, 2)), np.float32), 32, 2, 1.0)
    opts = roam.render_opts(0.025, 64, bg=(0.25, 0.5, 0.75))
    # camera inside, and camera outside looking away from the grid
    cams = [room32.cams[0], F.Camera(F.PERSPECTIVE, 33, 17, 1.0, np.eye(3), np.array([-5.0, 1.6, 1.6]))]
    cams[1].R = F.yaw_pitch(math.pi, 0)        # looking along -z, away from the box
    rgb, depth, op = r.render(cams, opts)
    torch.cuda.synchronize()
    assert torch.allclose(rgb, torch.tensor([0.25, 0.5, 0.75], device="cuda").expand_as(rgb))
    assert float(op.abs().max()) == 0.0
    r.close()


def test_render_floor256_f32_sampled(roam, floor_ctx, floor, floor_grid):
    """Full-size render of both views (the benchmark's launch configuration);
    the oracle checks a sample of pixels one by one."""
    opts = roam.render_opts(floor.delta, floor.n_max)
    rgb, depth, op = floor_ctx.render(floor.cams, opts)
    torch.cuda.synchronize()
    floor_ctx.check()
    rng = np.random.default_rng(17)
    sizes = [c.n_pixels for c in floor.cams]
    starts = np.concatenate([[0], np.cumsum(sizes)])
    n = 6000
    view = rng.integers(0, 2, n)
    pix = np.array([rng.integers(0, sizes[v]) for v in view])
    rays = np.stack([view, pix], 1).astype(np.uint32)
    cnt, recs = records(floor_ctx, floor.cams, opts, rays)
    gi = starts[view] + pix
    rep = P.check_render(floor_grid, floor.weights, floor.affine, floor.W, floor.H, floor.sigma_scale,
                         F.camera_array(floor.cams), rays, floor.delta, floor.n_max, cnt, recs,
                         rgb.cpu().numpy()[gi], depth.cpu().numpy()[gi], op.cpu().numpy()[gi], tol=1e-4)
    assert_render(rep, depth_tol=1e-4 * max(1.0, float(np.abs(depth.cpu().numpy()[gi]).max())), opacity_tol=1e-4)


def test_errors_are_reported(roam, room, room32):
    opts = roam.render_opts(room32.delta, 0)
    with pytest.raises(roam.RoamError) as e:
        room.render(room32.cams, opts)
    assert e.value.status == -1
    opts = roam.render_opts(-1.0, 8)
    with pytest.raises(roam.RoamError):
        room.render(room32.cams, opts)
    bad_cam = F.Camera(7, 8, 8, 0.0, np.eye(3), np.zeros(3))
    with pytest.raises(roam.RoamError):
        room.render([bad_cam], roam.render_opts(room32.delta, 8))
    r = roam.Roam(0)
    with pytest.raises(roam.RoamError) as e:
        r.render(room32.cams, roam.render_opts(room32.delta, 8))
    assert e.value.status == -4
    with pytest.raises(roam.RoamError):
        r.load_grid(np.zeros(10, np.uint32), (33, 32, 32), (0, 0, 0), 0.1)
    r.load_grid(room32.scene.bits, room32.scene.dims, room32.scene.origin, room32.scene.vox)
    with pytest.raises(roam.RoamError):        # wrong occupied count
        r.load_fields(room32.part.field_of_rank[:-1], room32.affine)
    lab = room32.part.field_of_rank.copy()
    lab[0] = 99
    with pytest.raises(roam.RoamError):        # label >= n_fields
        r.load_fields(lab, room32.affine)
    r.load_fields(room32.part.field_of_rank, room32.affine)
    w = room32.weights.copy()
    w[3, 5] = np.nan
    with pytest.raises(roam.RoamError):
        r.load_weights(w, room32.W, room32.H, room32.sigma_scale)
    r.close()

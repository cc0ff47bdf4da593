"""The tensor-core (tcgen05, BF16 operands, FP32 accumulation) adjoint of
the per-field MLPs through the C ABI, against the oracle's adjoint on the
same output gradients.

Parity is against the oracle's BF16 reading of the same arithmetic (BF16
inputs, weights and biases in the forward layers; BF16 output gradients,
inputs and weights in the adjoint products; sums in FP64): cosine >=
0.99995 and within 3e-2 of max |g| per parameter -- FP32 accumulation
makes values round to neighbouring BF16 numbers, and a pre-activation
within rounding of zero flips a ReLU mask, which moves single entries by
up to ~2 % of max |g|.  Against the FP64
adjoint the BF16 arithmetic itself moves the gradient by 1-6 % of max |g|
(cosine 0.998-0.9995 on these networks): a sanity bar of 8e-2 and cosine
0.995.  Cases span several 128-sample tiles per field with a ragged last
tile, more tiles than CTAs (the TMEM accumulators carry across tiles of
one field and are flushed at field changes), fields without samples, and
every supported (W, H)."""
import numpy as np
import pytest

import fixtures as F
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIGMA_SCALE = 2.0


@pytest.fixture(scope="module")
def roam():
    import paper_2208_02705_gb300 as roam
    from paper_2208_02705_gb300 import build
    build.build()
    return roam


def _ctx(roam, wl, W, H, w):
    r = roam.Roam(0)
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    r.load_fields(wl.part.field_of_rank, wl.affine)
    r.load_weights(w, W, H, SIGMA_SCALE)
    return r


def _close(g, ref, what, tol, cos_min):
    gm = np.abs(ref).max()
    assert gm > 0
    err = np.abs(g - ref).max() / gm
    cos = float((g * ref).sum() / (np.linalg.norm(g) * np.linalg.norm(ref)))
    print(f"{what}: max err {err:.3e} of max|g|, cosine {cos:.6f}")
    assert err <= tol and cos >= cos_min, (what, err, cos)
    return err, cos


@pytest.mark.parametrize("W,H,per_field", [(32, 1, 700), (32, 2, 4000), (32, 3, 1500), (32, 4, 1000),
                                           (64, 1, 1000), (64, 2, 700), (64, 3, 4000)])
def test_bf16_adjoint_matches_oracle(roam, room32, W, H, per_field):
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.1)
    r = _ctx(roam, room32, W, H, w)
    p, d, f = F.distill_points(room32.scene, room32.part, 3, per_field)
    keep = (f != 2) & (f != 5)                      # two fields without samples
    p, d, f = p[keep], d[keep], f[keep]
    dl = (np.random.default_rng(W + H).normal(size=(p.shape[0], 4)) * 0.05).astype(np.float32)
    pt, dt = torch.from_numpy(p).cuda(), torch.from_numpy(d).cuda()
    ft = torch.from_numpy(f.astype(np.int16)).cuda()
    dlt = torch.from_numpy(dl).cuda()
    g = r.mlp_backward(pt, dt, ft, dlt, precision=roam.ROAM_BF16)
    g32 = r.mlp_backward(pt, dt, ft, dlt, precision=roam.ROAM_F32)
    torch.cuda.synchronize()
    r.check()
    g = g.cpu().numpy().astype(np.float64)
    g_b, _ = O.mlp_grad_points(w, room32.affine, W, H, SIGMA_SCALE, p, d, f, dl, quant=2)
    g_o, _ = O.mlp_grad_points(w, room32.affine, W, H, SIGMA_SCALE, p, d, f, dl)
    assert np.all(g[2] == 0) and np.all(g[5] == 0)
    _close(g, g_b, f"W{W}H{H} vs oracle BF16 reading", 3e-2, 0.99995)
    _close(g, g_o, f"W{W}H{H} vs oracle FP64", 8e-2, 0.995)
    _close(g, g32.cpu().numpy().astype(np.float64), f"W{W}H{H} vs FP32 adjoint", 8e-2, 0.995)
    # deterministic up to the order of the flush atomics: a second run agrees closely
    g2 = r.mlp_backward(pt, dt, ft, dlt, precision=roam.ROAM_BF16)
    torch.cuda.synchronize()
    assert np.abs(g2.cpu().numpy() - g).max() <= 1e-5 * np.abs(g).max()
    r.close()


def test_bf16_adjoint_empty_and_unsupported(roam, room32):
    W, H = 64, 3
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.1)
    r = _ctx(roam, room32, W, H, w)
    z3 = torch.zeros((0, 3), device="cuda")
    g = r.mlp_backward(z3, z3, torch.zeros(0, dtype=torch.int16, device="cuda"),
                       torch.zeros((0, 4), device="cuda"), precision=roam.ROAM_BF16)
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(g)) == 0
    r.close()
    w4 = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, 64, 4, bias_scale=0.1)
    r = _ctx(roam, room32, 64, 4, w4)
    p, d, f = F.distill_points(room32.scene, room32.part, 3, 16)
    with pytest.raises(roam.RoamError):
        r.mlp_backward(torch.from_numpy(p).cuda(), torch.from_numpy(d).cuda(),
                       torch.from_numpy(f.astype(np.int16)).cuda(), torch.zeros((p.shape[0], 4), device="cuda"),
                       precision=roam.ROAM_BF16)
    r.close()


def test_train_backward_bf16_tensor_cores_floor256(roam):
    """The fine-tuning step's adjoint on the 256^3 floor (512 W=64/H=3
    fields, 16384 random rays): after a BF16 forward it runs on the tensor
    cores; against the FP32 adjoint after an FP32 forward (itself pinned to
    FP64 finite differences) within the BF16 sanity bar."""
    wl = F.floor256()
    W, H = wl.W, wl.H
    student = F.xavier_weights(2, F.ROLE_STUDENT, wl.part.n_fields, W, H, bias_scale=0.05)
    r = roam.Roam(0)
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    r.load_fields(wl.part.field_of_rank, wl.affine)
    r.load_weights(student, W, H, wl.sigma_scale)
    rng = np.random.default_rng(21)
    n = 16384
    view = rng.integers(0, len(wl.cams), n)
    pix = np.array([rng.integers(0, wl.cams[v].n_pixels) for v in view])
    rays = torch.from_numpy(np.stack([view, pix], 1).astype(np.int32)).cuda()
    tgt = torch.from_numpy(rng.uniform(0, 1, (n, 3)).astype(np.float32)).cuda()
    grads = {}
    r.profile(True)
    for prec in (roam.ROAM_F32, roam.ROAM_BF16):
        opts = roam.render_opts(wl.delta, wl.n_max, precision=prec)
        rgb = r.train_forward(wl.cams, rays, opts)
        dl = ((2.0 / (3.0 * n)) * (rgb - tgt)).contiguous()
        grads[prec] = r.train_backward(dl).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    names = set(r.profile_read())
    r.check()
    assert "mlp_bwd_bf16_tcgen05" in names and "mlp_bwd" in names
    _close(grads[roam.ROAM_BF16], grads[roam.ROAM_F32], "floor256 BF16 vs FP32 adjoint", 8e-2, 0.995)
    r.close()


def test_train_backward_bf16_floor256_against_oracle(roam):
    """The fine-tuning step of the 256^3 floor as the training benchmark runs
    it (512 W=64/H=3 student fields; targets rendered by the teacher weights
    plus N(0, 0.01^2) noise; BF16 forward, tensor-core adjoint) on 8192
    random rays, against the oracle's FP64 analytic gradient of the same
    loss (no BF16 reading): within 3e-2 of max|g|, cosine >= 0.999."""
    wl = F.floor256()
    W, H = wl.W, wl.H
    g_o = O.Grid(wl.scene, wl.part)
    cams = F.camera_array(wl.cams)
    student = F.xavier_weights(2, F.ROLE_STUDENT, wl.part.n_fields, W, H, bias_scale=0.05)
    rng = np.random.default_rng(41)
    n = 8192
    view = rng.integers(0, len(wl.cams), n)
    pix = np.array([rng.integers(0, wl.cams[v].n_pixels) for v in view])
    rays_np = np.stack([view, pix], 1).astype(np.uint32)
    teacher = O.render(g_o, wl.weights, wl.affine, W, H, wl.sigma_scale, cams, rays_np, wl.delta, wl.n_max)
    target = (teacher["rgb"] + F.rng_for(3, F.ROLE_NOISE).normal(0, 0.01, (n, 3))).astype(np.float32)
    r = roam.Roam(0)
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    r.load_fields(wl.part.field_of_rank, wl.affine)
    r.load_weights(student, W, H, wl.sigma_scale)
    rays = torch.from_numpy(rays_np.astype(np.int32)).cuda()
    opts = roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16)
    rgb = r.train_forward(wl.cams, rays, opts)
    dl = ((2.0 / (3.0 * n)) * (rgb - torch.from_numpy(target).cuda())).contiguous()
    g = r.train_backward(dl).cpu().numpy().astype(np.float64)
    r.check()
    _, go, _, _ = O.loss_grad(g_o, student, wl.affine, W, H, wl.sigma_scale, cams, rays_np, target, wl.delta,
                              wl.n_max)
    _close(g, go, "floor256 BF16 adjoint vs oracle FP64", 3e-2, 0.999)
    r.close()

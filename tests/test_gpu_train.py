"""Training step (fine-tuning with the L2 photometric loss) through the C ABI
against the FP64 oracle: forward colours, the hand-written adjoint of
compositing + MLPs + encoding, finite differences, and Adam.

Tolerances (derived): FP32 gradients within 1e-3 of max|g| of the oracle's
analytic FP64 gradient (FP32 sums of O(10^3) terms per weight);
BF16-forward gradients within 3e-2 of max|g| with cosine >= 0.999."""
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


def _ctx(roam, wl, weights, W, H):
    r = roam.Roam(0)
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    r.load_fields(wl.part.field_of_rank, wl.affine)
    r.load_weights(weights, W, H, wl.sigma_scale)
    return r


def _rays(wl, n, seed):
    rng = np.random.default_rng(seed)
    sizes = [c.n_pixels for c in wl.cams]
    view = rng.integers(0, len(sizes), n)
    pix = np.array([rng.integers(0, sizes[v]) for v in view])
    return np.stack([view, pix], 1).astype(np.uint32)


def _grad_gpu(roam, r, wl, rays_np, target, precision):
    rays = torch.from_numpy(rays_np.astype(np.int32)).cuda()
    opts = roam.render_opts(wl.delta, wl.n_max, precision=precision)
    rgb = r.train_forward(wl.cams, rays, opts)
    tgt = torch.from_numpy(target).cuda()
    n = rays_np.shape[0]
    dl = (2.0 / (3.0 * n)) * (rgb - tgt)
    g = r.train_backward(dl.contiguous())
    torch.cuda.synchronize()
    r.check()
    return rgb.cpu().numpy(), g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", [0, 1])
def test_train_forward_equals_render(roam, room32, prec):
    r = roam.Roam(0)
    r.load_workload(room32)
    rays_np = _rays(room32, 1500, 3)
    rays = torch.from_numpy(rays_np.astype(np.int32)).cuda()
    opts = roam.render_opts(room32.delta, room32.n_max, precision=prec)
    rgb_t = r.train_forward(room32.cams, rays, opts).clone()
    rgb_r, _, _ = r.render(room32.cams, opts)
    torch.cuda.synchronize()
    assert torch.equal(rgb_t, rgb_r[rays[:, 1].long()])
    r.close()


def test_train_backward_matches_oracle_gradient_f32(roam, room32, room32_grid):
    W, H = 32, 2
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.1)
    r = _ctx(roam, room32, w, W, H)
    rays_np = _rays(room32, 2048, 5)
    target = np.random.default_rng(6).uniform(0, 1, (2048, 3)).astype(np.float32)
    rgb, g = _grad_gpu(roam, r, room32, rays_np, target, roam.ROAM_F32)
    loss, go, _, rgb_o = O.loss_grad(room32_grid, w, room32.affine, W, H, room32.sigma_scale,
                                     F.camera_array(room32.cams), rays_np, target, room32.delta, room32.n_max)
    assert np.abs(rgb - rgb_o).max() < 1e-4
    gmax = np.abs(go).max()
    assert gmax > 0
    assert np.abs(g - go).max() <= 1e-3 * gmax, np.abs(g - go).max() / gmax
    assert np.linalg.norm(g - go) <= 1e-3 * np.linalg.norm(go)
    r.close()


def test_train_backward_bf16_forward_close_to_oracle(roam, room32, room32_grid):
    W, H = 32, 2
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.1)
    r = _ctx(roam, room32, w, W, H)
    rays_np = _rays(room32, 2048, 7)
    target = np.random.default_rng(8).uniform(0, 1, (2048, 3)).astype(np.float32)
    _, g = _grad_gpu(roam, r, room32, rays_np, target, roam.ROAM_BF16)
    _, go, _, _ = O.loss_grad(room32_grid, w, room32.affine, W, H, room32.sigma_scale, F.camera_array(room32.cams),
                              rays_np, target, room32.delta, room32.n_max)
    cos = float((g * go).sum() / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert cos >= 0.999, cos
    assert np.abs(g - go).max() <= 3e-2 * np.abs(go).max()
    r.close()


def test_train_backward_floor256_finite_differences(roam):
    """The 256^3 floor with 512 W=64/H=3 fields: student weights, targets
    from the teacher weights plus N(0, 0.01^2) noise, a batch of random rays;
    GPU gradients against FP64 central differences (h = 1e-4) on 32 sampled
    weights, each difference evaluated on the rays that touch its field."""
    wl = F.floor256()
    g_o = O.Grid(wl.scene, wl.part)
    W, H = wl.W, wl.H
    student = F.xavier_weights(2, F.ROLE_STUDENT, wl.part.n_fields, W, H, bias_scale=0.05)
    n = 8192
    rays_np = _rays(wl, n, 11)
    cams = F.camera_array(wl.cams)
    teacher = O.render(g_o, wl.weights, wl.affine, W, H, wl.sigma_scale, cams, rays_np, wl.delta, wl.n_max)
    noise = F.rng_for(3, F.ROLE_NOISE).normal(0, 0.01, (n, 3))
    target = (teacher["rgb"] + noise).astype(np.float32)
    r = _ctx(roam, wl, student, W, H)
    _, g = _grad_gpu(roam, r, wl, rays_np, target, roam.ROAM_F32)
    gmax = np.abs(g).max()
    rng = np.random.default_rng(12)
    # fields that the batch hits, weighted by how often
    hit = np.nonzero(np.abs(g).sum(axis=1) > 0)[0]
    assert hit.size > 50
    h = 1e-4
    checked = 0
    P = student.shape[1]
    for _ in range(64):
        f = int(rng.choice(hit))
        k = int(rng.integers(P))
        mask = O.rays_touching(g_o, cams, rays_np, wl.delta, wl.n_max, f)
        sub, tsub = rays_np[mask], target[mask]
        wp, wm = student.copy(), student.copy()
        wp[f, k] = np.float32(student[f, k] + h)
        wm[f, k] = np.float32(student[f, k] - h)
        lp, _, sp, _ = O.loss_grad(g_o, wp, wl.affine, W, H, wl.sigma_scale, cams, sub, tsub, wl.delta, wl.n_max,
                                   want_grad=False, loss_norm=3.0 * n)
        lm, _, sm, _ = O.loss_grad(g_o, wm, wl.affine, W, H, wl.sigma_scale, cams, sub, tsub, wl.delta, wl.n_max,
                                   want_grad=False, loss_norm=3.0 * n)
        _, _, s0, _ = O.loss_grad(g_o, student, wl.affine, W, H, wl.sigma_scale, cams, sub, tsub, wl.delta, wl.n_max,
                                  want_grad=False, loss_norm=3.0 * n)
        if sp != s0 or sm != s0:
            continue      # the step crosses a ReLU kink or changes a termination index
        fd = (lp - lm) / (float(wp[f, k]) - float(wm[f, k]))
        assert abs(fd - g[f, k]) <= 1e-3 * gmax + 1e-3 * abs(fd), (f, k, fd, g[f, k], gmax)
        checked += 1
        if checked == 32:
            break
    assert checked == 32
    r.close()


def test_adam_matches_oracle_and_refreshes_copies(roam, room32, room32_grid):
    W, H = 32, 2
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.1)
    r = _ctx(roam, room32, w, W, H)
    rng = np.random.default_rng(21)
    wo, m, v = w.astype(np.float64).ravel(), np.zeros(w.size), np.zeros(w.size)
    for step in (1, 2, 3):
        grad = (rng.normal(size=w.shape) * 10.0 ** rng.uniform(-4, -1, w.shape)).astype(np.float32)
        r.adam_step(torch.from_numpy(grad).cuda(), lr=1e-3, step=step)
        wo, m, v = O.adam(wo, m, v, grad.astype(np.float64), 1e-3, step)
    wg = r.get_weights().cpu().numpy().astype(np.float64).ravel()
    assert np.abs(wg - wo).max() <= 1e-6
    # every derived copy (SIMT transposed, row-padded, BF16 images) follows the masters
    new_w = wg.reshape(w.shape).astype(np.float32)
    ref = O.render(room32_grid, new_w, room32.affine, W, H, room32.sigma_scale, F.camera_array(room32.cams), None,
                   room32.delta, room32.n_max)
    cams16 = F.camera_array(room32.cams)

    def parity(prec, rgb, tol, rr, quant=0):
        cnt, recs = records(r, room32.cams, roam.render_opts(room32.delta, room32.n_max, precision=prec))
        rep = P.check_render(room32_grid, new_w, room32.affine, W, H, room32.sigma_scale, cams16, None, room32.delta,
                             room32.n_max, cnt, recs, rgb, tol=tol, quant=quant, ref=rr)
        assert_render(rep)

    for prec, tol in ((roam.ROAM_F32, 1e-4), (roam.ROAM_BF16, 2e-2)):
        rgb, _, _ = r.render(room32.cams, roam.render_opts(room32.delta, room32.n_max, precision=prec))
        torch.cuda.synchronize()
        parity(prec, rgb.cpu().numpy(), tol, ref)
    # the BF16 images that Adam refreshes in place equal a fresh packing of
    # the updated masters: bit-identical renders
    r2 = _ctx(roam, room32, new_w, W, H)
    o16 = roam.render_opts(room32.delta, room32.n_max, precision=roam.ROAM_BF16)
    a16, _, _ = r.render(room32.cams, o16)
    b16, _, _ = r2.render(room32.cams, o16)
    torch.cuda.synchronize()
    assert torch.equal(a16, b16)
    r2.close()
    # the FP8 images, rebuilt lazily at the first FP8 launch after the steps
    ref8 = O.render(room32_grid, new_w, room32.affine, W, H, room32.sigma_scale, F.camera_array(room32.cams), None,
                    room32.delta, room32.n_max, quant=1)
    rgb8, _, _ = r.render(room32.cams, roam.render_opts(room32.delta, room32.n_max, precision=roam.ROAM_FP8))
    torch.cuda.synchronize()
    parity(roam.ROAM_FP8, rgb8.cpu().numpy(), 2e-2, ref8, quant=1)
    # the row-padded copy of the FP32 adjoint, rebuilt at its first launch
    rays_np = _rays(room32, 1024, 23)
    target = np.random.default_rng(24).uniform(0, 1, (1024, 3)).astype(np.float32)
    _, g = _grad_gpu(roam, r, room32, rays_np, target, roam.ROAM_F32)
    _, go, _, _ = O.loss_grad(room32_grid, new_w, room32.affine, W, H, room32.sigma_scale, F.camera_array(room32.cams),
                              rays_np, target, room32.delta, room32.n_max)
    assert np.abs(g - go).max() <= 1e-3 * np.abs(go).max()
    r.close()


def test_training_reduces_loss(roam, room32):
    """Student fitted to teacher renders for 30 Adam steps (lr 1e-3,
    beta = (0.9, 0.99)): the loss goes down."""
    W, H = 32, 2
    teacher = roam.Roam(0)
    teacher.load_workload(room32)
    rgb_t, _, _ = teacher.render(room32.cams, roam.render_opts(room32.delta, room32.n_max))
    student = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H)
    r = _ctx(roam, room32, student, W, H)
    n = 4096
    rays_np = _rays(room32, n, 31)
    rays = torch.from_numpy(rays_np.astype(np.int32)).cuda()
    tgt = rgb_t[rays[:, 1].long()].clone()
    opts = roam.render_opts(room32.delta, room32.n_max, precision=roam.ROAM_BF16)
    losses = []
    for step in range(1, 31):
        rgb = r.train_forward(room32.cams, rays, opts)
        diff = rgb - tgt
        losses.append(float((diff * diff).mean()))
        g = r.train_backward((2.0 / (3.0 * n)) * diff)
        r.adam_step(g, lr=1e-3, step=step)
    torch.cuda.synchronize()
    assert losses[-1] < 0.7 * losses[0], losses
    r.close()
    teacher.close()


def test_l2_loss_kernel_and_local_grad(roam, room32):
    W, H = 32, 2
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.1)
    r = _ctx(roam, room32, w, W, H)
    n = 1000
    rays_np = _rays(room32, n, 41)
    rays = torch.from_numpy(rays_np.astype(np.int32)).cuda()
    target = torch.rand((n, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    opts = roam.render_opts(room32.delta, room32.n_max)
    rgb = r.train_forward(room32.cams, rays, opts).clone()
    norm = 3.0 * 4 * n                     # e.g. a global batch four times this one
    loss, dl = r.l2_loss(rgb, target, norm)
    torch.cuda.synchronize()
    e = (rgb - target).double()
    assert abs(float(loss) - float((e * e).sum() / norm)) <= 1e-5 * float((e * e).sum() / norm)
    assert torch.allclose(dl.double(), 2 * e / norm, rtol=1e-6, atol=1e-12)
    # local_grad = forward + loss + backward on the same rays
    loss2, g2 = r.local_grad(room32.cams, rays, target, opts, norm)
    g1 = r.train_backward(dl)
    torch.cuda.synchronize()
    assert torch.equal(loss2, loss)
    # the per-field gradient is flushed with atomics from several CTAs, so the
    # FP32 sums differ in order between runs: compare to the sums' rounding
    assert (g1 - g2).abs().max() <= 1e-5 * g1.abs().max()
    r.close()


def test_dp_step_single_process_matches_manual_step(roam, room32):
    """dp_train_step without a process group is local_grad + Adam."""
    from paper_2208_02705_gb300.dp import dp_train_step
    W, H = 32, 2
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.1)
    a, b = _ctx(roam, room32, w, W, H), _ctx(roam, room32, w, W, H)
    n = 512
    rays = torch.from_numpy(_rays(room32, n, 43).astype(np.int32)).cuda()
    target = torch.rand((n, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(6))
    opts = roam.render_opts(room32.delta, room32.n_max, precision=roam.ROAM_BF16)
    dp_train_step(a, room32.cams, rays, target, opts, n, 1, 1e-3)
    loss, g = b.local_grad(room32.cams, rays, target, opts, 3.0 * n)
    b.adam_step(g, lr=1e-3, step=1)
    torch.cuda.synchronize()
    # Adam moves each weight by about lr = 1e-3; gradient sums that differ in
    # the last bits (atomic order) move it by a tiny fraction of that
    assert (a.get_weights() - b.get_weights()).abs().max() <= 1e-5
    a.close()
    b.close()

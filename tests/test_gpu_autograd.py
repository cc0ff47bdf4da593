"""The hand-written adjoint behind torch.autograd (RoamRender): loss.backward()
through the library's training forward gives the oracle's FP64 gradient of
the L2 photometric loss (fine-tuning stage) and agrees with FP64 central
differences; the forward follows the weight tensor after an optimizer step;
a backward whose forward state has been replaced raises.

Bars as for the training entry points: FP32 within 1e-3 of max|g| of the
oracle's analytic gradient; BF16 forward + tensor-core adjoint cosine >= 0.999
and within 3e-2 of max|g|; central differences (h = 1e-4, FP64) within
1e-3 of max|g| + 1e-3 relative."""
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


def _setup(roam, wl, w):
    r = roam.Roam(0)
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    r.load_fields(wl.part.field_of_rank, wl.affine)
    r.load_weights(w, wl.W, wl.H, wl.sigma_scale)
    return r


def _batch(wl, n, seed):
    rng = np.random.default_rng(seed)
    rays = np.stack([np.zeros(n, np.int64), rng.integers(0, wl.cams[0].n_pixels, n)], 1).astype(np.uint32)
    target = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    return rays, target


def _loss_and_grad(roam, r, Fn, wt, wl, rays, target, prec):
    opts = roam.render_opts(wl.delta, wl.n_max, precision=prec)
    rgb = Fn.apply(wt, r, wl.cams, torch.from_numpy(rays.astype(np.int32)).cuda(), opts)
    loss = ((rgb - torch.from_numpy(target).cuda()) ** 2).mean()
    loss.backward()
    torch.cuda.synchronize()
    return float(loss), wt.grad.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_autograd_gradient_matches_oracle(roam, room32, room32_grid, prec):
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, room32.W, room32.H, bias_scale=0.1)
    r = _setup(roam, room32, w)
    Fn = roam.render_function()
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    rays, target = _batch(room32, 2048, 31)
    p = roam.ROAM_F32 if prec == "f32" else roam.ROAM_BF16
    loss, g = _loss_and_grad(roam, r, Fn, wt, room32, rays, target, p)
    lo, go, _, _ = O.loss_grad(room32_grid, w, room32.affine, room32.W, room32.H, room32.sigma_scale,
                               F.camera_array(room32.cams), rays, target, room32.delta, room32.n_max)
    gmax = np.abs(go).max()
    assert g.shape == go.shape and gmax > 0
    if prec == "f32":
        assert abs(loss - lo) <= 1e-5 * max(1.0, lo)
        assert np.abs(g - go).max() <= 1e-3 * gmax, np.abs(g - go).max() / gmax
    else:
        cos = float((g * go).sum() / (np.linalg.norm(g) * np.linalg.norm(go)))
        assert cos >= 0.999, cos
        assert np.abs(g - go).max() <= 3e-2 * gmax
    r.close()


def test_autograd_gradient_matches_central_differences(roam, room32, room32_grid):
    """FP64 central differences (h = 1e-4) of the oracle's loss on 16 sampled
    weights of fields the batch touches, steps that cross no ReLU kink and
    change no termination index."""
    w = F.xavier_weights(3, F.ROLE_STUDENT, room32.part.n_fields, room32.W, room32.H, bias_scale=0.1)
    r = _setup(roam, room32, w)
    Fn = roam.render_function()
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    rays, target = _batch(room32, 1024, 33)
    _, g = _loss_and_grad(roam, r, Fn, wt, room32, rays, target, roam.ROAM_F32)
    cams = F.camera_array(room32.cams)
    gmax = np.abs(g).max()
    rng = np.random.default_rng(34)
    hit = np.nonzero(np.abs(g).sum(axis=1) > 0)[0]
    P = w.shape[1]
    h = 1e-4
    checked = 0
    for _ in range(64):
        f, k = int(rng.choice(hit)), int(rng.integers(P))
        wp, wm = w.copy(), w.copy()
        wp[f, k] = np.float32(w[f, k] + h)
        wm[f, k] = np.float32(w[f, k] - h)
        args = (room32.affine, room32.W, room32.H, room32.sigma_scale, cams, rays, target, room32.delta, room32.n_max)
        lp, _, sp, _ = O.loss_grad(room32_grid, wp, *args, want_grad=False)
        lm, _, sm, _ = O.loss_grad(room32_grid, wm, *args, want_grad=False)
        _, _, s0, _ = O.loss_grad(room32_grid, w, *args, want_grad=False)
        if sp != s0 or sm != s0:
            continue
        fd = (lp - lm) / (float(wp[f, k]) - float(wm[f, k]))
        assert abs(fd - g[f, k]) <= 1e-3 * gmax + 1e-3 * abs(fd), (f, k, fd, g[f, k], gmax)
        checked += 1
        if checked == 16:
            break
    assert checked == 16
    r.close()


def test_autograd_forward_follows_the_weight_tensor(roam, room32):
    """After an in-place update of the weight tensor (an SGD step under
    no_grad, as torch.optim makes it) the next forward renders with the new
    values: bit-identical to a fresh context loaded with them."""
    w = F.xavier_weights(5, F.ROLE_STUDENT, room32.part.n_fields, room32.W, room32.H, bias_scale=0.1)
    r = _setup(roam, room32, w)
    Fn = roam.render_function()
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    rays, target = _batch(room32, 512, 35)
    opts = roam.render_opts(room32.delta, room32.n_max)
    rays_t = torch.from_numpy(rays.astype(np.int32)).cuda()
    rgb0 = Fn.apply(wt, r, room32.cams, rays_t, opts)
    ((rgb0 - torch.from_numpy(target).cuda()) ** 2).mean().backward()
    opt = torch.optim.SGD([wt], lr=50.0)
    opt.step()
    rgb1 = Fn.apply(wt, r, room32.cams, rays_t, opts).detach().clone()
    r2 = _setup(roam, room32, wt.detach().cpu().numpy())
    ref = r2.train_forward(room32.cams, rays_t, opts)
    torch.cuda.synchronize()
    assert not torch.equal(rgb0.detach(), rgb1)
    assert torch.equal(rgb1, ref)
    # the library's own copy of the masters is the tensor's
    assert torch.equal(r.get_weights(), wt.detach())
    r2.close()
    r.close()


def test_autograd_stale_backward_raises(roam, room32):
    w = F.xavier_weights(6, F.ROLE_STUDENT, room32.part.n_fields, room32.W, room32.H, bias_scale=0.1)
    r = _setup(roam, room32, w)
    Fn = roam.render_function()
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    rays, target = _batch(room32, 256, 36)
    rays_t = torch.from_numpy(rays.astype(np.int32)).cuda()
    opts = roam.render_opts(room32.delta, room32.n_max)
    first = Fn.apply(wt, r, room32.cams, rays_t, opts)
    second = Fn.apply(wt, r, room32.cams, rays_t[:128], opts)
    with pytest.raises(RuntimeError):
        first.sum().backward()
    second.sum().backward()          # the live forward's backward still works
    torch.cuda.synchronize()
    assert wt.grad is not None and torch.isfinite(wt.grad).all()
    r.close()

"""Helpers of the GPU parity tests: the library's own kept-sample lists for
a set of rays (roam_march with the render's options gives exactly the
samples roam_render composites), and the checks of the render parity rule
(``oracle.parity``) with the bars the tests use."""
import numpy as np

import oracle.parity as P


def records(ctx, cams, opts, rays_np=None):
    """(count [n], recs [n, n_max]) of the library's march of these rays
    (None: every pixel of every view) under the render options `opts`."""
    import torch
    rays_t = torch.from_numpy(np.ascontiguousarray(rays_np).astype(np.int32)).cuda() if rays_np is not None else None
    cnt, recs = ctx.march(cams, opts, rays=rays_t)
    torch.cuda.synchronize()
    return cnt.cpu().numpy(), recs.cpu().numpy()


def assert_march(rep, n_rays: int):
    """Every mismatch certified, and certified mismatches under 0.1% of rays."""
    assert not rep.uncertified, f"uncertified march mismatches at rays {rep.uncertified[:10]}"
    assert len(rep.certified) <= 0.001 * n_rays, (len(rep.certified), n_rays)


def assert_render(rep, psnr_min=None, got=None, depth_tol=None, opacity_tol=None):
    """The march rule above, every ray's colour within its bar, and (BF16)
    the PSNR over all rays against the references the rule assigns."""
    assert_march(rep, rep.n)
    over = rep.over
    assert over.size == 0, (rep.summary(), over[:10], rep.err[over[:10]])
    if psnr_min is not None:
        assert rep.psnr(got) >= psnr_min, (rep.psnr(got), rep.summary())
    if depth_tol is not None and rep.err_depth is not None:
        assert rep.err_depth.max() <= depth_tol, rep.err_depth.max()
    if opacity_tol is not None and rep.err_opacity is not None:
        assert rep.err_opacity.max() <= opacity_tol, rep.err_opacity.max()

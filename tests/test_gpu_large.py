"""The 512^3 twenty-room floor at its full size, in the launch
configuration the benchmark times: 4096 kd fields of W=128/H=4 MLPs, one
2048x1024 equirectangular view, <= 192 samples per ray.  Sampled pixels
against the FP64 oracle: BF16 >= 40 dB PSNR and <= 2e-2 max abs; FP8
against the oracle's FP8 reading by the same bars (and within 0.1 of the
FP64 colours), every ray under the render parity rule (oracle.parity)."""
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


def _psnr(a, b):
    mse = float(((a - b) ** 2).mean())
    return 10 * np.log10(1.0 / mse) if mse > 0 else np.inf


def test_floor512_bf16_and_fp8_sampled(roam):
    wl = F.floor512()
    r = roam.Roam(0)
    r.load_workload(wl)
    rng = np.random.default_rng(71)
    n_pix = wl.cams[0].n_pixels
    rays = np.stack([np.zeros(1500, dtype=np.int64), rng.integers(0, n_pix, 1500)], 1).astype(np.uint32)
    g = O.Grid(wl.scene, wl.part)
    cams = F.camera_array(wl.cams)
    ref = O.render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, rays, wl.delta, wl.n_max)
    ref8 = O.render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, rays, wl.delta, wl.n_max, quant=1)
    gi = rays[:, 1].astype(np.int64)
    for prec, rr, quant in ((roam.ROAM_BF16, ref, 0), (roam.ROAM_FP8, ref8, 1)):
        opts = roam.render_opts(wl.delta, wl.n_max, precision=prec)
        rgb, _, _ = r.render(wl.cams, opts)
        torch.cuda.synchronize()
        r.check()
        got = rgb.cpu().numpy()[gi].astype(np.float64)
        cnt, recs = records(r, wl.cams, opts, rays)
        rep = P.check_render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, rays, wl.delta, wl.n_max,
                             cnt, recs, got, tol=2e-2, quant=quant, ref=rr)
        assert_render(rep, psnr_min=40.0, got=got)
        if prec == roam.ROAM_FP8:
            rep64 = P.check_render(g, wl.weights, wl.affine, wl.W, wl.H, wl.sigma_scale, cams, rays, wl.delta,
                                   wl.n_max, cnt, recs, got, tol=0.1, ref=ref)
            assert rep64.over.size == 0, rep64.summary()
    st = r.get_stats()
    assert st.n_rounds >= 1 and st.n_used > 0
    r.close()

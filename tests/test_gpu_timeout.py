"""The bounded device-side waits of the tensor-core MLP kernel: a launch whose
weight-image copy is withheld (roam_selftest_wait_timeout) must give up after
the requested limit, surface ROAM_ERR_TIMEOUT to the host, free its tensor
memory and return -- the context, and the GPU, keep working: the next
renders use the tensor memory again and give the same bits as before."""
import time

import numpy as np
import pytest

import fixtures as F

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def roam():
    import paper_2208_02705_gb300 as roam
    from paper_2208_02705_gb300 import build
    build.build()
    return roam


@pytest.mark.parametrize("W,H", [(32, 2), (64, 3), (128, 2)])
def test_wait_timeout_is_reported_and_the_context_stays_usable(roam, room32, W, H):
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.1)
    r = roam.Roam(0)
    r.load_grid(room32.scene.bits, room32.scene.dims, room32.scene.origin, room32.scene.vox)
    r.load_fields(room32.part.field_of_rank, room32.affine)
    r.load_weights(w, W, H, room32.sigma_scale)
    opts = roam.render_opts(room32.delta, room32.n_max, precision=roam.ROAM_BF16)
    ref = [x.clone() for x in r.render(room32.cams, opts)]
    torch.cuda.synchronize()
    r.check()
    limit = 50_000_000                         # 50 ms
    t0 = time.perf_counter()
    status = r.selftest_wait_timeout(limit)
    dt = time.perf_counter() - t0
    assert status == -5, status                # ROAM_ERR_TIMEOUT
    assert 0.05 <= dt < 1.0, dt                # it waited about the limit, not the 2 s default
    r.check()                                  # the flag does not outlive the self-test
    for _ in range(3):                         # TMEM was freed: the kernels allocate it again
        out = r.render(room32.cams, opts)
        torch.cuda.synchronize()
        for a, b in zip(ref, out):
            assert torch.equal(a, b)
    r.check()
    with pytest.raises(roam.RoamError):
        r.selftest_wait_timeout(10)            # below the allowed range
    r.close()

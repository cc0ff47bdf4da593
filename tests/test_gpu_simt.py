"""Parity of the FP32 SIMT MLP path with the FP64 oracle, over every
supported shape (both forms of the kernel: the field's weights in shared
memory for W <= 64, through the read-only path for W = 128) and over tile
layouts that exercise the per-block runs of one field: one long run that
crosses block boundaries, single-sample fields, and fewer tiles than
blocks.

Bars (FP32 arithmetic against the FP64 definition): colours within 2e-5;
density within 1e-4 of max(1, sigma) -- FP32 rounding of the field-local
coordinate (6e-8 relative) is amplified by the 2^9 pi encoding frequency
to ~1e-4 in the features, and sigma carries sigma_scale on top."""
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


def _points(wl, f, rng):
    boxes = wl.part.boxes
    lo = boxes[f, 0, :] * wl.scene.vox
    hi = boxes[f, 1, :] * wl.scene.vox
    p = lo + rng.uniform(0, 1, (len(f), 3)) * (hi - lo)
    d = rng.normal(size=(len(f), 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return p.astype(np.float32), d.astype(np.float32)


def _eval_and_check(roam, wl, W, H, f, seed, check=None):
    """Evaluates every point on the GPU; compares the points `check` (all by
    default) with the oracle."""
    w = F.xavier_weights(1, F.ROLE_STUDENT, wl.part.n_fields, W, H, bias_scale=0.3)
    r = roam.Roam(0)
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    r.load_fields(wl.part.field_of_rank, wl.affine)
    r.load_weights(w, W, H, wl.sigma_scale)
    rng = np.random.default_rng(seed)
    p, d = _points(wl, f, rng)
    out = r.mlp_eval(torch.from_numpy(p).cuda(), torch.from_numpy(d).cuda(),
                     torch.from_numpy(f.astype(np.int16)).cuda(), roam.ROAM_F32)
    torch.cuda.synchronize()
    r.check()
    out = out.cpu().numpy().astype(np.float64)
    r.close()
    assert np.all(np.isfinite(out))
    idx = np.arange(len(f)) if check is None else check
    out = out[idx]
    ref = np.array([O.mlp(w[f[i]], W, H, wl.sigma_scale, wl.affine[f[i]], p[i].astype(np.float64),
                          d[i].astype(np.float64)) for i in idx])
    err_c = np.abs(out[:, 1:] - ref[:, 1:]).max()
    err_s = (np.abs(out[:, 0] - ref[:, 0]) / np.maximum(1.0, ref[:, 0])).max()
    assert err_c <= 2e-5, (W, H, err_c)
    assert err_s <= 1e-4, (W, H, err_s)


@pytest.mark.parametrize("W", [32, 64, 128])
@pytest.mark.parametrize("H", [1, 2, 3, 4])
def test_simt_every_shape_matches_oracle(roam, room32, W, H):
    rng = np.random.default_rng(100 * W + H)
    n = 700 if W == 128 else 900
    f = rng.integers(0, room32.part.n_fields, n).astype(np.uint16)
    _eval_and_check(roam, room32, W, H, f, W + H)


@pytest.mark.parametrize("W,H", [(64, 3), (32, 2), (128, 2)])
def test_simt_long_run_beside_single_samples(roam, room32, W, H):
    """One field with 300 tiles (more tiles than blocks: its run starts in
    one block's tile range and ends in another's), one field with a partial
    second tile, the others one sample each (a partial tile per field);
    every point is evaluated, the short fields' points and 2500 of the long
    field's are checked."""
    n_f = room32.part.n_fields
    long_f, two_f = n_f // 2, n_f // 2 + 1
    f = np.concatenate([np.full(300 * 128 + 77, long_f), np.full(130, two_f),
                        [k for k in range(n_f) if k not in (long_f, two_f)]]).astype(np.uint16)
    rng = np.random.default_rng(3)
    rng.shuffle(f)
    short = np.nonzero(f != long_f)[0]
    sample = rng.choice(np.nonzero(f == long_f)[0], 2500, replace=False)
    _eval_and_check(roam, room32, W, H, f, 7, check=np.concatenate([short, sample]))


def test_simt_fewer_tiles_than_blocks(roam, room32):
    """Three samples of three fields: most blocks get no tile at all."""
    f = np.array([0, room32.part.n_fields - 1, 1], dtype=np.uint16)
    _eval_and_check(roam, room32, 64, 3, f, 11)

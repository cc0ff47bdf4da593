"""Fields of mixed MLP widths (32/64/128 drawn per field) through the C ABI,
and the batched multi-view render (many cameras of different models and
sizes in one call, with and without CUDA-graph replay).

Internally the library groups the fields by width (a permutation of the
field ids) and runs one MLP kernel per width over that width's tiles; every
field id seen through the ABI stays the caller's, which the march records
and roam_mlp_eval keys check.  Colour bars as for one width, on every ray
under the render parity rule (oracle.parity): FP32 <= 1e-4, BF16 >= 40 dB
and <= 2e-2, FP8 >= 40 dB and <= 2e-2 against the oracle's FP8 reading."""
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


H_MIX = 3


@pytest.fixture(scope="module")
def mixed(room32):
    widths = F.mixed_widths(1, room32.part.n_fields)
    w = F.xavier_weights_mixed(1, F.ROLE_STUDENT, widths, H_MIX, bias_scale=0.1)
    return widths, w


@pytest.fixture(scope="module")
def mixed_ctx(roam, room32, mixed):
    widths, w = mixed
    r = roam.Roam(0)
    r.load_grid(room32.scene.bits, room32.scene.dims, room32.scene.origin, room32.scene.vox)
    r.load_fields(room32.part.field_of_rank, room32.affine)
    r.load_weights_mixed(w, widths, H_MIX, room32.sigma_scale)
    yield r
    r.close()


def _psnr(a, b):
    mse = float(((a - b) ** 2).mean())
    return 10 * math.log10(1.0 / mse) if mse > 0 else float("inf")


def test_mixed_widths_are_mixed(mixed):
    widths, _ = mixed
    assert set(widths.tolist()) == {32, 64, 128}


@pytest.mark.parametrize("precision", ["f32", "bf16", "fp8"])
def test_render_room32_mixed_widths(roam, room32, room32_grid, mixed, mixed_ctx, precision):
    widths, w = mixed
    prec = {"f32": roam.ROAM_F32, "bf16": roam.ROAM_BF16, "fp8": roam.ROAM_FP8}[precision]
    opts = roam.render_opts(room32.delta, room32.n_max, precision=prec)
    rgb, _, _ = mixed_ctx.render(room32.cams, opts)
    torch.cuda.synchronize()
    mixed_ctx.check()
    cnt, recs = records(mixed_ctx, room32.cams, opts)
    got = rgb.cpu().numpy().astype(np.float64)
    rep = P.check_render(room32_grid, w, room32.affine, 0, H_MIX, room32.sigma_scale, F.camera_array(room32.cams),
                         None, room32.delta, room32.n_max, cnt, recs, got, tol=1e-4 if precision == "f32" else 2e-2,
                         widths=widths, quant=1 if precision == "fp8" else 0)
    assert_render(rep, psnr_min=None if precision == "f32" else 40.0, got=got)


def test_mlp_eval_mixed_widths_takes_callers_field_ids(roam, room32, mixed, mixed_ctx):
    widths, w = mixed
    offs = np.concatenate([[0], np.cumsum([F.n_params(int(W), H_MIX) for W in widths])])
    rng = np.random.default_rng(44)
    n = 1000
    f = rng.integers(0, room32.part.n_fields, n)
    boxes = room32.part.boxes
    p = (boxes[f, 0, :] + rng.uniform(0, 1, (n, 3)) * (boxes[f, 1, :] - boxes[f, 0, :])) * room32.scene.vox
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p, d = p.astype(np.float32), d.astype(np.float32)
    args = (torch.from_numpy(p).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(f.astype(np.int16)).cuda())
    out32 = mixed_ctx.mlp_eval(*args, roam.ROAM_F32).cpu().numpy()
    out16 = mixed_ctx.mlp_eval(*args, roam.ROAM_BF16).cpu().numpy()
    ref = np.array([O.mlp(w[offs[f[i]]:offs[f[i] + 1]], int(widths[f[i]]), H_MIX, room32.sigma_scale,
                          room32.affine[f[i]], p[i].astype(np.float64), d[i].astype(np.float64)) for i in range(n)])
    assert np.abs(out32[:, 1:] - ref[:, 1:]).max() <= 1e-4
    assert np.all(np.abs(out32[:, 0] - ref[:, 0]) <= 1e-4 * np.maximum(1.0, ref[:, 0]))
    assert np.abs(out16[:, 1:] - ref[:, 1:]).max() <= 2e-2


def test_march_records_keep_callers_field_ids(roam, room32, room32_grid, mixed_ctx):
    opts = roam.render_opts(room32.delta, room32.n_max)
    cnt, recs = records(mixed_ctx, room32.cams, opts)
    _, rep, _ = P.check_march(room32_grid, F.camera_array(room32.cams), None, room32.delta, room32.n_max, cnt, recs)
    assert_march(rep, rep.n)
    assert rep.n_equal > 0.99 * rep.n


def test_get_weights_round_trip_mixed(mixed, mixed_ctx):
    _, w = mixed
    got = mixed_ctx.get_weights().cpu().numpy()
    assert np.array_equal(got, w)


def test_single_width_reload_restores_field_order(roam, room32, room32_grid):
    """Mixed, then one width again: labels and affines return to the
    caller's order (the render equals a fresh context's)."""
    r = roam.Roam(0)
    r.load_workload(room32)
    opts = roam.render_opts(room32.delta, room32.n_max)
    fresh, _, _ = r.render(room32.cams, opts)
    fresh = fresh.clone()
    widths = F.mixed_widths(1, room32.part.n_fields)
    r.load_weights_mixed(F.xavier_weights_mixed(1, 2, widths, 2), widths, 2, room32.sigma_scale)
    r.render(room32.cams, opts)
    r.load_weights(room32.weights, room32.W, room32.H, room32.sigma_scale)
    again, _, _ = r.render(room32.cams, opts)
    torch.cuda.synchronize()
    assert torch.equal(fresh, again)
    r.close()


def test_training_refuses_mixed_widths(roam, room32, mixed_ctx):
    rays = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(roam.RoamError) as e:
        mixed_ctx.train_forward(room32.cams, rays, roam.render_opts(room32.delta, room32.n_max))
    assert e.value.status == -7


def test_multiview_batched_render_matches_oracle_and_graph(roam):
    """The 384^3 mixed-width floor with 8 of its views (both camera models,
    four sizes) in one call: sampled pixels against the oracle; the
    graph-replayed batch, and the views rendered one call each, give the
    same bits as the plain batched call."""
    specs = F.multiview_specs()[:8]
    wl = F.floor384(specs=specs)
    g = O.Grid(wl.scene, wl.part)
    r = roam.Roam(0)
    r.load_workload(wl)
    opts = roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16)
    rgb, _, _ = r.render(wl.cams, opts)
    rgb = rgb.clone()
    gopts = roam.render_opts(wl.delta, wl.n_max, precision=roam.ROAM_BF16, use_graph=True)
    for _ in range(2):
        rgb_g, _, _ = r.render(wl.cams, gopts)
    per = [r.render([c], opts)[0].clone() for c in wl.cams]
    torch.cuda.synchronize()
    r.check()
    assert torch.equal(rgb, rgb_g)
    assert torch.equal(rgb, torch.cat(per))
    rng = np.random.default_rng(384)
    sizes = [c.n_pixels for c in wl.cams]
    starts = np.concatenate([[0], np.cumsum(sizes)])
    view = rng.integers(0, len(sizes), 3000)
    pix = np.array([rng.integers(0, sizes[v]) for v in view])
    rays = np.stack([view, pix], 1).astype(np.uint32)
    cnt, recs = records(r, wl.cams, opts, rays)
    got = rgb.cpu().numpy()[starts[view] + pix].astype(np.float64)
    rep = P.check_render(g, wl.weights, wl.affine, 0, wl.H, wl.sigma_scale, F.camera_array(wl.cams), rays, wl.delta,
                         wl.n_max, cnt, recs, got, tol=2e-2, widths=wl.widths)
    assert_render(rep, psnr_min=40.0, got=got)
    r.close()

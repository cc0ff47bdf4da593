"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics (closed forms, special values, brute force, invariants), chosen so
that a dropped term, a wrong sign or index, or a transposed operand anywhere
in the oracle fails at least one of them.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import fixtures as F
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def cam16(model=0, W=64, H=32, fov=0.0, R=None, o=(0.0, 0.0, 0.0)):
    R = np.eye(3) if R is None else np.asarray(R)
    return np.concatenate([[model, W, H, fov], R.reshape(9), o]).astype(np.float64)


# ----------------------------------------------------------------------------
# parameter counts (Appendix, network architecture details)
# ----------------------------------------------------------------------------

def test_param_count_matches_paper():
    g = json.load(open(GOLDEN))
    assert O.param_count(32, 2) == g["tiny_mlp_params"]["value"] == 6212
    # 200 tiny networks ~ 1.2M parameters (ablation on the number of networks)
    total = 200 * O.param_count(32, 2)
    assert abs(total - g["n200_total_params_approx"]["value"]) / 1.2e6 < 0.05
    # the larger widths used by the workloads
    assert O.param_count(64, 3) == 22724
    assert O.param_count(128, 4) == 94724
    assert F.n_params(32, 2) == 6212 and F.n_params(64, 3) == 22724


# ----------------------------------------------------------------------------
# ray generation (Eq. 2, Eq. 3)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("uc,vc,expect", [
    (32.0, 16.0, (0.0, 0.0, 1.0)),      # image centre: phi = 0, theta = 0
    (48.0, 16.0, (1.0, 0.0, 0.0)),      # u = 3W/4: phi = +pi/2
    (16.0, 16.0, (-1.0, 0.0, 0.0)),     # u = W/4: phi = -pi/2
    (0.0, 16.0, (0.0, 0.0, -1.0)),      # left edge: phi = -pi
    (32.0, 0.0, (0.0, -1.0, 0.0)),      # top edge: theta = +pi/2, y = -sin(theta)
    (32.0, 32.0, (0.0, 1.0, 0.0)),      # bottom edge: theta = -pi/2
])
def test_equirect_special_pixels(uc, vc, expect):
    o, d = O.ray(cam16(), uc, vc)
    assert np.allclose(d, expect, atol=1e-12)
    assert np.allclose(o, 0.0)


def test_equirect_round_trip_through_eq2():
    rng = np.random.default_rng(7)
    W, H = 128, 64
    for _ in range(200):
        uc, vc = rng.uniform(0.01, W - 0.01), rng.uniform(0.01, H - 0.01)
        _, d = O.ray(cam16(W=W, H=H), uc, vc)
        assert abs(np.linalg.norm(d) - 1.0) < 1e-13
        # invert Eq. 3, then apply Eq. 2 forwards
        phi = math.atan2(d[0], d[2])
        theta = math.asin(-d[1])
        u = phi * W / (2 * math.pi) + W / 2
        v = -theta * H / math.pi + H / 2
        assert abs(u - uc) < 1e-9 and abs(v - vc) < 1e-9


def test_camera_rotation_and_origin():
    R = F.yaw_pitch(0.7, 0.2)
    o = np.array([1.0, 2.0, 3.0])
    rng = np.random.default_rng(3)
    for _ in range(20):
        uc, vc = rng.uniform(0, 64), rng.uniform(0, 32)
        _, d0 = O.ray(cam16(), uc, vc)
        oo, d1 = O.ray(cam16(R=R, o=o), uc, vc)
        assert np.allclose(oo, o)
        assert np.allclose(R.T @ d1, d0, atol=1e-13)


def test_perspective_pixels():
    W, H, fov = 200, 100, math.pi / 2
    _, d = O.ray(cam16(1, W, H, fov), W / 2, H / 2)
    assert np.allclose(d, (0, 0, 1), atol=1e-14)
    # the right edge of a 90 degree view is 45 degrees off axis
    _, d = O.ray(cam16(1, W, H, fov), W, H / 2)
    assert np.allclose(d, (math.sqrt(0.5), 0, math.sqrt(0.5)), atol=1e-14)
    # rows grow downwards (+y), and pixels are square
    _, d = O.ray(cam16(1, W, H, fov), W / 2, H)
    assert np.allclose(d, np.array([0, 0.5, 1]) / math.sqrt(1.25), atol=1e-14)


# ----------------------------------------------------------------------------
# labels: rank order versus brute-force point-in-box
# ----------------------------------------------------------------------------

def test_label_map_matches_partition_boxes(room32, room32_grid):
    occ = room32.scene.occ
    lab = room32_grid.label.reshape(occ.shape)
    assert room32_grid.n_occupied == occ.sum()
    assert ((lab >= 0) == occ).all()
    z, y, x = np.nonzero(occ)
    for xx, yy, zz in zip(x, y, z):
        inside = [f for f, (lo, hi) in enumerate(room32.part.boxes)
                  if lo[0] <= xx < hi[0] and lo[1] <= yy < hi[1] and lo[2] <= zz < hi[2]]
        assert len(inside) == 1
        assert lab[zz, yy, xx] == inside[0]


def test_label_map_kd_partition_brute_force():
    """A 64^3 floor with a 16-leaf kd partition: every occupied voxel lies in
    exactly one leaf box and the oracle's rank lookup returns that leaf."""
    scene = F.floor_scene(9, 64, 2, 2, 0.1)
    part = F.kd_partition(scene, 16)
    g = O.Grid(scene, part)
    lab = g.label.reshape(scene.occ.shape)
    z, y, x = np.nonzero(scene.occ)
    xyz = np.stack([x, y, z], 1)
    hits = np.zeros(xyz.shape[0], dtype=np.int64)
    expect = np.full(xyz.shape[0], -1)
    for f, (lo, hi) in enumerate(part.boxes):
        inside = np.all((xyz >= lo) & (xyz < hi), axis=1)
        hits += inside
        expect[inside] = f
    assert (hits == 1).all()
    assert (lab[z, y, x] == expect).all()
    assert (lab[~scene.occ] == -1).all()


# ----------------------------------------------------------------------------
# marching: analytic chord counts, empty and full grids
# ----------------------------------------------------------------------------

class _Scene:
    def __init__(self, occ, vox=0.1):
        self.dims = (occ.shape[2], occ.shape[1], occ.shape[0])
        self.origin = (0.0, 0.0, 0.0)
        self.vox = vox
        self.occ = occ
        self.bits = F.pack_bits(occ)


class _Part:
    def __init__(self, n):
        self.field_of_rank = np.zeros(n, dtype=np.uint16)


def _grid(occ, vox=0.1):
    s = _Scene(occ, vox)
    return O.Grid(s, _Part(int(occ.sum())))


def _slab_interval(o, d, lo, hi):
    t0, t1 = -np.inf, np.inf
    for a in range(3):
        ta, tb = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return t0, t1


def test_march_single_voxel_chord_count():
    rng = np.random.default_rng(11)
    G, vox = 32, 0.1
    delta = O.f32(vox / 4)
    checked = 0
    for trial in range(300):
        occ = np.zeros((G, G, G), dtype=bool)
        iv = rng.integers(4, 28, size=3)
        occ[iv[2], iv[1], iv[0]] = True
        g = _grid(occ, vox)
        o = rng.uniform(0.2, 3.0, size=3)
        target = (iv + rng.uniform(0.1, 0.9, size=3)) * O.f32(vox)
        d = target - o
        d /= np.linalg.norm(d)
        lo, hi = iv * g.vox, (iv + 1) * g.vox
        t0, t1 = _slab_interval(o, d, lo, hi)
        t0 = max(t0, 0.0)
        # count j with t0 <= (j + 1/2) delta < t1; skip grazing cases
        js = np.arange(0, int(t1 / delta) + 3)
        tj = (js + 0.5) * delta
        if np.min(np.abs(np.concatenate([tj - t0, tj - t1]))) < 1e-9:
            continue
        expect = js[(tj >= t0) & (tj < t1)]
        got, fields, _ = O.march(g, o, d, delta, 64)
        assert np.array_equal(got, expect), (trial, got, expect)
        assert (fields == 0).all()
        checked += 1
    assert checked > 250


def test_march_empty_and_full_grids():
    G, vox = 32, 0.1
    delta = O.f32(vox / 4)
    o = np.array([1.55, 1.62, 1.48])
    rng = np.random.default_rng(5)
    g_empty = _grid(np.zeros((G, G, G), dtype=bool), vox)
    g_full = _grid(np.ones((G, G, G), dtype=bool), vox)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        js, _, _ = O.march(g_empty, o, d, delta, 1024)
        assert js.size == 0
        # full grid: every j whose point is before the exit of the box
        t0, t1 = _slab_interval(o, d, np.zeros(3), np.full(3, G * g_full.vox))
        js, _, _ = O.march(g_full, o, d, delta, 1024)
        expect = np.arange(0, int(np.ceil(t1 / delta - 0.5)))
        assert np.array_equal(js, expect)
        js_cap, _, _ = O.march(g_full, o, d, delta, 17)
        assert np.array_equal(js_cap, expect[:17])


def test_march_fields_match_boxes(room32, room32_grid):
    """Kept samples of real rays: the field of every sample is the partition
    box containing its point (brute force over all boxes)."""
    cams = O.cams_f32(F.camera_array(room32.cams))
    vox = room32_grid.vox
    rng = np.random.default_rng(2)
    for _ in range(200):
        uc, vc = rng.uniform(0, 128), rng.uniform(0, 64)
        o, d = O.ray(cams[0], uc, vc)
        js, fs, ties = O.march(room32_grid, o, d, room32.delta, 64)
        for j, f in zip(js, fs):
            p = o + (j + 0.5) * O.f32(room32.delta) * d
            iv = np.floor(p / vox).astype(int)
            assert room32.scene.occ[iv[2], iv[1], iv[0]]
            boxes = [k for k, (lo, hi) in enumerate(room32.part.boxes) if np.all(iv >= lo) and np.all(iv < hi)]
            assert boxes == [f]


# ----------------------------------------------------------------------------
# positional encoding and the tiny MLP
# ----------------------------------------------------------------------------

S2, S3 = math.sqrt(2.0) / 2, math.sqrt(3.0) / 2


def test_encoding_special_values():
    # x = (1/6, 1/4, 1/2): exact trigonometric values for pi x, 2 pi x, 4 pi x
    x = np.array([1.0 / 6, 0.25, 0.5])
    e = O.encode(x, 3)
    assert e.shape == (21,)
    assert np.allclose(e[0:3], x, atol=0)
    # k = 0: sin(pi/6, pi/4, pi/2), cos(...)
    assert np.allclose(e[3:6], [0.5, S2, 1.0], atol=1e-15)
    assert np.allclose(e[6:9], [S3, S2, 0.0], atol=1e-15)
    # k = 1: angles pi/3, pi/2, pi
    assert np.allclose(e[9:12], [S3, 1.0, 0.0], atol=1e-15)
    assert np.allclose(e[12:15], [0.5, 0.0, -1.0], atol=1e-15)
    # k = 2: angles 2pi/3, pi, 2pi
    assert np.allclose(e[15:18], [S3, 0.0, 0.0], atol=1e-14)
    assert np.allclose(e[18:21], [-0.5, -1.0, 1.0], atol=1e-14)
    assert O.encode(x, 10).shape == (63,) and O.encode(x, 4).shape == (27,)


def _offsets(W, H):
    offs, o = [], 0
    for (n_out, n_in) in F.layer_shapes(W, H):
        offs.append((o, o + n_out * n_in, n_out, n_in))
        o += n_out * n_in + n_out
    return offs, o


def test_mlp_zero_weights_closed_form():
    W, H = 16, 3
    offs, P = _offsets(W, H)
    rng = np.random.default_rng(1)
    w = np.zeros(P, dtype=np.float32)
    for (wo, bo, n_out, _) in offs:
        w[bo:bo + n_out] = rng.uniform(-1, 1, n_out)
    b_head = w[offs[H][1]:offs[H][1] + 1 + W]
    b_out = w[offs[H + 2][1]:offs[H + 2][1] + 3]
    aff = np.array([1, 1, 1, 0, 0, 0], dtype=np.float32)
    for _ in range(5):
        p, d = rng.uniform(-1, 1, 3), rng.normal(size=3)
        out = O.mlp(w, W, H, 2.5, aff, p, d)
        s = float(b_head[0])
        assert abs(out[0] - O.f32(2.5) * math.log(1 + math.exp(s))) < 1e-12
        assert np.allclose(out[1:], 1 / (1 + np.exp(-b_out.astype(np.float64))), atol=1e-15)


@pytest.mark.parametrize("m,mp,xl,dv,pe_m,pe_dm", [
    # index m of F(x_loc) (L = 10) and m' of F(d) (L = 4), with their values
    # known exactly from trigonometry:
    #  m=4: sin(pi x1), x1=1/4 -> sqrt(2)/2;     m'=10: sin(2 pi d1), d1=1/4 -> 1
    (4, 10, (1 / 6, 0.25, 0.5), (0.5, 0.25, 1 / 6), S2, 1.0),
    #  m=1: raw x1 = -0.7;                         m'=0: raw d0 = 0.6
    (1, 0, (0.3, -0.7, 0.1), (0.6, 0.0, 0.8), -0.7, 0.6),
    #  m=8: cos(pi x2), x2=-1/3 -> 1/2;            m'=26: cos(8 pi d2), d2=1/24 -> 1/2
    (8, 26, (0.2, 0.4, -1 / 3), (0.0, 1.0, 1 / 24), 0.5, 0.5),
    #  m=62: cos(512 pi x2), x2=1/1536 -> 1/2;     m'=13: cos(2 pi d1), d1=1/6 -> 1/2
    (62, 13, (0.1, 0.2, 1 / 1536), (0.3, 1 / 6, 0.2), 0.5, 0.5),
])
def test_mlp_one_hot_closed_form(m, mp, xl, dv, pe_m, pe_dm):
    """Weights that route one encoded feature through every layer: the
    density sees relu(F(x)[m]); the green channel sees
    relu(relu(F(x)[m]) + F(d)[m']).  Asymmetric row/column choices catch a
    transposed operand, a shifted layer offset or a misplaced encoding index."""
    W, H = 8, 2
    offs, P = _offsets(W, H)
    w = np.zeros(P, dtype=np.float32)
    l1, l2, head, col, out = offs
    w[l1[0] + 0 * 63 + m] = 1.0              # h1[0] = relu(F(x)[m])
    w[l2[0] + 0 * W + 0] = 1.0               # h2[0] = h1[0]
    w[head[0] + 0 * W + 0] = 1.0             # s = h2[0]
    w[head[0] + (1 + 2) * W + 0] = 1.0       # feat[2] = h2[0]
    Kc = W + 27
    w[col[0] + 5 * Kc + 2] = 1.0             # g[5] = relu(feat[2] + F(d)[m'])
    w[col[0] + 5 * Kc + W + mp] = 1.0
    w[out[0] + 1 * W + 5] = 1.0              # green = sigmoid(g[5])
    w[out[1] + 2] = 0.75                     # blue bias
    aff = np.array([1, 1, 1, 0, 0, 0], dtype=np.float32)
    got = O.mlp(w, W, H, 1.0, aff, np.array(xl, dtype=np.float64), np.array(dv, dtype=np.float64))
    relu = lambda v: max(v, 0.0)
    assert abs(got[0] - math.log1p(math.exp(relu(pe_m)))) < 1e-12
    assert abs(got[1] - 0.5) < 1e-15
    g5 = relu(relu(pe_m) + pe_dm)
    assert abs(got[2] - 1 / (1 + math.exp(-g5))) < 1e-12
    assert abs(got[3] - 1 / (1 + math.exp(-0.75))) < 1e-12


def test_mlp_affine_maps_field_box():
    """x_loc = scale * p + offset: a point at the box centre encodes as 0."""
    W, H = 8, 2
    offs, P = _offsets(W, H)
    w = np.zeros(P, dtype=np.float32)
    w[offs[0][0] + 0 * 63 + 0] = 1.0   # h1[0] = relu(x_loc[0])
    w[offs[1][0]] = 1.0
    w[offs[2][0]] = 1.0                # s = relu(x_loc[0])
    scale = np.array([4.0, 2.0, 1.0]); off = np.array([-3.0, 0.5, 0.0])
    aff = np.concatenate([scale, off]).astype(np.float32)
    for px in (0.5, 0.75, 1.0, 0.9):
        p = np.array([px, 0.0, 0.0])
        got = O.mlp(w, W, H, 1.0, aff, p, np.array([0, 0, 1.0]))
        xl0 = 4.0 * px - 3.0
        assert abs(got[0] - math.log1p(math.exp(max(xl0, 0.0)))) < 1e-12


# ----------------------------------------------------------------------------
# the FP8 E4M3 reading of the matrix layers (a precision choice of the
# library; the paper fixes no arithmetic format)
# ----------------------------------------------------------------------------

def test_e4m3_hand_values():
    cases = [(1.0625, 1.0), (1.1875, 1.25), (2.0 ** -10, 0.0), (3 * 2.0 ** -11, 2.0 ** -9), (470.0, 448.0),
             (448.0, 448.0), (-0.3, -0.3125), (0.0, 0.0), (2.0 ** -6, 2.0 ** -6), (1.96875, 2.0), (-1e9, -448.0)]
    for x, want in cases:
        assert float(O.e4m3(x)) == want, (x, want)


def test_e4m3_rounding_matches_torch_float8():
    """Every finite E4M3 value, every midpoint between neighbours (ties) and
    random values over the whole range against torch's own conversion."""
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    codes = torch.arange(0, 127, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    mids = 0.5 * (codes[1:] + codes[:-1])
    rng = np.random.default_rng(8)
    logu = np.exp2(rng.uniform(-12, 8.8, 20000)) * rng.choice([-1.0, 1.0], 20000)
    x = np.concatenate([codes, -codes, mids, -mids, logu, rng.uniform(-1, 1, 5000)])
    x = x[np.abs(x) < 464].astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = O.e4m3(x.astype(np.float64))
    assert np.array_equal(got, ref)


def _np_encode(v, L):
    out = [v]
    for k in range(L):
        out += [np.sin(2.0 ** k * math.pi * v), np.cos(2.0 ** k * math.pi * v)]
    return np.concatenate(out)


def _np_mlp_fp8(w, W, H, sig, aff, p, d, quant):
    """The FP8 reading written independently: NumPy matrices, torch's float8
    conversion as the rounding."""
    torch = pytest.importorskip("torch")
    q8 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.float8_e4m3fn) \
        .to(torch.float64).numpy()
    offs, _ = _offsets(W, H)

    def dense(i, x, quantised=True):
        wo, bo, n_out, n_in = offs[i]
        Wm = w[wo:wo + n_out * n_in].reshape(n_out, n_in)
        b = w[bo:bo + n_out].astype(np.float64)
        if not (quant and quantised):
            return b + Wm.astype(np.float64) @ x
        amax = np.abs(Wm).max(axis=1)
        s = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
        Wq = q8((Wm / s[:, None]).astype(np.float32))
        return b + s.astype(np.float64) * (Wq @ q8(x.astype(np.float32)))

    xl = aff[:3].astype(np.float64) * p + aff[3:].astype(np.float64)
    h = np.maximum(dense(0, _np_encode(xl, 10)), 0)
    for k in range(1, H):
        h = np.maximum(dense(k, h), 0)
    z = dense(H, h)
    sigma = O.f32(sig) * np.log1p(np.exp(z[0]))
    g = np.maximum(dense(H + 1, np.concatenate([z[1:], _np_encode(d, 4)])), 0)
    rgb = 1 / (1 + np.exp(-dense(H + 2, g, quantised=False)))
    return np.concatenate([[sigma], rgb])


@pytest.mark.parametrize("W,H", [(16, 2), (32, 3)])
def test_mlp_fp8_reading_matches_independent_chain(W, H):
    rng = np.random.default_rng(W + H)
    w = F.xavier_weights(9, 2, 1, W, H, bias_scale=0.3)[0]
    aff = np.array([1.5, 0.8, 1.1, -0.2, 0.1, 0.05], dtype=np.float32)
    for _ in range(20):
        p = rng.uniform(-0.6, 0.6, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        got = O.mlp(w, W, H, 2.0, aff, p, d, quant=1)
        want = _np_mlp_fp8(w, W, H, 2.0, aff, p, d, True)
        assert np.abs(got - want).max() <= 1e-9
        full = O.mlp(w, W, H, 2.0, aff, p, d)
        assert np.abs(full - _np_mlp_fp8(w, W, H, 2.0, aff, p, d, False)).max() <= 1e-9
        # the rounding is really applied, and stays within a few E4M3 steps
        assert 1e-6 < np.abs(got[1:] - full[1:]).max() < 0.1


def test_mlp_fp8_biases_are_not_rounded():
    """Zero matrices: only the (unrounded) biases reach the outputs, so the
    FP8 reading equals the FP64 one exactly."""
    W, H = 16, 3
    offs, P = _offsets(W, H)
    rng = np.random.default_rng(3)
    w = np.zeros(P, dtype=np.float32)
    for (wo, bo, n_out, _) in offs:
        w[bo:bo + n_out] = rng.uniform(-1, 1, n_out)
    aff = np.array([1, 1, 1, 0, 0, 0], dtype=np.float32)
    p, d = rng.uniform(-1, 1, 3), np.array([0.0, 0.6, 0.8])
    assert np.array_equal(O.mlp(w, W, H, 2.5, aff, p, d, quant=1), O.mlp(w, W, H, 2.5, aff, p, d))


# ----------------------------------------------------------------------------
# compositing (Eq. 4, Eq. 5) with early termination
# ----------------------------------------------------------------------------

def test_composite_two_samples_closed_form():
    a, b, delta = 3.0, 7.0, 0.05
    c0, c1 = np.array([0.2, 0.5, 0.9]), np.array([0.7, 0.1, 0.3])
    bg = np.array([0.1, 0.2, 0.3])
    out, used, _ = O.composite([a, b], np.stack([c0, c1]), [1.0, 2.0], delta, 0.0, bg)
    w0 = 1 - math.exp(-a * delta)
    w1 = math.exp(-a * delta) * (1 - math.exp(-b * delta))
    Tend = math.exp(-(a + b) * delta)
    assert used == 2
    assert np.allclose(out[:3], w0 * c0 + w1 * c1 + Tend * bg, atol=1e-15)
    assert abs(out[3] - (w0 * 1.0 + w1 * 2.0)) < 1e-15
    assert abs(out[4] - (1 - Tend)) < 1e-15


def test_composite_constant_slab_and_sum_of_weights():
    sigma, delta, n = 1.7, 0.01, 80
    rgb = np.tile([0.25, 0.5, 0.75], (n, 1))
    t = (np.arange(n) + 0.5) * delta
    out, used, _ = O.composite(np.full(n, sigma), rgb, t, delta, 0.0)
    ell = n * delta
    assert used == n
    assert abs(out[4] - (1 - math.exp(-sigma * ell))) < 1e-14           # opacity
    assert np.allclose(out[:3], (1 - math.exp(-sigma * ell)) * rgb[0], atol=1e-14)
    # random densities: sum of weights = 1 - T_end <= 1
    rng = np.random.default_rng(0)
    s = rng.uniform(0, 50, 64)
    out, used, _ = O.composite(s, rng.uniform(0, 1, (64, 3)), np.arange(64.0), 0.02, 0.0)
    assert 0 <= out[4] <= 1
    assert abs(out[4] - (1 - math.exp(-s.sum() * 0.02))) < 1e-13


def test_composite_termination_and_truncation_bound():
    rng = np.random.default_rng(4)
    for _ in range(100):
        n = int(rng.integers(1, 60))
        s = rng.uniform(0, 80, n)
        rgb = rng.uniform(0, 1, (n, 3))
        t = np.cumsum(rng.uniform(0.01, 0.1, n))
        full, nf, _ = O.composite(s, rgb, t, 0.05, 0.0)
        trunc, nu, _ = O.composite(s, rgb, t, 0.05, 1e-4)
        tau = np.cumsum(s * 0.05)
        T_after = np.exp(-tau)
        if (T_after < 1e-4).any():
            assert nu == int(np.argmax(T_after < 1e-4)) + 1
        else:
            assert nu == n
        assert nf == n
        assert np.max(np.abs(full[:3] - trunc[:3])) <= 1e-4


def test_composite_empty_ray_is_background():
    out, used, _ = O.composite([], np.zeros((0, 3)), [], 0.1, 1e-4, (0.3, 0.2, 0.1))
    assert used == 0
    assert np.allclose(out, [0.3, 0.2, 0.1, 0.0, 0.0])


# ----------------------------------------------------------------------------
# whole rays through the oracle's render
# ----------------------------------------------------------------------------

def _const_weights(W, H, b_sigma, b_rgb):
    offs, P = _offsets(W, H)
    w = np.zeros(P, dtype=np.float32)
    w[offs[H][1]] = b_sigma
    w[offs[H + 2][1]:offs[H + 2][1] + 3] = b_rgb
    return w


def test_render_empty_grid_is_background(room32):
    occ = np.zeros((32, 32, 32), dtype=bool)
    g = _grid(occ)
    W, H = 8, 2
    w = _const_weights(W, H, 1.0, [0, 0, 0])[None, :]
    aff = np.array([[1, 1, 1, 0, 0, 0]], dtype=np.float32)
    cams = F.camera_array(room32.cams)
    r = O.render(g, w, aff, W, H, 10.0, cams, None, 0.025, 64, bg=(0.25, 0.5, 0.75))
    assert (r["n_kept"] == 0).all()
    assert np.allclose(r["rgb"], np.array([0.25, 0.5, 0.75], dtype=np.float32), atol=0)
    assert np.allclose(r["opacity"], 0) and np.allclose(r["depth"], 0)


def test_render_slab_transmittance_matches_exp_sigma_l():
    """A fully occupied slab z in [16, 24) voxels, constant density: the ray's
    opacity converges to 1 - exp(-sigma * chord) as delta -> 0, and for each
    delta equals 1 - exp(-sigma * n * delta) with n the samples inside."""
    G, vox = 32, 0.1
    occ = np.zeros((G, G, G), dtype=bool)
    occ[16:24, :, :] = True
    g = _grid(occ, vox)
    W, H = 8, 2
    b_sigma = 0.3
    w = _const_weights(W, H, b_sigma, [0.4, -0.2, 1.0])[None, :]
    aff = np.array([[1, 1, 1, 0, 0, 0]], dtype=np.float32)
    sigma = O.f32(4.0) * math.log1p(math.exp(O.f32(b_sigma)))
    # camera at (1.6, 1.6, 0.45) looking along +z tilted by 0.3 rad in x
    R = F.yaw_pitch(0.3, 0.0)
    cam = np.concatenate([[1, 64, 64, math.pi / 2], R.reshape(9), [1.6, 1.6, 0.45]])[None, :]
    rays = np.array([[0, 32 * 64 + 32]], dtype=np.uint32)     # the central pixel
    camf = O.cams_f32(cam)
    o, d = O.ray(camf[0], 32.5, 32.5)
    z0, z1 = 16 * O.f32(vox), 24 * O.f32(vox)
    chord = (z1 - z0) / d[2]
    errs = []
    for delta in (0.02, 0.01, 0.005, 0.0025):
        r = O.render(g, w, aff, W, H, 4.0, cam, rays, delta, 1024, t_stop=0.0)
        n = int(r["n_kept"][0])
        df = O.f32(delta)
        assert abs(r["opacity"][0] - (1 - math.exp(-sigma * n * df))) < 1e-12
        errs.append(abs(r["opacity"][0] - (1 - math.exp(-sigma * chord))))
    assert errs[-1] < 0.01 and errs[-1] < errs[0]


def _axis_camera(o):
    """A 3x3 perspective camera whose central pixel looks along world +x."""
    R = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]])
    return np.concatenate([[1, 3, 3, math.pi / 2], R.reshape(9), o])[None, :]


def test_render_records_geometric_series_and_routing():
    """Given kept-sample lists: with sigma * delta = ln 2 every sample halves
    the transmittance, so the weights are 1/2, 1/4, 1/8, 1/16 whatever the
    sample indices; colours route to each record's own field and depths to
    its own t = (j + 1/2) delta."""
    G = 32
    occ = np.zeros((G, G, G), dtype=bool)
    occ[:, :, 8:20] = True                         # any grid: the records are given
    g = _grid(occ, 0.1)
    W, H = 8, 2
    b0, b1 = np.array([0.4, -0.2, 1.0]), np.array([-1.0, 0.5, 0.25])
    w = np.stack([_const_weights(W, H, 0.0, b0), _const_weights(W, H, 0.0, b1)])
    aff = np.tile(np.array([1, 1, 1, 0, 0, 0], dtype=np.float32), (2, 1))
    delta, sigma_scale = 0.25, 4.0                 # 4 * softplus(0) * 0.25 = ln 2
    cam = _axis_camera([0.35, 1.05, 1.05])
    rays = np.array([[0, 4], [0, 4], [0, 4]], dtype=np.uint32)       # the central pixel, three record sets
    js = np.array([[3, 10, 11, 40], [0, 1, 2, 3], [5, 0, 0, 0]])
    fs = np.array([[0, 1, 1, 0], [1, 1, 1, 1], [1, 0, 0, 0]])
    cnt = np.array([4, 4, 0])
    bg = (0.1, 0.2, 0.3)
    r = O.render_records(g, w, aff, W, H, sigma_scale, cam, rays, cnt, js, fs, delta, t_stop=1e-4, bg=bg)
    c0, c1 = 1 / (1 + np.exp(-b0.astype(np.float32).astype(np.float64))), \
        1 / (1 + np.exp(-b1.astype(np.float32).astype(np.float64)))
    wts = np.array([1 / 2, 1 / 4, 1 / 8, 1 / 16])
    bgv = np.array(bg, dtype=np.float32).astype(np.float64)
    assert np.allclose(r["rgb"][0], (wts[0] + wts[3]) * c0 + (wts[1] + wts[2]) * c1 + bgv / 16, atol=1e-14)
    assert np.allclose(r["rgb"][1], (15 / 16) * c1 + bgv / 16, atol=1e-14)
    assert abs(r["depth"][0] - float((wts * (js[0] + 0.5) * delta).sum())) < 1e-13
    assert abs(r["opacity"][0] - 15 / 16) < 1e-14 and r["n_used"][0] == 4
    assert np.allclose(r["rgb"][2], bgv, atol=0) and r["opacity"][2] == 0 and r["depth"][2] == 0
    # termination: t_stop = 0.1 stops after the fourth halving (T = 1/16 < 0.1)
    js5 = np.array([[0, 1, 2, 3, 4, 5]])
    r2 = O.render_records(g, w[:1], aff[:1], W, H, sigma_scale, cam, rays[:1], [6], js5, np.zeros((1, 6)), delta,
                          t_stop=0.1)
    assert r2["n_used"][0] == 4 and abs(r2["opacity"][0] - 15 / 16) < 1e-14
    with pytest.raises(ValueError):        # a field id outside the partition
        O.render_records(g, w, aff, W, H, sigma_scale, cam, rays[:1], [1], [[0]], [[2]], delta)


def test_render_records_of_the_oracle_march_is_the_render(room32, room32_grid):
    """Fed the oracle's own march, the records render is the render."""
    cams = F.camera_array(room32.cams)
    rng = np.random.default_rng(8)
    rays = np.stack([np.zeros(300, np.int64), rng.integers(0, 128 * 64, 300)], 1).astype(np.uint32)
    ref = O.render(room32_grid, room32.weights, room32.affine, room32.W, room32.H, room32.sigma_scale, cams, rays,
                   room32.delta, room32.n_max)
    cnt, js, fs, _ = O.march_rays(room32_grid, cams, rays, room32.delta, room32.n_max)
    got = O.render_records(room32_grid, room32.weights, room32.affine, room32.W, room32.H, room32.sigma_scale, cams,
                           rays, cnt, js, fs, room32.delta)
    for k in ("rgb", "depth", "opacity", "n_used"):
        assert np.array_equal(got[k], ref[k]), k
    assert cnt.sum() > 1000


def test_sample_tie_distance_closed_form():
    """Distance to the nearest face whose two sides differ, along +x through
    one occupied voxel x in [1.0, 1.1) (y, z at its centre), and a field
    boundary between two occupied voxels."""
    G, vox = 32, 0.1
    occ = np.zeros((G, G, G), dtype=bool)
    occ[10, 10, 10] = True
    g = _grid(occ, vox)
    x0 = 0.3125
    cam = _axis_camera([x0, 1.05, 1.05])
    delta = 0.0078125
    vf = O.f32(vox)
    y_fr = O.f32(1.05) / vf - 10                     # the y and z faces of the occupied voxel
    js = np.arange(0, 130)
    dist = O.sample_tie_distance(g, cam, np.array([[0, 4]], np.uint32), np.zeros(js.size, np.int64), js, delta)
    for j, dd in zip(js, dist):
        xv = (x0 + (j + 0.5) * delta) / vf
        ix = math.floor(xv)
        fr = xv - ix
        if ix == 10:
            expect = min(fr, 1 - fr, y_fr, 1 - y_fr)
        elif ix == 9:
            expect = 1 - fr
        elif ix == 11:
            expect = fr
        else:
            expect = math.inf
        assert dd == expect or abs(dd - expect) < 1e-12, (j, dd, expect)
    # two occupied voxels of different fields: their shared face counts
    occ2 = np.zeros((G, G, G), dtype=bool)
    occ2[10, 10, 10:12] = True
    s = _Scene(occ2, vox)
    part = _Part(2)
    part.field_of_rank = np.array([0, 1], dtype=np.uint16)
    g2 = O.Grid(s, part)
    d2 = O.sample_tie_distance(g2, cam, np.array([[0, 4]], np.uint32), np.zeros(js.size, np.int64), js, delta)
    for j, dd in zip(js, d2):
        xv = (x0 + (j + 0.5) * delta) / vf
        ix, fr = math.floor(xv), xv - math.floor(xv)
        if ix == 10:
            assert abs(dd - min(fr, 1 - fr, y_fr, 1 - y_fr)) < 1e-12
        elif ix == 11:
            assert abs(dd - min(fr, 1 - fr, y_fr, 1 - y_fr)) < 1e-12


# ----------------------------------------------------------------------------
# gradient: analytic reverse mode versus central finite differences
# ----------------------------------------------------------------------------

def test_render_mixed_widths_assembles_per_field_mlps(room32, room32_grid):
    """A render whose fields have different MLP widths equals the composite of
    each sample's own field MLP (its own width, its own slice of the weights)
    along the marched samples; uniform widths passed per field equal the
    single-width render."""
    H = 2
    widths = F.mixed_widths(1, room32.part.n_fields)
    assert len(set(widths.tolist())) > 1
    w = F.xavier_weights_mixed(1, F.ROLE_STUDENT, widths, H, bias_scale=0.2)
    offs = np.concatenate([[0], np.cumsum([F.n_params(int(W), H) for W in widths])])
    cams = F.camera_array(room32.cams)
    cf = O.cams_f32(cams)
    rng = np.random.default_rng(5)
    pix = rng.choice(room32.cams[0].n_pixels, 60, replace=False)
    rays = np.stack([np.zeros_like(pix), pix], 1).astype(np.uint32)
    ref = O.render(room32_grid, w, room32.affine, 0, H, room32.sigma_scale, cams, rays, room32.delta,
                   room32.n_max, widths=widths)
    cnt, js, fs, _ = O.march_rays(room32_grid, cams, rays, room32.delta, room32.n_max)
    delta = O.f32(room32.delta)
    width_px = room32.cams[0].width
    checked = 0
    for r in range(len(pix)):
        o, d = O.ray(cf[0], pix[r] % width_px + 0.5, pix[r] // width_px + 0.5)
        sig, rgb, t = [], [], []
        for k in range(cnt[r]):
            f = fs[r, k]
            tt = (js[r, k] + 0.5) * delta
            out = O.mlp(w[offs[f]:offs[f + 1]], int(widths[f]), H, room32.sigma_scale, room32.affine[f], o + tt * d, d)
            sig.append(out[0]); rgb.append(out[1:]); t.append(tt)
        got, _, _ = O.composite(np.array(sig), np.array(rgb).reshape(-1, 3), np.array(t), delta)
        assert np.abs(got[:3] - ref["rgb"][r]).max() <= 1e-12
        checked += cnt[r] > 0
    assert checked > 10
    wu = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, 32, H)
    a = O.render(room32_grid, wu, room32.affine, 32, H, room32.sigma_scale, cams, rays, room32.delta, room32.n_max)
    b = O.render(room32_grid, wu.reshape(-1), room32.affine, 0, H, room32.sigma_scale, cams, rays, room32.delta,
                 room32.n_max, widths=np.full(room32.part.n_fields, 32))
    assert np.array_equal(a["rgb"], b["rgb"])


def test_loss_gradient_matches_central_differences(room32, room32_grid):
    W, H = 16, 2
    n_fields = room32.part.n_fields
    w = F.xavier_weights(1, F.ROLE_STUDENT, n_fields, W, H, bias_scale=0.1)
    cams = F.camera_array(room32.cams)
    rays = F.ray_batch(1, room32.cams, 96)
    rng = np.random.default_rng(12)
    target = rng.uniform(0, 1, (96, 3)).astype(np.float32)
    args = (room32_grid, w, room32.affine, W, H, room32.sigma_scale, cams, rays, target, room32.delta, 64)
    loss, grad, sig, _ = O.loss_grad(*args)
    assert loss > 0 and np.abs(grad).max() > 0
    h = 1e-4
    gmax = np.abs(grad).max()
    P = w.shape[1]
    checked = 0
    for _ in range(60):
        f = int(rng.integers(n_fields))
        k = int(rng.integers(P))
        wp, wm = w.copy(), w.copy()
        # perturb in FP64 terms: the oracle reads FP32 weights, so use an
        # FP32-representable step and measure the step actually taken
        wp[f, k] = np.float32(w[f, k] + h)
        wm[f, k] = np.float32(w[f, k] - h)
        lp, _, sp, _ = O.loss_grad(room32_grid, wp, *args[2:], want_grad=False)
        lm, _, sm, _ = O.loss_grad(room32_grid, wm, *args[2:], want_grad=False)
        if sp != sig or sm != sig:
            continue     # the step crossed a ReLU kink or a termination index
        fd = (lp - lm) / (float(wp[f, k]) - float(wm[f, k]))
        assert abs(fd - grad[f, k]) <= 1e-6 * gmax + 1e-7 * abs(grad[f, k]) + 1e-10, (f, k, fd, grad[f, k])
        checked += 1
    assert checked >= 40


# ----------------------------------------------------------------------------
# Adam
# ----------------------------------------------------------------------------

def test_adam_first_steps_closed_form():
    """With zero moments, bias correction makes the first update exactly
    lr * g / (|g| + eps) (= lr * sign(g) for |g| >> eps), and a constant
    gradient keeps that update on later steps."""
    rng = np.random.default_rng(0)
    g = rng.normal(size=1000) * 10.0 ** rng.uniform(-3, 2, 1000)
    w0 = rng.normal(size=1000)
    lr, eps = 1e-3, 1e-8
    w, m, v = O.adam(w0, np.zeros(1000), np.zeros(1000), g, lr, 1, eps=eps)
    assert np.allclose(w0 - w, lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    for t in range(2, 11):
        w_prev = w
        w, m, v = O.adam(w, m, v, g, lr, t, eps=eps)
        assert np.allclose(w_prev - w, lr * g / (np.abs(g) + eps), rtol=1e-9, atol=0)
    # the moments are the exponential averages
    assert np.allclose(m, g * (1 - 0.9 ** 10), rtol=1e-12)
    assert np.allclose(v, g * g * (1 - 0.99 ** 10), rtol=1e-12)


# ----------------------------------------------------------------------------
# progressive probabilistic occupancy (Eq. 6, Alg. 1 stage I)
# ----------------------------------------------------------------------------

def _sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


def test_occupancy_clamp_bounds_match_paper():
    """The paper states the log-odds range [-2, 3.5] as occupancy
    probabilities 0.12 and 0.97 (golden values)."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    occ = gold["occupancy"]
    assert abs(_sigmoid(occ["logit_min"]) - occ["p_min"]) < 5e-3
    assert abs(_sigmoid(occ["logit_max"]) - occ["p_max"]) < 5e-3
    assert occ["logit_max"] > math.log(occ["p_occupied"] / (1 - occ["p_occupied"]))


def test_segment_voxels_axis_aligned_closed_form():
    dims, org, vox = (32, 32, 32), (0.0, 0.0, 0.0), 0.1
    for axis in range(3):
        for sgn in (1.0, -1.0):
            o = np.array([1.55, 1.65, 1.75])
            d = np.zeros(3)
            d[axis] = sgn
            got = O.segment_voxels(dims, org, vox, o, d, 0.93)
            c0 = np.floor(o / vox).astype(int)
            u_end = (o[axis] + sgn * 0.93) / vox
            cells = np.arange(c0[axis], int(np.floor(u_end)) + sgn, int(sgn))
            want = []
            for k in cells:
                c = c0.copy()
                c[axis] = k
                want.append((c[2] * 32 + c[1]) * 32 + c[0])
            assert got.tolist() == want, (axis, sgn)


def test_segment_voxels_match_dense_sampling():
    """Random segments: the voxels met by points sampled every 1e-4 voxel
    along the segment are exactly the traversal's voxels (no near-ties at
    these random parameters)."""
    rng = np.random.default_rng(6)
    dims, org, vox = (32, 32, 32), (0.0, 0.0, 0.0), 0.1
    for _ in range(20):
        o = rng.uniform(0.2, 3.0, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        t_end = rng.uniform(0.05, 1.5)
        got = O.segment_voxels(dims, org, vox, o, d, t_end)
        ts = np.linspace(0, t_end, int(t_end / vox * 1e4) + 2)[1:-1]
        pts = o[None, :] + ts[:, None] * d[None, :]
        c = np.floor(pts / vox).astype(np.int64)
        ok = np.all((c >= 0) & (c < 32), axis=1)
        lin = (c[ok, 2] * 32 + c[ok, 1]) * 32 + c[ok, 0]
        seq = lin[np.concatenate([[True], lin[1:] != lin[:-1]])]
        assert got.tolist() == seq.tolist()


def _cam_pixels(dirs, o):
    """One 1x1 perspective view per direction, looking along it (its only
    pixel's ray is the view axis)."""
    cams = []
    for d in dirs:
        d = np.asarray(d, dtype=np.float64)
        d = d / np.linalg.norm(d)
        # camera z axis = d; any orthonormal completion
        a = np.array([1.0, 0, 0]) if abs(d[0]) < 0.9 else np.array([0, 1.0, 0])
        x = np.cross(a, d); x /= np.linalg.norm(x)
        y = np.cross(d, x)
        R = np.stack([x, y, d], axis=1)        # columns: camera axes in world
        cams.append(F.Camera(F.PERSPECTIVE, 1, 1, 1.0, R, np.asarray(o, dtype=np.float64)))
    return cams


def test_occupancy_hits_clamp_and_threshold():
    """One voxel hit by a confident ray in every scan: L grows by
    logit(0.7) per scan, is clamped at 3.5, and the voxel becomes occupied
    only once L > logit(0.97); the voxels before it go free, clamped at -2."""
    dims, org, vox = (32, 32, 32), (0.0, 0.0, 0.0), 0.1
    o = np.array([0.55, 1.65, 1.75])
    cams = _cam_pixels([[1.0, 0, 0]] * 7, o)
    cam16 = F.camera_array(cams)
    o32 = O.cams_f32(cam16)[0, 13:16]
    depth = np.full(7, 1.0, np.float32)        # end point 1.0 further along +x, A = 1
    opac = np.ones(7, np.float32)
    L = np.zeros(32 ** 3)
    lh, lm = math.log(0.7 / 0.3), math.log(0.4 / 0.6)
    for n in range(1, 8):
        bits, _ = O.occupancy_update(dims, org, vox, L, cam16[n - 1:n], depth[:1], opac[:1])
        e = np.floor((o32 + np.array([1.0, 0, 0])) / vox).astype(int)
        ie = (e[2] * 32 + e[1]) * 32 + e[0]
        assert abs(L[ie] - min(n * lh, 3.5)) < 1e-12
        occupied = bool(bits[ie >> 5] >> (ie & 31) & 1)
        assert occupied == (min(n * lh, 3.5) > math.log(0.97 / 0.03))
        first = (np.floor(o32 / vox).astype(int))
        i0 = (first[2] * 32 + first[1]) * 32 + first[0]
        assert abs(L[i0] - max(n * lm, -2.0)) < 1e-12


def test_occupancy_confidence_scaling_and_opacity_floor():
    """A ray of opacity A ending in voxel v moves v by logit(1/2 + 0.2 A)
    and every voxel it crosses by logit(0.4), nothing else; a ray below the
    opacity floor (0.5) changes nothing."""
    dims, org, vox = (32, 32, 32), (0.0, 0.0, 0.0), 0.1
    o = np.array([0.55, 1.65, 1.75])
    cam16 = F.camera_array(_cam_pixels([[1.0, 0, 0]], o))
    L = np.zeros(32 ** 3)
    a = float(np.float32(0.6))
    O.occupancy_update(dims, org, vox, L, cam16, np.array([0.6], np.float32), np.array([0.6], np.float32))
    o32 = O.cams_f32(cam16)[0, 13:16]
    e = np.floor((o32 + np.array([1.0, 0, 0])) / vox).astype(int)
    ie = (e[2] * 32 + e[1]) * 32 + e[0]
    ph = 0.5 + 0.2 * a
    assert abs(L[ie] - math.log(ph / (1 - ph))) < 1e-12
    nz = np.nonzero(L)[0]
    seg = O.segment_voxels(dims, org, vox, o32, np.array([1.0, 0, 0]), float(np.float32(0.6)) / a)
    assert set(nz.tolist()) == set(seg.tolist()) | {ie}
    assert np.allclose(L[seg[seg != ie]], math.log(0.4 / 0.6), atol=1e-12)
    L2 = L.copy()
    O.occupancy_update(dims, org, vox, L2, cam16, np.array([0.2], np.float32), np.array([0.45], np.float32))
    assert np.array_equal(L, L2)


def test_occupancy_scan_with_many_rays_matches_per_voxel_rules():
    """A 16x8 equirect scan: every updated voxel took exactly one update --
    a voxel where rays end takes the hit update of the largest opacity among
    them (even if other rays cross it), a voxel only crossed takes one free
    update however many rays cross it -- rebuilt here from the traversal
    alone."""
    dims, org, vox = (32, 32, 32), (0.0, 0.0, 0.0), 0.1
    rng = np.random.default_rng(9)
    cam = F.Camera(F.EQUIRECT, 16, 8, 0.0, F.yaw_pitch(0.4, 0.1), np.array([1.62, 1.57, 1.71]))
    cam16 = F.camera_array([cam])
    depth = rng.uniform(0.2, 1.2, 128).astype(np.float32)
    opac = rng.uniform(0.3, 1.0, 128).astype(np.float32)
    depth *= opac                               # D = A * (expected depth)
    L = np.zeros(32 ** 3)
    O.occupancy_update(dims, org, vox, L, cam16, depth, opac)
    cf = O.cams_f32(cam16)[0]
    conf, free = {}, set()
    for p in range(128):
        if opac[p] < 0.5:
            continue
        o, d = O.ray(cf, p % 16 + 0.5, p // 16 + 0.5)
        t_end = float(depth[p]) / float(opac[p])
        free |= set(O.segment_voxels(dims, org, vox, o, d, t_end).tolist())
        e = np.floor((o + t_end * d) / vox).astype(int)
        ie = int((e[2] * 32 + e[1]) * 32 + e[0])
        conf[ie] = max(conf.get(ie, 0.0), float(opac[p]))
    want = np.zeros(32 ** 3)
    for i in free:
        want[i] = math.log(0.4 / 0.6)
    for i, a in conf.items():
        ph = 0.5 + 0.2 * a
        want[i] = math.log(ph / (1 - ph))
    assert np.allclose(L, want, atol=1e-12)


# ----------------------------------------------------------------------------
# adaptive assignment of occupied voxels to networks (Alg. 1 stage II)
# ----------------------------------------------------------------------------

def test_assign_fields_line_is_contiguous_runs():
    """Occupied voxels on one row: every anchor is the leftmost unassigned
    voxel and its nearest unassigned neighbours are the next ones to the
    right, so networks are runs of s = S // n (the last takes the rest)."""
    dims = (64, 4, 4)
    S, n = 61, 6
    lin = np.arange(S, dtype=np.int64)          # x = 0..60, y = z = 0
    f = O.assign_fields(dims, lin, n)
    s = S // n
    assert np.array_equal(f, np.minimum(np.arange(S) // s, n - 1))


def _assign_brute(dims, lin, n):
    gx, gy = dims[0], dims[1]
    xyz = np.stack([lin % gx, (lin // gx) % gy, lin // (gx * gy)], axis=1)
    S = lin.size
    s = S // n
    field = np.full(S, -1)
    for k in range(n):
        free = np.nonzero(field < 0)[0]
        if k == n - 1:
            field[free] = k
            break
        a = free[np.argmin(lin[free])]
        d2 = ((xyz[free] - xyz[a]) ** 2).sum(axis=1)
        order = np.lexsort((lin[free], d2))      # by distance, then by linear index
        field[free[order[:s]]] = k
    return field


def test_assign_fields_matches_full_sort():
    rng = np.random.default_rng(12)
    for dims, S, n in [((32, 8, 8), 300, 7), ((16, 16, 16), 500, 13), ((32, 32, 32), 1000, 10)]:
        total = dims[0] * dims[1] * dims[2]
        lin = np.sort(rng.choice(total, S, replace=False)).astype(np.int64)
        f = O.assign_fields(dims, lin, n)
        assert np.array_equal(f, _assign_brute(dims, lin, n))
        counts = np.bincount(f, minlength=n)
        assert np.all(counts[:-1] == S // n) and counts[-1] == S - (n - 1) * (S // n)


# ----------------------------------------------------------------------------
# the global 360NeRF teacher and the distillation loss (Eq. 7)
# ----------------------------------------------------------------------------

def test_teacher_param_count_matches_paper():
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    t = gold["teacher_360nerf"]
    assert O.teacher_param_count() == sum(o * i + o for o, i in F.teacher_layer_shapes())
    assert abs(O.teacher_param_count() - t["params"]) <= t["tolerance"]


def _np_teacher(w, aff, p, d):
    """The teacher written independently with NumPy matrices."""
    shapes = F.teacher_layer_shapes()
    mats, o = [], 0
    for (n_out, n_in) in shapes:
        Wm = w[o:o + n_out * n_in].reshape(n_out, n_in).astype(np.float64)
        b = w[o + n_out * n_in:o + n_out * n_in + n_out].astype(np.float64)
        mats.append((Wm, b))
        o += n_out * n_in + n_out
    relu = lambda v: np.maximum(v, 0)
    xg = aff[:3].astype(np.float64) * p + aff[3:].astype(np.float64)
    pe, ped = _np_encode(xg, 10), _np_encode(d, 4)
    h = relu(mats[0][0] @ pe + mats[0][1])
    for k in (1, 2, 3):
        h = relu(mats[k][0] @ h + mats[k][1])
    h = relu(mats[4][0] @ np.concatenate([h, pe]) + mats[4][1])
    for k in (5, 6):
        h = relu(mats[k][0] @ h + mats[k][1])
    h = mats[7][0] @ h + mats[7][1]
    sigma = relu(mats[8][0] @ h + mats[8][1])[0]
    f = relu(mats[9][0] @ h + mats[9][1])
    g = relu(mats[10][0] @ np.concatenate([f, ped]) + mats[10][1])
    rgb = 1 / (1 + np.exp(-(mats[11][0] @ g + mats[11][1])))
    return np.concatenate([[sigma], rgb])


def test_teacher_matches_independent_chain():
    w = F.teacher_weights(3, bias_scale=0.2)
    aff = np.array([0.3, 0.25, 0.2, -1.0, -0.9, -0.8], dtype=np.float32)
    rng = np.random.default_rng(31)
    p = rng.uniform(0, 6, (8, 3))
    d = rng.normal(size=(8, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = O.teacher_eval(w, aff, p, d)
    for i in range(8):
        assert np.abs(got[i] - _np_teacher(w, aff, p[i], d[i])).max() <= 1e-10


def test_teacher_skip_and_concat_routing():
    """Only the skip path carries F(x)[m] (layers 1-4 are zero); the colour
    sees [feature; F(d)] in that order: sigma = relu(F(x)[m]) and
    green = sigmoid(relu(relu(F(x)[m]) + F(d)[m']))."""
    shapes = F.teacher_layer_shapes()
    offs, o = [], 0
    for (n_out, n_in) in shapes:
        offs.append((o, n_in))
        o += n_out * n_in + n_out
    w = np.zeros(o, dtype=np.float32)
    m, mp = 8, 13                       # cos(pi x2) and cos(2 pi d1), values known below
    w[offs[4][0] + 0 * offs[4][1] + 256 + m] = 1.0          # layer 5 unit 0 <- F(x)[m]
    for k in (5, 6, 7):
        w[offs[k][0] + 0] = 1.0                            # identity on unit 0
    w[offs[8][0] + 0] = 1.0                                 # density <- unit 0
    w[offs[9][0] + 2 * 256 + 0] = 1.0                       # feature 2 <- unit 0
    w[offs[10][0] + 5 * offs[10][1] + 2] = 1.0              # g5 <- feature 2
    w[offs[10][0] + 5 * offs[10][1] + 256 + mp] = 1.0       #     + F(d)[m']
    w[offs[11][0] + 1 * 128 + 5] = 1.0                      # green <- g5
    aff = np.array([1, 1, 1, 0, 0, 0], dtype=np.float32)
    p = np.array([0.2, 0.4, -1.0 / 3.0])                    # cos(pi x2) = 1/2
    d = np.array([0.3, 1.0 / 6.0, 0.2])                     # cos(2 pi d1) = 1/2
    got = O.teacher_eval(w, aff, p[None], d[None])[0]
    assert abs(got[0] - 0.5) < 1e-12
    assert abs(got[2] - 1 / (1 + math.exp(-1.0))) < 1e-12
    assert abs(got[1] - 0.5) < 1e-15 and abs(got[3] - 0.5) < 1e-15


def test_distill_gradient_matches_central_differences(room32):
    W, H = 16, 2
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.2)
    p, d, f = F.distill_points(room32.scene, room32.part, 1, 6)
    target = np.random.default_rng(4).uniform(0.1, 0.9, (p.shape[0], 4))
    loss, g = O.distill_loss_grad(w, room32.affine, W, H, 1.5, p, d, f, target, 6.0)
    rng = np.random.default_rng(8)
    checked = 0
    for _ in range(40):
        fi, k = int(rng.integers(0, w.shape[0])), int(rng.integers(0, w.shape[1]))
        if not np.any(f == fi):
            continue
        h = 1e-3 * max(1.0, abs(float(w[fi, k])))
        wp, wm = w.copy(), w.copy()
        wp[fi, k] += h
        wm[fi, k] -= h
        lp, _ = O.distill_loss_grad(wp, room32.affine, W, H, 1.5, p, d, f, target, 6.0)
        lm, _ = O.distill_loss_grad(wm, room32.affine, W, H, 1.5, p, d, f, target, 6.0)
        fd = (lp - lm) / (float(wp[fi, k]) - float(wm[fi, k]))
        assert abs(fd - g[fi, k]) <= 1e-5 * max(1.0, abs(fd)), (fi, k, fd, g[fi, k])
        checked += 1
    assert checked >= 10


def test_point_adjoint_matches_central_differences(room32):
    """The adjoint at points for given output gradients is the weight
    gradient of sum_i dl_i . MLP(x_i), checked by central differences of the
    forward pass; the reported kink margin is a positive distance."""
    W, H = 16, 3
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.2)
    p, d, f = F.distill_points(room32.scene, room32.part, 2, 3)
    dl = np.random.default_rng(5).normal(size=(p.shape[0], 4))
    g, margin = O.mlp_grad_points(w, room32.affine, W, H, 1.5, p, d, f, dl)
    assert np.all(margin > 0) and np.all(np.isfinite(margin))

    def functional(wt):
        return sum(float(dl[i] @ O.mlp(wt[f[i]], W, H, 1.5, room32.affine[f[i]], p[i], d[i]))
                   for i in range(p.shape[0]))

    rng = np.random.default_rng(9)
    checked = 0
    for _ in range(30):
        fi, k = int(rng.integers(0, w.shape[0])), int(rng.integers(0, w.shape[1]))
        if not np.any(f == fi):
            continue
        h = 1e-3 * max(1.0, abs(float(w[fi, k])))
        wp, wm = w.copy(), w.copy()
        wp[fi, k] += h
        wm[fi, k] -= h
        fd = (functional(wp) - functional(wm)) / (float(wp[fi, k]) - float(wm[fi, k]))
        assert abs(fd - g[fi, k]) <= 1e-5 * max(1.0, abs(fd)), (fi, k, fd, g[fi, k])
        checked += 1
    assert checked >= 8


# ---- the BF16 reading (the library's BF16 tensor-core path) ----

def test_bf16_rounding_matches_library_conversion():
    """Nearest-even rounding to 8 significant bits: closed-form cases, and
    PyTorch's float32 -> bfloat16 conversion on FP32 inputs."""
    torch = pytest.importorskip("torch")
    assert O.bf16(1.0 + 2.0 ** -8) == 1.0                       # tie, to even
    assert O.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # tie, to even (upwards)
    assert O.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert O.bf16(-3.14159) == -3.140625
    assert O.bf16(0.0) == 0.0
    x = np.random.default_rng(3).normal(size=2000).astype(np.float32) * np.float32(10.0) ** \
        np.random.default_rng(4).integers(-8, 8, 2000).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([O.bf16(float(v)) for v in x])
    assert np.array_equal(got, ref)


def _bf16_np(x):
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(np.abs(x))
    q = np.ldexp(1.0, e - 8)
    return np.where(x == 0, 0.0, np.copysign(np.round(np.abs(x) / q) * q, x))


def _pe_np(x, L):
    cols = [x]
    for k in range(L):
        cols.append(np.sin(np.pi * 2.0 ** k * x))
        cols.append(np.cos(np.pi * 2.0 ** k * x))
    return np.concatenate(cols, axis=1)


def _bf16_reading_np(wf, aff, W, H, sig, p, d, dl):
    """An independent NumPy chain of the BF16 reading for one field: every
    matrix layer but the 3-output one on BF16 inputs, weights and biases;
    the adjoint on BF16 output gradients, inputs and weights."""
    R = _bf16_np
    layers, o = [], 0
    for r, c in [(W, 63)] + [(W, W)] * (H - 1) + [(1 + W, W), (W, W + 27), (3, W)]:
        layers.append((wf[o:o + r * c].reshape(r, c).astype(np.float64), wf[o + r * c:o + r * c + r].astype(np.float64)))
        o += r * c + r
    x = p * aff[:3] + aff[3:]
    h, ins, zs = _pe_np(x, 10), [], []
    for l in range(H):
        M, b = layers[l]
        ins.append(R(h))
        z = R(h) @ R(M).T + R(b)
        zs.append(z)
        h = np.maximum(z, 0)
    M, b = layers[H]
    ins.append(R(h))
    hd = R(h) @ R(M).T + R(b)
    inc = np.concatenate([hd[:, 1:], _pe_np(d, 4)], axis=1)
    Mc, bc = layers[H + 1]
    zc = R(inc) @ R(Mc).T + R(bc)
    g = np.maximum(zc, 0)
    Mo, bo = layers[H + 2]
    rgb = 1 / (1 + np.exp(-(g @ Mo.T + bo)))
    out = np.concatenate([(sig * np.log1p(np.exp(hd[:, :1]))), rgb], axis=1)
    grads = [None] * (H + 3)
    dzo = dl[:, 1:] * rgb * (1 - rgb)
    grads[H + 2] = (R(dzo).T @ R(g), R(dzo).sum(0))
    dzc = R((dzo @ Mo) * (zc > 0))
    grads[H + 1] = (dzc.T @ R(inc), dzc.sum(0))
    dfeat = dzc @ R(Mc)[:, :W]
    dsig = dl[:, 0] * sig / (1 + np.exp(-hd[:, 0]))
    dzh = R(np.concatenate([dsig[:, None], dfeat], axis=1))
    grads[H] = (dzh.T @ ins[H], dzh.sum(0))
    dh = dzh @ R(M)
    for l in range(H - 1, -1, -1):
        dz = R(dh * (zs[l] > 0))
        grads[l] = (dz.T @ ins[l], dz.sum(0))
        if l > 0:
            dh = dz @ R(layers[l][0])
    return out, np.concatenate([np.concatenate([a.ravel(), b]) for a, b in grads])


def test_bf16_reading_matches_independent_chain(room32):
    W, H, sig = 16, 3, 1.5
    w = F.xavier_weights(1, F.ROLE_STUDENT, room32.part.n_fields, W, H, bias_scale=0.2)
    p, d, f = F.distill_points(room32.scene, room32.part, 2, 40)
    dl = np.random.default_rng(6).normal(size=(p.shape[0], 4))
    g, _ = O.mlp_grad_points(w, room32.affine, W, H, sig, p, d, f, dl, quant=2)
    g64, _ = O.mlp_grad_points(w, room32.affine, W, H, sig, p, d, f, dl)
    for fi in range(room32.part.n_fields):
        m = f == fi
        aff = room32.affine[fi].astype(np.float64)
        out, gn = _bf16_reading_np(w[fi], aff, W, H, sig, p[m].astype(np.float64), d[m].astype(np.float64), dl[m])
        assert np.allclose(g[fi], gn, rtol=1e-10, atol=1e-12 * np.abs(gn).max())
        for i in np.nonzero(m)[0][:3]:
            o = O.mlp(w[fi], W, H, sig, aff, p[i], d[i], quant=2)
            j = int(np.count_nonzero(m[:i]))
            assert np.allclose(o, out[j], rtol=1e-12, atol=1e-14)
    # the rounding is applied: the reading moves away from FP64, and stays
    # correlated with it (a few mask flips on 40 samples per field move
    # single entries by up to ~15 % of max |g|)
    rel = np.abs(g - g64).max() / np.abs(g64).max()
    cos = float((g * g64).sum() / (np.linalg.norm(g) * np.linalg.norm(g64)))
    assert 1e-5 < rel < 0.3 and cos > 0.99


def test_teacher_bf16_reading_matches_independent_chain():
    """The teacher's BF16 reading against a NumPy chain that rounds the same
    operands: inputs and weights of every matrix layer but the density head
    and layer 11, and the biases of layers 1, 5 and 10 (the ones the
    tensor-core kernel folds into its products)."""
    w = F.teacher_weights(3, bias_scale=0.2)
    aff = np.array([0.3, 0.25, 0.2, -1.0, -0.9, -0.8], dtype=np.float32)
    rng = np.random.default_rng(32)
    p = rng.uniform(0, 6, (6, 3))
    d = rng.normal(size=(6, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = O.teacher_eval(w, aff, p, d, quant=2)
    ref64 = O.teacher_eval(w, aff, p, d)
    R = _bf16_np
    mats, o = [], 0
    for (n_out, n_in) in F.teacher_layer_shapes():
        mats.append((w[o:o + n_out * n_in].reshape(n_out, n_in).astype(np.float64),
                     w[o + n_out * n_in:o + n_out * n_in + n_out].astype(np.float64)))
        o += n_out * n_in + n_out
    relu = lambda v: np.maximum(v, 0)
    for i in range(6):
        xg = aff[:3].astype(np.float64) * p[i] + aff[3:].astype(np.float64)
        pe, ped = _np_encode(xg, 10), _np_encode(d[i], 4)
        folded = lambda k, x: R(mats[k][0]) @ R(x) + R(mats[k][1])
        plain = lambda k, x: R(mats[k][0]) @ R(x) + mats[k][1]
        h = relu(folded(0, pe))
        for k in (1, 2, 3):
            h = relu(plain(k, h))
        h = relu(folded(4, np.concatenate([h, pe])))
        for k in (5, 6):
            h = relu(plain(k, h))
        h = plain(7, h)
        sigma = relu(mats[8][0] @ h + mats[8][1])[0]
        f = relu(plain(9, h))
        g = relu(folded(10, np.concatenate([f, ped])))
        rgb = 1 / (1 + np.exp(-(mats[11][0] @ g + mats[11][1])))
        assert np.abs(got[i] - np.concatenate([[sigma], rgb])).max() <= 1e-10 * max(1.0, abs(sigma))
    # the rounding is applied and stays a small perturbation of FP64
    diff = np.abs(got - ref64).max()
    assert 1e-6 < diff < 0.2

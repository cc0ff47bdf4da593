"""FP64 CPU oracle (ctypes front end of ``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs import this module; the rendering
library and its Python binding never do.  It shares no code with the CUDA
path: the only common module is ``fixtures`` (seeded input generators).

Every float input handed to the C code is first rounded to FP32, because the
library receives FP32 inputs; the oracle then computes in FP64 from exactly
the values the library sees.

Parity status of each function (what pins it; see tests/test_oracle_pins.py):
  ray             pinned: Eq. 2/3 special pixels, round trip through Eq. 2
  label map       pinned: brute-force point-in-box over the partition boxes
  march           pinned: analytic chord counts, empty/full grids
  encode / mlp    pinned: one-hot closed forms, zero-weight closed form,
                  parameter count 6,212 (Appendix)
  composite       pinned: two-sample closed form, constant slab exp(-sigma l),
                  sum of weights = 1 - T_end, empty ray = background
  loss / grad     pinned: central finite differences (h = 1e-4)
  adam            pinned: first-step update lr * sign(g), constant-gradient steps
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/liboracle.so (gcc, OpenMP, -O2)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        i32p, u32p, u16p, u8p = P(ctypes.c_int32), P(ctypes.c_uint32), P(ctypes.c_uint16), P(ctypes.c_uint8)
        f32p, f64p, u64p = P(ctypes.c_float), P(ctypes.c_double), P(ctypes.c_uint64)
        I, D, I64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        L.orc_param_count.argtypes = [I, I]; L.orc_param_count.restype = I64
        L.orc_threads.restype = I
        L.orc_set_threads.argtypes = [I]
        L.orc_ray.argtypes = [f64p, D, D, f64p, f64p]
        L.orc_label_map.argtypes = [I, I, I, u32p, u16p, I64, i32p]; L.orc_label_map.restype = I64
        L.orc_march.argtypes = [i32p, f64p, D, i32p, f64p, f64p, D, I, i32p, i32p, i32p]
        L.orc_march.restype = I
        L.orc_encode.argtypes = [f64p, I, f64p]
        L.orc_mlp.argtypes = [f32p, I, I, I, D, I, f64p, f64p, f64p, f64p]
        L.orc_e4m3.argtypes = [D]; L.orc_e4m3.restype = D
        L.orc_composite.argtypes = [I, f64p, f64p, f64p, D, D, f64p, f64p, f64p]
        L.orc_composite.restype = I
        L.orc_render.argtypes = [i32p, f64p, D, i32p, f32p, f32p, I, I, I, D, I, i32p, I, f64p, I, u32p, I64,
                                 D, I, D, f64p, f64p, f64p, f64p, i32p, i32p, i32p, f64p]
        L.orc_render.restype = I
        L.orc_march_rays.argtypes = [i32p, f64p, D, i32p, f64p, I, u32p, I64, D, I, i32p, i32p, i32p, i32p]
        L.orc_march_rays.restype = I
        L.orc_render_records.argtypes = [i32p, f64p, D, i32p, f32p, f32p, I, I, I, D, I, i32p, I, f64p, I, u32p,
                                         I64, D, D, f64p, i32p, i32p, i32p, I, f64p, f64p, f64p, i32p, f64p]
        L.orc_render_records.restype = I
        L.orc_sample_tie_distance.argtypes = [i32p, f64p, D, i32p, f64p, I, u32p, I64, ctypes.POINTER(ctypes.c_int64),
                                              i32p, D, f64p]
        L.orc_sample_tie_distance.restype = I
        L.orc_loss_grad.argtypes = [i32p, f64p, D, i32p, f32p, f32p, I, I, I, I, D, f64p, I, u32p, I64,
                                    D, I, D, f64p, f32p, D, f64p, u64p, f64p]
        L.orc_loss_grad.restype = D
        L.orc_rays_touching.argtypes = [i32p, f64p, D, i32p, f64p, I, u32p, I64, D, I, I, u8p]
        L.orc_rays_touching.restype = I
        L.orc_adam.argtypes = [I64, f64p, f64p, f64p, f64p, D, D, D, D, I]
        L.orc_occupancy_update.argtypes = [i32p, f64p, D, f64p, f64p, I, f32p, f32p, f64p, u32p,
                                           ctypes.POINTER(ctypes.c_int64)]
        L.orc_occupancy_update.restype = I
        L.orc_segment_voxels.argtypes = [i32p, f64p, D, f64p, f64p, D, ctypes.POINTER(ctypes.c_int64), I64]
        L.orc_segment_voxels.restype = I64
        L.orc_assign_fields.argtypes = [i32p, ctypes.POINTER(ctypes.c_int64), I64, I, i32p]
        L.orc_assign_fields.restype = I
        L.orc_teacher_param_count.restype = I64
        L.orc_teacher_eval.argtypes = [f32p, f64p, I64, f64p, f64p, f64p, I]
        L.orc_distill_loss_grad.argtypes = [f32p, f32p, I, I, I, I, D, I64, f64p, f64p, i32p, f64p, D, f64p]
        L.orc_distill_loss_grad.restype = D
        L.orc_mlp_grad_points.argtypes = [f32p, f32p, I, I, I, I, D, I, I64, f64p, f64p, i32p, f64p, f64p, f64p]
        L.orc_bf16.argtypes = [D]
        L.orc_bf16.restype = D
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def f32(x) -> float:
    """Round a Python float to the FP32 value the library receives."""
    return float(np.float32(x))


def threads() -> int:
    return int(lib().orc_threads())


def set_threads(n: int) -> None:
    """Host threads of the oracle's parallel loops from now on."""
    lib().orc_set_threads(int(n))


def param_count(W: int, H: int) -> int:
    return int(lib().orc_param_count(W, H))


def ray(cam16: np.ndarray, uc: float, vc: float):
    cam = np.ascontiguousarray(cam16, dtype=np.float64)
    o = np.zeros(3); d = np.zeros(3)
    lib().orc_ray(_p(cam, ctypes.c_double), uc, vc, _p(o, ctypes.c_double), _p(d, ctypes.c_double))
    return o, d


def encode(x, L: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(3 + 6 * L)
    lib().orc_encode(_p(x, ctypes.c_double), L, _p(out, ctypes.c_double))
    return out


def e4m3(x) -> np.ndarray:
    """Nearest FP8 E4M3 value of each element (ties to even, saturating at 448)."""
    x = np.asarray(x, dtype=np.float64)
    f = lib().orc_e4m3
    return np.vectorize(lambda v: f(float(v)), otypes=[np.float64])(x)


def mlp(w_field: np.ndarray, W: int, H: int, sigma_scale: float, aff: np.ndarray, p, d, act: int = 0,
        quant: int = 0):
    """One sample through one field's MLP: (sigma, r, g, b).  quant=1 takes the
    FP8 E4M3 reading of the matrix layers."""
    w = np.ascontiguousarray(w_field, dtype=np.float32)
    a = np.ascontiguousarray(np.asarray(aff, dtype=np.float32), dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_mlp(_p(w, ctypes.c_float), W, H, act, f32(sigma_scale), int(quant), _p(a, ctypes.c_double),
                  _p(p, ctypes.c_double), _p(d, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def composite(sigma, rgb, t, delta: float, t_stop: float = 1e-4, bg=(0.0, 0.0, 0.0)):
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    rgb = np.ascontiguousarray(rgb, dtype=np.float64).reshape(-1)
    t = np.ascontiguousarray(t, dtype=np.float64)
    bg = np.ascontiguousarray(bg, dtype=np.float64)
    out = np.zeros(5)
    margin = np.zeros(1)
    used = lib().orc_composite(int(sigma.size), _p(sigma, ctypes.c_double), _p(rgb, ctypes.c_double),
                               _p(t, ctypes.c_double), delta, t_stop, _p(bg, ctypes.c_double),
                               _p(out, ctypes.c_double), _p(margin, ctypes.c_double))
    return out, int(used), float(margin[0])


class Grid:
    """Occupancy grid + labels as the oracle sees them (dense label map)."""

    def __init__(self, scene, part):
        gx, gy, gz = scene.dims
        self.dims = np.array(scene.dims, dtype=np.int32)
        self.origin = np.array([f32(v) for v in scene.origin], dtype=np.float64)
        self.vox = f32(scene.vox)
        bits = np.ascontiguousarray(scene.bits, dtype=np.uint32)
        fr = np.ascontiguousarray(part.field_of_rank, dtype=np.uint16)
        self.label = np.empty(gx * gy * gz, dtype=np.int32)
        n = lib().orc_label_map(gx, gy, gz, _p(bits, ctypes.c_uint32), _p(fr, ctypes.c_uint16),
                                int(fr.size), _p(self.label, ctypes.c_int32))
        if n < 0:
            raise ValueError("field_of_rank length does not match the number of occupied voxels")
        self.n_occupied = int(n)

    def args(self):
        return (_p(self.dims, ctypes.c_int32), _p(self.origin, ctypes.c_double), self.vox,
                _p(self.label, ctypes.c_int32))


def cams_f32(cam16: np.ndarray) -> np.ndarray:
    """Camera rows with R and o rounded to FP32 (what the library receives)."""
    c = np.array(cam16, dtype=np.float64, copy=True).reshape(-1, 16)
    c[:, 3:] = c[:, 3:].astype(np.float32).astype(np.float64)
    return np.ascontiguousarray(c)


def march(grid: Grid, o, d, delta: float, n_max: int):
    o = np.ascontiguousarray(o, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    js = np.zeros(max(n_max, 1), dtype=np.int32)
    fs = np.zeros(max(n_max, 1), dtype=np.int32)
    ties = np.zeros(1, dtype=np.int32)
    n = lib().orc_march(*grid.args(), _p(o, ctypes.c_double), _p(d, ctypes.c_double), f32(delta), n_max,
                        _p(js, ctypes.c_int32), _p(fs, ctypes.c_int32), _p(ties, ctypes.c_int32))
    return js[:n].copy(), fs[:n].copy(), int(ties[0])


def march_rays(grid: Grid, cams16, rays: Optional[np.ndarray], delta: float, n_max: int):
    cams = cams_f32(cams16)
    n_rays = int(rays.shape[0]) if rays is not None else int(sum(c[1] * c[2] for c in cams))
    r = np.ascontiguousarray(rays, dtype=np.uint32) if rays is not None else None
    cnt = np.zeros(n_rays, dtype=np.int32)
    js = np.zeros((n_rays, n_max), dtype=np.int32)
    fs = np.zeros((n_rays, n_max), dtype=np.int32)
    ties = np.zeros(n_rays, dtype=np.int32)
    rc = lib().orc_march_rays(*grid.args(), _p(cams, ctypes.c_double), int(cams.shape[0]),
                              _p(r, ctypes.c_uint32), n_rays, f32(delta), n_max, _p(cnt, ctypes.c_int32),
                              _p(js, ctypes.c_int32), _p(fs, ctypes.c_int32), _p(ties, ctypes.c_int32))
    if rc:
        raise ValueError("orc_march_rays rejected its arguments")
    return cnt, js, fs, ties


def render(grid: Grid, weights, affine, W: int, H: int, sigma_scale: float, cams16,
           rays: Optional[np.ndarray], delta: float, n_max: int, t_stop: float = 1e-4,
           bg=(0.0, 0.0, 0.0), act: int = 0, quant: int = 0, widths=None):
    """Renders (view, pixel) rays, or every pixel of every view (rays=None).
    Returns a dict of per-ray arrays.  quant=1 takes the FP8 E4M3 reading of
    the matrix layers.  widths (int per field) gives every field its own MLP
    width; weights is then the fields' parameters one after another."""
    cams = cams_f32(cams16)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    aff = np.ascontiguousarray(affine, dtype=np.float32)
    wd = np.ascontiguousarray(widths, dtype=np.int32) if widths is not None else None
    n_fields = int(aff.shape[0])
    n_rays = int(rays.shape[0]) if rays is not None else int(sum(c[1] * c[2] for c in cams))
    r = np.ascontiguousarray(rays, dtype=np.uint32) if rays is not None else None
    bgv = np.array([f32(b) for b in bg], dtype=np.float64)
    out = dict(rgb=np.zeros((n_rays, 3)), depth=np.zeros(n_rays), opacity=np.zeros(n_rays),
               n_kept=np.zeros(n_rays, np.int32), n_used=np.zeros(n_rays, np.int32),
               ties=np.zeros(n_rays, np.int32), margin=np.zeros(n_rays))
    rc = lib().orc_render(*grid.args(), _p(w, ctypes.c_float), _p(aff, ctypes.c_float), W, H, act,
                          f32(sigma_scale), int(quant), _p(wd, ctypes.c_int32), n_fields,
                          _p(cams, ctypes.c_double), int(cams.shape[0]),
                          _p(r, ctypes.c_uint32), n_rays, f32(delta), n_max, f32(t_stop),
                          _p(bgv, ctypes.c_double), _p(out["rgb"], ctypes.c_double),
                          _p(out["depth"], ctypes.c_double), _p(out["opacity"], ctypes.c_double),
                          _p(out["n_kept"], ctypes.c_int32), _p(out["n_used"], ctypes.c_int32),
                          _p(out["ties"], ctypes.c_int32), _p(out["margin"], ctypes.c_double))
    if rc:
        raise ValueError("orc_render rejected its arguments")
    return out


def render_records(grid: Grid, weights, affine, W: int, H: int, sigma_scale: float, cams16,
                   rays: Optional[np.ndarray], counts, js, fields, delta: float, t_stop: float = 1e-4,
                   bg=(0.0, 0.0, 0.0), act: int = 0, quant: int = 0, widths=None):
    """Eq. 4-5 over a GIVEN kept-sample set per ray (counts [n], js and fields
    [n, stride]) instead of the oracle's own march: the plain composite of
    another march's records.  Returns a dict like render() (rgb, depth,
    opacity, n_used, margin)."""
    cams = cams_f32(cams16)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    aff = np.ascontiguousarray(affine, dtype=np.float32)
    wd = np.ascontiguousarray(widths, dtype=np.int32) if widths is not None else None
    n_fields = int(aff.shape[0])
    cnt = np.ascontiguousarray(counts, dtype=np.int32)
    n_rays = int(cnt.shape[0])
    jj = np.ascontiguousarray(js, dtype=np.int32).reshape(n_rays, -1)
    ff = np.ascontiguousarray(fields, dtype=np.int32).reshape(n_rays, -1)
    stride = int(jj.shape[1])
    r = np.ascontiguousarray(rays, dtype=np.uint32) if rays is not None else None
    bgv = np.array([f32(b) for b in bg], dtype=np.float64)
    out = dict(rgb=np.zeros((n_rays, 3)), depth=np.zeros(n_rays), opacity=np.zeros(n_rays),
               n_used=np.zeros(n_rays, np.int32), margin=np.zeros(n_rays))
    if n_rays == 0:
        return out
    rc = lib().orc_render_records(*grid.args(), _p(w, ctypes.c_float), _p(aff, ctypes.c_float), W, H, act,
                                  f32(sigma_scale), int(quant), _p(wd, ctypes.c_int32), n_fields,
                                  _p(cams, ctypes.c_double), int(cams.shape[0]), _p(r, ctypes.c_uint32), n_rays,
                                  f32(delta), f32(t_stop), _p(bgv, ctypes.c_double), _p(cnt, ctypes.c_int32),
                                  _p(jj, ctypes.c_int32), _p(ff, ctypes.c_int32), stride,
                                  _p(out["rgb"], ctypes.c_double), _p(out["depth"], ctypes.c_double),
                                  _p(out["opacity"], ctypes.c_double), _p(out["n_used"], ctypes.c_int32),
                                  _p(out["margin"], ctypes.c_double))
    if rc:
        raise ValueError("orc_render_records rejected its arguments")
    return out


def sample_tie_distance(grid: Grid, cams16, rays: Optional[np.ndarray], q_ray, q_j, delta: float) -> np.ndarray:
    """Distance (voxel units) from sample q_j[k] of ray q_ray[k] to the nearest
    face of its voxel whose two sides differ; inf if none does."""
    cams = cams_f32(cams16)
    qr = np.ascontiguousarray(q_ray, dtype=np.int64)
    qj = np.ascontiguousarray(q_j, dtype=np.int32)
    r = np.ascontiguousarray(rays, dtype=np.uint32) if rays is not None else None
    dist = np.zeros(qr.size)
    rc = lib().orc_sample_tie_distance(*grid.args(), _p(cams, ctypes.c_double), int(cams.shape[0]),
                                       _p(r, ctypes.c_uint32), int(qr.size),
                                       qr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _p(qj, ctypes.c_int32),
                                       f32(delta), _p(dist, ctypes.c_double))
    if rc:
        raise ValueError("orc_sample_tie_distance rejected its arguments")
    return dist


def loss_grad(grid: Grid, weights, affine, W: int, H: int, sigma_scale: float, cams16, rays,
              target, delta: float, n_max: int, t_stop: float = 1e-4, bg=(0.0, 0.0, 0.0),
              want_grad: bool = True, loss_norm: Optional[float] = None, act: int = 0):
    """Mean-squared photometric loss over the rays and its gradient w.r.t.
    every weight ([F][P] float64).  Returns (loss, grad or None, signature,
    rendered rgb)."""
    cams = cams_f32(cams16)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    n_fields = int(w.shape[0])
    aff = np.ascontiguousarray(affine, dtype=np.float32)
    r = np.ascontiguousarray(rays, dtype=np.uint32)
    n_rays = int(r.shape[0])
    tg = np.ascontiguousarray(target, dtype=np.float32)
    bgv = np.array([f32(b) for b in bg], dtype=np.float64)
    grad = np.zeros(w.shape, dtype=np.float64) if want_grad else None
    sig = np.zeros(1, dtype=np.uint64)
    rgb = np.zeros((n_rays, 3))
    norm = float(loss_norm) if loss_norm is not None else 3.0 * n_rays
    loss = lib().orc_loss_grad(*grid.args(), _p(w, ctypes.c_float), _p(aff, ctypes.c_float), n_fields, W, H,
                               act, f32(sigma_scale), _p(cams, ctypes.c_double), int(cams.shape[0]),
                               _p(r, ctypes.c_uint32), n_rays, f32(delta), n_max, f32(t_stop),
                               _p(bgv, ctypes.c_double), _p(tg, ctypes.c_float), norm,
                               _p(grad, ctypes.c_double), _p(sig, ctypes.c_uint64), _p(rgb, ctypes.c_double))
    if not np.isfinite(loss):
        raise ValueError("orc_loss_grad failed")
    return float(loss), grad, int(sig[0]), rgb


def rays_touching(grid: Grid, cams16, rays, delta: float, n_max: int, field: int) -> np.ndarray:
    cams = cams_f32(cams16)
    r = np.ascontiguousarray(rays, dtype=np.uint32)
    mask = np.zeros(r.shape[0], dtype=np.uint8)
    lib().orc_rays_touching(*grid.args(), _p(cams, ctypes.c_double), int(cams.shape[0]), _p(r, ctypes.c_uint32),
                            int(r.shape[0]), f32(delta), n_max, field, _p(mask, ctypes.c_uint8))
    return mask.astype(bool)


def adam(w, m, v, g, lr: float, step: int, b1: float = 0.9, b2: float = 0.99, eps: float = 1e-8):
    """One Adam step in FP64 on copies; returns (w, m, v)."""
    w = np.array(w, dtype=np.float64).ravel().copy()
    m = np.array(m, dtype=np.float64).ravel().copy()
    v = np.array(v, dtype=np.float64).ravel().copy()
    g = np.ascontiguousarray(np.array(g, dtype=np.float64).ravel())
    lib().orc_adam(int(w.size), _p(w, ctypes.c_double), _p(m, ctypes.c_double), _p(v, ctypes.c_double),
                   _p(g, ctypes.c_double), lr, b1, b2, eps, int(step))
    return w, m, v


# occupancy parameters: p_hit, p_miss, l_min, l_max, p_occ, a_min
OCC_DEFAULT = (0.7, 0.4, -2.0, 3.5, 0.97, 0.5)


def segment_voxels(dims, origin, vox: float, o, d, t_end: float) -> np.ndarray:
    """Linear indices (x fastest) of the voxels whose interior o + t d,
    0 < t < t_end, crosses, in traversal order."""
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    org = np.ascontiguousarray(origin, dtype=np.float64)
    o = np.ascontiguousarray(o, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    cap = 4 * int(dims.sum()) + 16
    out = np.zeros(cap, dtype=np.int64)
    n = lib().orc_segment_voxels(_p(dims, ctypes.c_int32), _p(org, ctypes.c_double), float(vox),
                                 _p(o, ctypes.c_double), _p(d, ctypes.c_double), float(t_end),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap)
    if n < 0:
        raise ValueError("segment crosses too many voxels")
    return out[:n].copy()


def occupancy_update(dims, origin, vox: float, logit: np.ndarray, cams16, depth, opacity, params=OCC_DEFAULT):
    """Eq. 6 over one scan per camera (in order).  logit: float64 [n_voxels],
    updated in place.  Returns (occupancy bits u32 [n_voxels / 32],
    near-tie count)."""
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    org = np.ascontiguousarray([f32(v) for v in origin], dtype=np.float64)
    cams = cams_f32(cams16)
    dep = np.ascontiguousarray(depth, dtype=np.float32)
    opa = np.ascontiguousarray(opacity, dtype=np.float32)
    prm = np.ascontiguousarray(params, dtype=np.float64)
    assert logit.dtype == np.float64 and logit.flags.c_contiguous
    bits = np.zeros(int(np.prod(dims)) // 32, dtype=np.uint32)
    ties = ctypes.c_int64(0)
    rc = lib().orc_occupancy_update(_p(dims, ctypes.c_int32), _p(org, ctypes.c_double), f32(vox),
                                    _p(logit, ctypes.c_double), _p(cams, ctypes.c_double), int(cams.shape[0]),
                                    _p(dep, ctypes.c_float), _p(opa, ctypes.c_float), _p(prm, ctypes.c_double),
                                    _p(bits, ctypes.c_uint32), ctypes.byref(ties))
    if rc:
        raise ValueError("orc_occupancy_update rejected its arguments")
    return bits, int(ties.value)


def assign_fields(dims, occ_linear: np.ndarray, n: int) -> np.ndarray:
    """Alg. 1 stage II: network id (int32) of every occupied voxel, the
    voxels given by their linear indices (x fastest) in increasing order."""
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    idx = np.ascontiguousarray(occ_linear, dtype=np.int64)
    out = np.zeros(idx.size, dtype=np.int32)
    rc = lib().orc_assign_fields(_p(dims, ctypes.c_int32), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 int(idx.size), int(n), _p(out, ctypes.c_int32))
    if rc:
        raise ValueError("orc_assign_fields rejected its arguments")
    return out


def teacher_param_count() -> int:
    return int(lib().orc_teacher_param_count())


def teacher_eval(weights, aff_global, p, d, quant: int = 0) -> np.ndarray:
    """The global 360NeRF at points p [n, 3] with directions d [n, 3]:
    (sigma, r, g, b) per point.  quant=2 takes the BF16 reading (BF16
    inputs and weights of the matrix layers but the density head and layer
    11; the bias of layers 1, 5 and 10 rounded too)."""
    w = np.ascontiguousarray(weights, dtype=np.float32)
    a = np.ascontiguousarray(np.asarray(aff_global, dtype=np.float32), dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((p.shape[0], 4))
    lib().orc_teacher_eval(_p(w, ctypes.c_float), _p(a, ctypes.c_double), int(p.shape[0]), _p(p, ctypes.c_double),
                           _p(d, ctypes.c_double), _p(out, ctypes.c_double), int(quant))
    return out


def distill_loss_grad(weights, affine, W: int, H: int, sigma_scale: float, p, d, field, target, I: float,
                      act: int = 0):
    """Eq. 7 summed over fields: (loss, gradient [F, P]) of the students."""
    w = np.ascontiguousarray(weights, dtype=np.float32)
    aff = np.ascontiguousarray(affine, dtype=np.float32)
    F_ = int(aff.shape[0])
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    fl = np.ascontiguousarray(field, dtype=np.int32)
    t = np.ascontiguousarray(target, dtype=np.float64).reshape(-1, 4)
    P = param_count(W, H)
    g = np.zeros((F_, P))
    loss = lib().orc_distill_loss_grad(_p(w, ctypes.c_float), _p(aff, ctypes.c_float), F_, W, H, act,
                                       f32(sigma_scale), int(p.shape[0]), _p(p, ctypes.c_double),
                                       _p(d, ctypes.c_double), _p(fl, ctypes.c_int32), _p(t, ctypes.c_double),
                                       float(I), _p(g, ctypes.c_double))
    return float(loss), g


def bf16(x: float) -> float:
    """Nearest BF16 value (ties to even)."""
    return lib().orc_bf16(float(x))


def mlp_grad_points(weights, affine, W: int, H: int, sigma_scale: float, p, d, field, dl, act: int = 0,
                    quant: int = 0):
    """The MLP adjoint at points for given output gradients dl [n, 4]:
    (gradient [F, P], smallest |ReLU pre-activation| per sample).  quant=2
    takes the BF16 reading of the forward pass and the adjoint."""
    w = np.ascontiguousarray(weights, dtype=np.float32)
    aff = np.ascontiguousarray(affine, dtype=np.float32)
    F_ = int(aff.shape[0])
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    fl = np.ascontiguousarray(field, dtype=np.int32)
    g_out = np.ascontiguousarray(dl, dtype=np.float64).reshape(-1, 4)
    g = np.zeros((F_, param_count(W, H)))
    margin = np.zeros(p.shape[0])
    lib().orc_mlp_grad_points(_p(w, ctypes.c_float), _p(aff, ctypes.c_float), F_, W, H, act, f32(sigma_scale),
                              int(quant), int(p.shape[0]), _p(p, ctypes.c_double), _p(d, ctypes.c_double),
                              _p(fl, ctypes.c_int32), _p(g_out, ctypes.c_double), _p(g, ctypes.c_double),
                              _p(margin, ctypes.c_double))
    return g, margin

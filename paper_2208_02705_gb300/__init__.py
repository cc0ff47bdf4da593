"""Python binding of the roam C ABI (``include/roam.h``): argument marshalling
only.  Every step of the render and training path runs in the CUDA kernels
of ``libroam.so``; PyTorch supplies device memory and streams.

There is no CPU fallback: importing works without a GPU (so that the library
can be inspected), but creating a context needs the built library and a
GB300, and every failure raises ``RoamError``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libroam.so")

ROAM_F32, ROAM_BF16, ROAM_FP8 = 0, 1, 2
ROAM_EQUIRECT, ROAM_PERSPECTIVE = 0, 1
ROAM_SOFTPLUS, ROAM_RELU = 0, 1

STATUS = {0: "ROAM_OK", -1: "ROAM_ERR_ARG", -2: "ROAM_ERR_OOM", -3: "ROAM_ERR_CUDA", -4: "ROAM_ERR_STATE",
          -5: "ROAM_ERR_TIMEOUT", -6: "ROAM_ERR_DATA", -7: "ROAM_ERR_UNSUPPORTED"}

# every entry point declared in include/roam.h
ENTRY_POINTS = ("roam_create", "roam_destroy", "roam_last_error", "roam_check", "roam_load_grid",
                "roam_load_fields", "roam_load_weights", "roam_load_weights_mixed", "roam_get_weights", "roam_render",
                "roam_get_stats", "roam_tune_round_size", "roam_occupancy_update", "roam_assign_fields", "roam_teacher_load", "roam_teacher_eval",
                "roam_distill_loss", "roam_mlp_backward", "roam_march", "roam_bucket", "roam_mlp_eval", "roam_composite", "roam_train_forward",
                "roam_train_backward", "roam_adam_step", "roam_profile", "roam_profile_read",
                "roam_bucket_static", "roam_l2_loss", "roam_set_tile_padding", "roam_selftest_wait_timeout")


class RoamError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class roam_grid_desc(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("origin", ctypes.c_float * 3), ("vox", ctypes.c_float)]


class roam_mlp_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("n_hidden", ctypes.c_int32), ("sigma_scale", ctypes.c_float),
                ("density_act", ctypes.c_int32)]


class roam_camera(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fov_h", ctypes.c_float), ("R", ctypes.c_float * 9), ("o", ctypes.c_float * 3)]


class roam_occ_params(ctypes.Structure):
    _fields_ = [("p_hit", ctypes.c_float), ("p_miss", ctypes.c_float), ("l_min", ctypes.c_float),
                ("l_max", ctypes.c_float), ("p_occ", ctypes.c_float), ("a_min", ctypes.c_float)]


def occ_params(p_hit: float = 0.7, p_miss: float = 0.4, l_min: float = -2.0, l_max: float = 3.5,
               p_occ: float = 0.97, a_min: float = 0.5) -> roam_occ_params:
    q = roam_occ_params()
    q.p_hit, q.p_miss, q.l_min, q.l_max, q.p_occ, q.a_min = p_hit, p_miss, l_min, l_max, p_occ, a_min
    return q


class roam_render_opts(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_float), ("n_max", ctypes.c_int32), ("t_stop", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("precision", ctypes.c_int32), ("round_size", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("first_round_size", ctypes.c_int32)]


class roam_stats(ctypes.Structure):
    _fields_ = [("n_rays", ctypes.c_int64), ("n_samples", ctypes.c_int64), ("n_used", ctypes.c_int64),
                ("n_rounds", ctypes.c_int32), ("n_fields_hit", ctypes.c_int32)]


class roam_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class roam_adam_cfg(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("step", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libroam.so (build it with ``paper_2208_02705_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RoamError(-7, f"{path} is missing: build the CUDA library first "
                            "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    P = ctypes.POINTER
    L.roam_create.argtypes = [P(vp), i32]
    L.roam_destroy.argtypes = [vp]
    L.roam_last_error.restype = ctypes.c_char_p
    L.roam_check.argtypes = [vp]
    L.roam_load_grid.argtypes = [vp, P(roam_grid_desc), vp, i32]
    L.roam_load_fields.argtypes = [vp, i32, vp, i64, vp, i32]
    L.roam_load_weights.argtypes = [vp, P(roam_mlp_desc), vp, i32]
    L.roam_load_weights_mixed.argtypes = [vp, P(roam_mlp_desc), vp, vp, i32]
    L.roam_tune_round_size.argtypes = [vp, vp, i32, P(roam_render_opts), vp, vp, vp, vp]
    L.roam_occupancy_update.argtypes = [vp, vp, i32, vp, vp, P(roam_occ_params), vp, vp, vp]
    L.roam_assign_fields.argtypes = [vp, i32, vp, vp, vp]
    L.roam_teacher_load.argtypes = [vp, vp, vp, i32]
    L.roam_teacher_eval.argtypes = [vp, vp, vp, i64, i32, vp, vp]
    L.roam_distill_loss.argtypes = [vp, vp, vp, i64, ctypes.c_float, vp, vp, vp]
    L.roam_mlp_backward.argtypes = [vp, vp, vp, vp, i64, i32, vp, vp, vp]
    L.roam_get_weights.argtypes = [vp, vp, i32]
    L.roam_render.argtypes = [vp, P(roam_camera), i32, P(roam_render_opts), vp, vp, vp, i32, vp]
    L.roam_get_stats.argtypes = [vp, P(roam_stats)]
    L.roam_march.argtypes = [vp, P(roam_camera), i32, vp, i64, P(roam_render_opts), vp, vp, vp]
    L.roam_bucket.argtypes = [vp, vp, i64, vp, vp, vp]
    L.roam_mlp_eval.argtypes = [vp, vp, vp, vp, i64, i32, vp, vp]
    L.roam_composite.argtypes = [vp, i64, i32, vp, vp, vp, P(roam_render_opts), vp, vp, vp, vp, vp]
    L.roam_train_forward.argtypes = [vp, P(roam_camera), i32, vp, i64, P(roam_render_opts), vp, vp]
    L.roam_train_backward.argtypes = [vp, vp, vp, vp]
    L.roam_adam_step.argtypes = [vp, vp, P(roam_adam_cfg), vp]
    L.roam_bucket_static.argtypes = [vp, i64, i32, vp, vp, vp]
    L.roam_l2_loss.argtypes = [vp, vp, vp, i64, ctypes.c_float, vp, vp, vp]
    L.roam_set_tile_padding.argtypes = [vp, i32]
    L.roam_selftest_wait_timeout.argtypes = [vp, ctypes.c_uint64, P(ctypes.c_int32), vp]
    L.roam_profile.argtypes = [vp, i32]
    L.roam_profile_read.argtypes = [vp, P(roam_kernel_time), i32, P(ctypes.c_int)]
    for name in ENTRY_POINTS:
        if name != "roam_last_error":
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise RoamError(status, load_library().roam_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream=None) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def camera_struct(cam) -> roam_camera:
    """From any object with model, width, height, fov_h, R (3x3), o (3)."""
    c = roam_camera()
    c.model = int(cam.model)
    c.width = int(cam.width)
    c.height = int(cam.height)
    c.fov_h = float(cam.fov_h)
    R = np.asarray(cam.R, dtype=np.float32).reshape(9)
    o = np.asarray(cam.o, dtype=np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.o[i] = float(o[i])
    return c


def camera_array(cams: Sequence) -> ctypes.Array:
    arr = (roam_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera_struct(c)
    return arr


def render_opts(delta: float, n_max: int, t_stop: float = 1e-4, bg=(0.0, 0.0, 0.0),
                precision: int = ROAM_F32, round_size: int = 0, use_graph: bool = False,
                first_round_size: int = 0) -> roam_render_opts:
    o = roam_render_opts()
    o.delta = float(delta)
    o.n_max = int(n_max)
    o.t_stop = float(t_stop)
    for i in range(3):
        o.bg[i] = float(bg[i])
    o.precision = int(precision)
    o.round_size = int(round_size)
    o.use_graph = int(bool(use_graph))
    o.first_round_size = int(first_round_size)
    return o


class Roam:
    """One roam context on one CUDA device.  Methods mirror the C entry
    points (roam_<name>) and take torch tensors on that device."""

    def __init__(self, device: int = 0):
        self.L = load_library()
        self.device = device
        h = ctypes.c_void_p()
        _check(self.L.roam_create(ctypes.byref(h), device))
        self.h = h
        self.n_pixels = 0
        self.fwd_gen = 0            # counts train_forward calls (the state train_backward consumes)
        self._wkey = None           # (pointer, version, shape) of the weight tensor last loaded, if any

    def close(self):
        if getattr(self, "h", None):
            self.L.roam_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self):
        import torch
        return torch.device("cuda", self.device)

    # ---- scene ----
    def load_grid(self, bits, dims, origin, vox):
        d = roam_grid_desc()
        for i in range(3):
            d.dims[i] = int(dims[i])
            d.origin[i] = float(origin[i])
        d.vox = float(vox)
        on_dev = not isinstance(bits, np.ndarray)
        if not on_dev:
            bits = np.ascontiguousarray(bits, dtype=np.uint32)
        _check(self.L.roam_load_grid(self.h, ctypes.byref(d), _ptr(bits), int(on_dev)))
        host_bits = bits if not on_dev else bits.cpu().numpy()
        self.n_occupied = int(np.unpackbits(np.ascontiguousarray(host_bits).view(np.uint8)).sum())
        self.dims = tuple(int(x) for x in dims)

    def load_fields(self, field_of_rank, affine):
        on_dev = not isinstance(field_of_rank, np.ndarray)
        if not on_dev:
            field_of_rank = np.ascontiguousarray(field_of_rank, dtype=np.uint16)
            affine = np.ascontiguousarray(affine, dtype=np.float32)
        n_fields = int(affine.shape[0])
        _check(self.L.roam_load_fields(self.h, n_fields, _ptr(field_of_rank), int(field_of_rank.shape[0]),
                                       _ptr(affine), int(on_dev)))
        self.n_fields = n_fields

    def load_weights(self, weights, W: int, H: int, sigma_scale: float, act: int = ROAM_SOFTPLUS):
        d = roam_mlp_desc()
        d.width, d.n_hidden, d.sigma_scale, d.density_act = int(W), int(H), float(sigma_scale), int(act)
        on_dev = not isinstance(weights, np.ndarray)
        if not on_dev:
            weights = np.ascontiguousarray(weights, dtype=np.float32)
        _check(self.L.roam_load_weights(self.h, ctypes.byref(d), _ptr(weights), int(on_dev)))
        self.W, self.H = W, H
        self.sigma_scale, self.act = float(sigma_scale), int(act)
        self.P = int(weights.shape[-1])
        self.n_params = self.P * self.n_fields
        self._wkey = None

    def sync_weights(self, weights):
        """Loads a device float32 tensor [n_fields, P] (layout of
        roam_load_weights) as the FP32 masters unless it is the tensor last
        loaded this way and unchanged since: same storage, same version
        counter (in-place updates under torch.no_grad(), as torch.optim makes
        them, advance it)."""
        import torch
        key = (weights.data_ptr(), weights._version, tuple(weights.shape))
        if key != self._wkey:
            if tuple(weights.shape) != (self.n_fields, self.P) or weights.dtype != torch.float32:
                raise RoamError(-1, f"weights must be float32 [{self.n_fields}, {self.P}]")
            self.load_weights(weights.detach().contiguous(), self.W, self.H, self.sigma_scale, self.act)
            self._wkey = key

    def load_weights_mixed(self, weights, widths, H: int, sigma_scale: float, act: int = ROAM_SOFTPLUS):
        """weights: the fields' parameters one after another (1-D), field f in
        the layout of width widths[f]."""
        d = roam_mlp_desc()
        d.width, d.n_hidden, d.sigma_scale, d.density_act = 0, int(H), float(sigma_scale), int(act)
        wd = np.ascontiguousarray(widths, dtype=np.int32)
        on_dev = not isinstance(weights, np.ndarray)
        if not on_dev:
            weights = np.ascontiguousarray(weights, dtype=np.float32).reshape(-1)
        _check(self.L.roam_load_weights_mixed(self.h, ctypes.byref(d), _ptr(wd), _ptr(weights), int(on_dev)))
        self.W, self.H = 0, H
        self.P = None
        self.n_params = int(weights.numel() if on_dev else weights.size)

    def get_weights(self):
        """FP32 masters: [n_fields, P] for one width, 1-D (field after field) when mixed."""
        import torch
        out = torch.empty(self.n_params, dtype=torch.float32, device=self._dev())
        _check(self.L.roam_get_weights(self.h, _ptr(out), 1))
        return out.view(self.n_fields, self.P) if self.P else out

    def load_workload(self, wl):
        """Loads grid, fields and weights of a fixtures.Workload."""
        self.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
        self.load_fields(wl.part.field_of_rank, wl.affine)
        if getattr(wl, "widths", None) is not None:
            self.load_weights_mixed(wl.weights, wl.widths, wl.H, wl.sigma_scale)
        else:
            self.load_weights(wl.weights, wl.W, wl.H, wl.sigma_scale)

    # ---- rendering ----
    def render(self, cams, opts: roam_render_opts, rgb=None, depth=None, opacity=None, stream=None):
        """Device outputs; returns (rgb [N,3], depth [N], opacity [N])."""
        import torch
        arr = camera_array(cams)
        n = sum(int(c.width) * int(c.height) for c in cams)
        dev = self._dev()
        rgb = rgb if rgb is not None else torch.empty((n, 3), dtype=torch.float32, device=dev)
        depth = depth if depth is not None else torch.empty(n, dtype=torch.float32, device=dev)
        opacity = opacity if opacity is not None else torch.empty(n, dtype=torch.float32, device=dev)
        _check(self.L.roam_render(self.h, arr, len(cams), ctypes.byref(opts), _ptr(rgb), _ptr(depth),
                                  _ptr(opacity), 1, _stream(stream)))
        return rgb, depth, opacity

    def render_host(self, cams, opts: roam_render_opts, rgb: np.ndarray, depth=None, opacity=None, stream=None):
        """Host outputs (pinned or pageable numpy arrays); synchronises."""
        arr = camera_array(cams)
        _check(self.L.roam_render(self.h, arr, len(cams), ctypes.byref(opts), _ptr(rgb), _ptr(depth),
                                  _ptr(opacity), 0, _stream(stream)))
        return rgb, depth, opacity

    def render_host_ptrs(self, cams_arr, n_views, opts, rgb_ptr, depth_ptr, op_ptr, stream_handle):
        _check(self.L.roam_render(self.h, cams_arr, n_views, ctypes.byref(opts), rgb_ptr, depth_ptr, op_ptr, 0,
                                  stream_handle))

    def tune_round_size(self, cams, opts: roam_render_opts, stream=None):
        """roam_tune_round_size: (best round size, best first-round size, its
        render time in ms)."""
        arr = camera_array(cams)
        best = ctypes.c_int32()
        best0 = ctypes.c_int32()
        ms = ctypes.c_float()
        _check(self.L.roam_tune_round_size(self.h, arr, len(cams), ctypes.byref(opts), ctypes.byref(best),
                                           ctypes.byref(best0), ctypes.byref(ms), _stream(stream)))
        return int(best.value), int(best0.value), float(ms.value)

    def occupancy_update(self, cams, depth, opacity, logit, bits=None, params=None, stream=None):
        """roam_occupancy_update: one scan per camera of (depth, opacity)
        device tensors; logit (device float, one per voxel) is updated in
        place; bits (device int32 words) receives the occupancy grid."""
        arr = camera_array(cams)
        q = params if params is not None else occ_params()
        _check(self.L.roam_occupancy_update(self.h, arr, len(cams), _ptr(depth), _ptr(opacity), ctypes.byref(q),
                                            _ptr(logit), _ptr(bits), _stream(stream)))
        return logit, bits

    def assign_fields(self, n_fields: int, stream=None):
        """roam_assign_fields (Alg. 1 stage II) on the loaded grid: returns
        (labels int16 [S] device, boxes int32 [n_fields, 6] device)."""
        import torch
        n_occ = self.n_occupied
        labels = torch.empty(n_occ, dtype=torch.int16, device=self._dev())
        boxes = torch.empty((n_fields, 6), dtype=torch.int32, device=self._dev())
        _check(self.L.roam_assign_fields(self.h, int(n_fields), _ptr(labels), _ptr(boxes), _stream(stream)))
        return labels, boxes

    # ---- distillation from the global 360NeRF (Eq. 7) ----
    def teacher_load(self, weights, affine):
        on_dev = not isinstance(weights, np.ndarray)
        if not on_dev:
            weights = np.ascontiguousarray(weights, dtype=np.float32)
        aff = np.ascontiguousarray(affine, dtype=np.float32)
        _check(self.L.roam_teacher_load(self.h, _ptr(weights), _ptr(aff), int(on_dev)))

    def teacher_eval(self, p, d, precision=None, stream=None):
        import torch
        n = int(p.shape[0])
        out = torch.empty((n, 4), dtype=torch.float32, device=self._dev())
        _check(self.L.roam_teacher_eval(self.h, _ptr(p), _ptr(d), n, ROAM_F32 if precision is None else int(precision),
                                        _ptr(out), _stream(stream)))
        return out

    def distill_loss(self, student, teacher, I: float, stream=None):
        import torch
        n = int(student.shape[0])
        dl = torch.empty_like(student)
        loss = torch.empty(1, dtype=torch.float32, device=self._dev())
        _check(self.L.roam_distill_loss(self.h, _ptr(student), _ptr(teacher), n, float(I), _ptr(dl), _ptr(loss),
                                        _stream(stream)))
        return loss, dl

    def mlp_backward(self, p, d, field, dl_dout, precision=ROAM_F32, stream=None):
        import torch
        grad = torch.empty((self.n_fields, self.P), dtype=torch.float32, device=self._dev())
        _check(self.L.roam_mlp_backward(self.h, _ptr(p), _ptr(d), _ptr(field), int(p.shape[0]), int(precision),
                                        _ptr(dl_dout), _ptr(grad), _stream(stream)))
        return grad

    def distill_step(self, p, d, field, I: float, lr: float, step: int, teacher_out=None, precision=None,
                     teacher_precision=None, stream=None):
        """One distillation step (Eq. 7): teacher targets (computed unless
        given), student outputs (FP32 by default), loss and its gradient,
        the adjoint in the same precision (FP32 SIMT or BF16 tcgen05) and
        Adam.  Returns the loss (device tensor)."""
        prec = ROAM_F32 if precision is None else precision
        t = teacher_out if teacher_out is not None else self.teacher_eval(p, d, teacher_precision, stream=stream)
        sdt = self.mlp_eval(p, d, field, prec, stream=stream)
        loss, dl = self.distill_loss(sdt, t, I, stream=stream)
        g = self.mlp_backward(p, d, field, dl, precision=prec, stream=stream)
        self.adam_step(g, lr=lr, step=step, stream=stream)
        return loss

    def get_stats(self) -> roam_stats:
        s = roam_stats()
        _check(self.L.roam_get_stats(self.h, ctypes.byref(s)))
        return s

    def check(self):
        _check(self.L.roam_check(self.h))

    def selftest_wait_timeout(self, limit_ns: int, stream=None) -> int:
        """roam_selftest_wait_timeout: the status (ROAM_ERR_TIMEOUT = -5 when the
        bounded-wait path works) of one MLP launch whose weight image is
        withheld, every wait limited to limit_ns."""
        obs = ctypes.c_int32(0)
        _check(self.L.roam_selftest_wait_timeout(self.h, int(limit_ns), ctypes.byref(obs), _stream(stream)))
        return int(obs.value)

    def set_tile_padding(self, tiles: int):
        """roam_set_tile_padding: pad every field's tile run to a multiple of
        `tiles` (0: each kernel's own tiles in flight)."""
        _check(self.L.roam_set_tile_padding(self.h, int(tiles)))

    def profile(self, enable: bool):
        _check(self.L.roam_profile(self.h, int(bool(enable))))

    def profile_read(self) -> dict:
        arr = (roam_kernel_time * 16)()
        n = ctypes.c_int()
        _check(self.L.roam_profile_read(self.h, arr, 16, ctypes.byref(n)))
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}

    # ---- single steps ----
    def march(self, cams, opts: roam_render_opts, rays=None, stream=None):
        import torch
        arr = camera_array(cams)
        n = int(rays.shape[0]) if rays is not None else sum(int(c.width) * int(c.height) for c in cams)
        dev = self._dev()
        count = torch.empty(n, dtype=torch.int32, device=dev)
        recs = torch.empty((n, opts.n_max), dtype=torch.int32, device=dev)
        _check(self.L.roam_march(self.h, arr, len(cams), _ptr(rays), n, ctypes.byref(opts), _ptr(count), _ptr(recs),
                                 _stream(stream)))
        return count, recs

    def bucket(self, keys, stream=None):
        import torch
        n = int(keys.shape[0])
        perm = torch.empty(n, dtype=torch.int32, device=self._dev())
        offsets = torch.empty(self.n_fields + 1, dtype=torch.int32, device=self._dev())
        _check(self.L.roam_bucket(self.h, _ptr(keys), n, _ptr(perm), _ptr(offsets), _stream(stream)))
        return perm, offsets

    def mlp_eval(self, p, d, field, precision: int = ROAM_F32, stream=None):
        import torch
        n = int(p.shape[0])
        out = torch.empty((n, 4), dtype=torch.float32, device=self._dev())
        _check(self.L.roam_mlp_eval(self.h, _ptr(p), _ptr(d), _ptr(field), n, int(precision), _ptr(out),
                                    _stream(stream)))
        return out

    def composite(self, count, sigma_rgb, t, opts: roam_render_opts, stream=None):
        import torch
        n, n_max = int(sigma_rgb.shape[0]), int(sigma_rgb.shape[1])
        dev = self._dev()
        rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
        depth = torch.empty(n, dtype=torch.float32, device=dev)
        op = torch.empty(n, dtype=torch.float32, device=dev)
        used = torch.empty(n, dtype=torch.int32, device=dev)
        _check(self.L.roam_composite(self.h, n, n_max, _ptr(count), _ptr(sigma_rgb), _ptr(t), ctypes.byref(opts),
                                     _ptr(rgb), _ptr(depth), _ptr(op), _ptr(used), _stream(stream)))
        return rgb, depth, op, used

    # ---- training ----
    def train_forward(self, cams, rays, opts: roam_render_opts, rgb=None, stream=None):
        import torch
        arr = camera_array(cams)
        n = int(rays.shape[0])
        rgb = rgb if rgb is not None else torch.empty((n, 3), dtype=torch.float32, device=self._dev())
        _check(self.L.roam_train_forward(self.h, arr, len(cams), _ptr(rays), n, ctypes.byref(opts), _ptr(rgb),
                                         _stream(stream)))
        self.fwd_gen += 1
        return rgb

    def train_backward(self, dl_drgb, grad=None, stream=None):
        import torch
        grad = grad if grad is not None else torch.empty((self.n_fields, self.P), dtype=torch.float32,
                                                         device=self._dev())
        _check(self.L.roam_train_backward(self.h, _ptr(dl_drgb), _ptr(grad), _stream(stream)))
        return grad

    def l2_loss(self, rgb, target, norm: float, stream=None):
        """(loss tensor [1], dl/drgb tensor [n, 3]) of sum (rgb - target)^2 / norm."""
        import torch
        n = int(rgb.shape[0])
        dl = torch.empty_like(rgb)
        loss = torch.zeros(1, dtype=torch.float32, device=rgb.device)
        _check(self.L.roam_l2_loss(self.h, _ptr(rgb), _ptr(target), n, float(norm), _ptr(dl), _ptr(loss),
                                   _stream(stream)))
        return loss, dl

    def local_grad(self, cams, rays, target, opts, norm: float, stream=None):
        """Forward, L2 loss (normalised by `norm`) and backward on this
        process's rays: returns (loss [1], gradient [F, P])."""
        rgb = self.train_forward(cams, rays, opts, stream=stream)
        loss, dl = self.l2_loss(rgb, target, norm, stream=stream)
        grad = self.train_backward(dl, stream=stream)
        return loss, grad

    def adam_step(self, grad, lr: float, step: int, beta1: float = 0.9, beta2: float = 0.99, eps: float = 1e-8,
                  stream=None):
        c = roam_adam_cfg()
        c.lr, c.beta1, c.beta2, c.eps, c.step = float(lr), float(beta1), float(beta2), float(eps), int(step)
        _check(self.L.roam_adam_step(self.h, _ptr(grad), ctypes.byref(c), _stream(stream)))


def bucket_static(keys, n_fields: int, stream=None):
    """roam_bucket_static: bucketing without a context and without any device
    allocation by the library (its scratch is a fixed device array).  keys is
    a device int16/uint16 tensor; returns (perm, offsets) tensors, which this
    Python helper allocates through torch -- a caller that must not allocate
    passes its own buffers to the C entry point instead."""
    import torch
    if keys.dtype not in (torch.int16, getattr(torch, "uint16", torch.int16)) or not keys.is_contiguous():
        raise RoamError(-1, "keys must be a contiguous int16 or uint16 tensor")
    L = load_library()
    n = int(keys.shape[0])
    # the C entry point works on the current device: make it the keys' device
    with torch.cuda.device(keys.device):
        perm = torch.empty(n, dtype=torch.int32, device=keys.device)
        offsets = torch.empty(n_fields + 1, dtype=torch.int32, device=keys.device)
        s = stream if stream is not None else torch.cuda.current_stream(keys.device)
        _check(L.roam_bucket_static(_ptr(keys), n, int(n_fields), _ptr(perm), _ptr(offsets), s.cuda_stream))
    return perm, offsets


def render_function():
    """torch.autograd.Function over the training forward/backward entry
    points (the hand-written adjoint of compositing, MLPs and encodings).

    ``RoamRender.apply(weights, roam, cams, rays, opts)`` returns rgb [n, 3]
    for the rays (int32 [n, 2] (view, pixel), on the device).  ``weights`` is a
    device float32 tensor [n_fields, P] in the layout of roam_load_weights;
    the forward loads it into the context whenever it is not the tensor last
    loaded or has changed since (Roam.sync_weights), so the render always
    uses the tensor's current values, and the backward returns d(loss)/d
    weights from roam_train_backward.  The context keeps the state of one
    forward only: a backward whose forward has been followed by another
    forward on the same context raises instead of returning that later
    forward's gradient."""
    import torch

    class RoamRender(torch.autograd.Function):
        @staticmethod
        def forward(ctx_, weights, roam: Roam, cams, rays, opts):
            roam.sync_weights(weights)
            rgb = roam.train_forward(cams, rays, opts)
            ctx_.roam = roam
            ctx_.gen = roam.fwd_gen
            ctx_.shape = tuple(weights.shape)
            return rgb

        @staticmethod
        def backward(ctx_, grad_rgb):
            if ctx_.roam.fwd_gen != ctx_.gen:
                raise RuntimeError("RoamRender.backward: another forward ran on this context since this "
                                   "one; its saved state is gone (run backward before the next forward)")
            grad = ctx_.roam.train_backward(grad_rgb.contiguous())
            return grad.view(ctx_.shape), None, None, None, None

    return RoamRender

"""Render parity rule: compares a renderer's output with the FP64 oracle ray
by ray, on the renderer's own sample records.

TEST INFRASTRUCTURE ONLY (the tests, ``__graft_entry__.smoke()`` and the
benchmark's accuracy check use it).  It takes the renderer's records and
images as numpy arrays and calls nothing but ``oracle``; the renderer is
never imported here.

The rule (integer work bit-exact, colours held to a bar on every ray):

* A ray whose kept-sample list (sample index j and field id of each kept
  sample) equals the oracle's own march is compared with the oracle's
  render of that ray.
* A ray whose list differs is a mismatch.  It is certified when every
  sample index at which the two lists disagree lies within ``TIE_EPS``
  voxel of a face whose two sides differ (occupancy or field): such a
  sample may land on either side of the face under the renderer's FP32
  coordinates.  Where both lists hit the sample cap, the samples past the
  earlier list's last index are the cap's consequence of an earlier
  difference, not differences of their own.  Certified mismatches are
  counted (the caller bounds their share); their colours are compared with
  the oracle recomputed on the renderer's own list (``render_records``),
  by the same bar.
* A ray whose transmittance crosses the stopping threshold within
  ``TERM_MARGIN`` (|ln(T / t_stop)|) of it may terminate one sample
  earlier or later; that sample weighs at most t_stop, so its bar is
  widened by t_stop (the truncation bound of Eq. 5 with early stopping).

``TIE_EPS`` = 1e-3 voxel: the renderer's sample coordinates are FP32,
fma(t, d / vox, (o - origin) / vox) with t = (j + 1/2) delta, and its
empty-space jumps compare FP32 exit distances; their rounding is a few
units of 2^-24 relative to |t d / vox| + |o - origin| / vox, i.e. up to
about 3e-4 voxel on a 512^3 grid (a chord of ~900 voxels).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import render, render_records, march_rays, sample_tie_distance

TIE_EPS = 1e-3
TERM_MARGIN = 1e-3


def differing_samples(cg: int, jg, fg, co: int, jo, fo, n_max: int):
    """Sample indices at which two kept-sample lists disagree (present in
    one only, or with different fields), less the cap's tail."""
    g = {int(j): int(f) for j, f in zip(jg[:cg], fg[:cg])}
    o = {int(j): int(f) for j, f in zip(jo[:co], fo[:co])}
    diff = sorted(set(g) ^ set(o) | {j for j in set(g) & set(o) if g[j] != o[j]})
    if cg == n_max and co == n_max and cg > 0:
        last = min(int(jg[cg - 1]), int(jo[co - 1]))
        diff = [j for j in diff if j <= last]
    return diff


@dataclass
class RenderParity:
    n: int
    n_equal: int
    certified: list = field(default_factory=list)      # ray indices: mismatches certified as near-ties
    uncertified: list = field(default_factory=list)    # ray indices: mismatches without a certificate
    term_ties: int = 0
    err: Optional[np.ndarray] = None                   # per-ray max |rgb - reference|
    bar: Optional[np.ndarray] = None                   # per-ray colour bar
    ref_rgb: Optional[np.ndarray] = None               # the reference each ray is held to
    err_depth: Optional[np.ndarray] = None
    err_opacity: Optional[np.ndarray] = None
    max_tie_distance: float = 0.0                      # largest face distance among certified samples

    @property
    def max_err(self) -> float:
        return float(self.err.max()) if self.err is not None and self.err.size else 0.0

    @property
    def over(self) -> np.ndarray:
        return np.nonzero(self.err > self.bar)[0]

    def psnr(self, got) -> float:
        mse = float(((np.asarray(got, np.float64) - self.ref_rgb) ** 2).mean())
        return 10 * math.log10(1.0 / mse) if mse > 0 else float("inf")

    def summary(self) -> dict:
        return {"rays": self.n, "records_equal": self.n_equal, "certified_mismatches": len(self.certified),
                "uncertified_mismatches": len(self.uncertified), "termination_ties": int(self.term_ties),
                "max_abs": self.max_err, "over_bar": int(self.over.size),
                "max_tie_distance_vox": self.max_tie_distance}


def check_march(grid, cams16, rays, delta: float, n_max: int, gpu_cnt, gpu_recs):
    """Record lists of the renderer (count [n], recs [n, n_max] = j | field << 16)
    against the oracle's march: (oracle march tuple, RenderParity without colours)."""
    cnt_o, js_o, fs_o, _ = march_rays(grid, cams16, rays, delta, n_max)
    cnt_g = np.asarray(gpu_cnt).astype(np.int64)
    recs = np.asarray(gpu_recs).astype(np.int64) & 0xFFFFFFFF
    js_g = recs & 0xFFFF
    fs_g = recs >> 16
    n = int(cnt_o.shape[0])
    rep = RenderParity(n=n, n_equal=0)
    q_ray, q_j, owner = [], [], []
    for r in range(n):
        c = int(cnt_g[r])
        if c == cnt_o[r] and np.array_equal(js_g[r, :c], js_o[r, :c]) and np.array_equal(fs_g[r, :c], fs_o[r, :c]):
            rep.n_equal += 1
            continue
        diff = differing_samples(c, js_g[r], fs_g[r], int(cnt_o[r]), js_o[r], fs_o[r], n_max)
        if not diff:                 # cap tail only (cannot happen alone)
            rep.uncertified.append(r)
            continue
        for j in diff:
            q_ray.append(r)
            q_j.append(j)
            owner.append(r)
    if q_ray:
        dist = sample_tie_distance(grid, cams16, rays, np.array(q_ray), np.array(q_j), delta)
        worst = {}
        for r, dd in zip(owner, dist):
            worst[r] = max(worst.get(r, 0.0), float(dd))
        for r, dd in sorted(worst.items()):
            if dd < TIE_EPS:
                rep.certified.append(r)
                rep.max_tie_distance = max(rep.max_tie_distance, dd)
            else:
                rep.uncertified.append(r)
    rep.uncertified.sort()
    return (cnt_o, js_o, fs_o), rep, (cnt_g, js_g, fs_g)


def check_render(grid, weights, affine, W: int, H: int, sigma_scale: float, cams16, rays, delta: float, n_max: int,
                 gpu_cnt, gpu_recs, rgb, depth=None, opacity=None, tol: float = 1e-4, t_stop: float = 1e-4,
                 bg=(0.0, 0.0, 0.0), act: int = 0, quant: int = 0, widths=None, ref=None) -> RenderParity:
    """Colours (and depth/opacity when given) of the rays `rays` (None: every
    pixel of every view) against the oracle under the rule above.  gpu_cnt /
    gpu_recs: the renderer's kept-sample lists of the same rays (its march
    with the same options).  ref: the oracle's own render of these rays, if
    already computed."""
    if ref is None:
        ref = render(grid, weights, affine, W, H, sigma_scale, cams16, rays, delta, n_max, t_stop, bg, act, quant,
                     widths)
    _, rep, (cnt_g, js_g, fs_g) = check_march(grid, cams16, rays, delta, n_max, gpu_cnt, gpu_recs)
    n = rep.n
    ref_rgb = np.array(ref["rgb"], dtype=np.float64, copy=True)
    ref_depth = np.array(ref["depth"], dtype=np.float64, copy=True)
    ref_op = np.array(ref["opacity"], dtype=np.float64, copy=True)
    margin = np.array(ref["margin"], dtype=np.float64, copy=True)
    mism = sorted(rep.certified + rep.uncertified)
    if mism:
        idx = np.array(mism, dtype=np.int64)
        sub_rays = rays[idx] if rays is not None else None
        if sub_rays is None:
            # every pixel: name the mismatched rays by (view, pixel)
            cams = np.asarray(cams16, dtype=np.float64).reshape(-1, 16)
            sizes = (cams[:, 1] * cams[:, 2]).astype(np.int64)
            starts = np.concatenate([[0], np.cumsum(sizes)])
            view = np.searchsorted(starts, idx, side="right") - 1
            sub_rays = np.stack([view, idx - starts[view]], 1).astype(np.uint32)
        rr = render_records(grid, weights, affine, W, H, sigma_scale, cams16, sub_rays, cnt_g[idx], js_g[idx],
                            fs_g[idx], delta, t_stop, bg, act, quant, widths)
        ref_rgb[idx] = rr["rgb"]
        ref_depth[idx] = rr["depth"]
        ref_op[idx] = rr["opacity"]
        margin[idx] = np.minimum(margin[idx], rr["margin"])
    term = margin < TERM_MARGIN
    rep.term_ties = int(term.sum())
    rep.ref_rgb = ref_rgb
    rep.err = np.abs(np.asarray(rgb, dtype=np.float64).reshape(n, 3) - ref_rgb).max(axis=1)
    rep.bar = np.where(term, tol + t_stop, tol)
    # one sample more or less at a termination tie moves depth by at most
    # t_stop times that sample's t, bounded by the ray's last kept sample
    last_j = np.where(cnt_g > 0, js_g[np.arange(n), np.maximum(cnt_g - 1, 0)], 0)
    t_last = (last_j + 0.5) * delta
    if depth is not None:
        rep.err_depth = np.abs(np.asarray(depth, np.float64) - ref_depth) - np.where(term, t_stop * t_last, 0.0)
    if opacity is not None:
        rep.err_opacity = np.abs(np.asarray(opacity, np.float64) - ref_op) - np.where(term, t_stop, 0.0)
    return rep

"""Stereoscopic roaming (the real-time roaming mode of Sec. "Real-time
Rendering Speedup", shown in monoscopic and stereoscopic form): every frame
renders the two eye views of the current pose in one call, replayed as a
CUDA graph, and the per-frame latency is what matters.  The headset display
itself is not part of this library (no graphics stack): frames stay in
device buffers.

Eye views: the pose's camera translated by -ipd/2 and +ipd/2 along its own
x axis (camera frame x right, y down, z forward), same orientation.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

import numpy as np


def stereo_pair(cam, ipd: float = 0.064):
    """(left, right) copies of `cam` (any object with R [3x3 camera-to-world]
    and o [3]) moved by -ipd/2 and +ipd/2 along the camera's x axis."""
    R = np.asarray(cam.R, dtype=np.float64)
    x = R[:, 0]
    left = dataclasses.replace(cam, o=np.asarray(cam.o, dtype=np.float64) - 0.5 * ipd * x)
    right = dataclasses.replace(cam, o=np.asarray(cam.o, dtype=np.float64) + 0.5 * ipd * x)
    return left, right


def roam_frames(engine, poses: Sequence, opts, ipd: float = 0.064, stream=None):
    """Renders both eyes of every pose (one call per frame) and returns the
    per-frame device time in ms (CUDA events on `stream`) and the last
    frame's (left, right) colour buffers."""
    import torch
    times: List[float] = []
    n = poses[0].width * poses[0].height
    rgb = torch.empty((2 * n, 3), dtype=torch.float32, device="cuda")
    depth = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    op = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    for cam in poses:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        eyes = stereo_pair(cam, ipd)
        a.record(st)
        engine.render(list(eyes), opts, rgb=rgb, depth=depth, opacity=op, stream=st)
        b.record(st)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return times, (rgb[:n], rgb[n:])

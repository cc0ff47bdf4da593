"""Bit-repeatability of the tensor-core renders, and independence from the
tile padding: every field's run of 128-sample tiles is padded to a multiple
of its MLP kernel's tiles in flight, and roam_set_tile_padding pads further
(a multiple of 4), so that kernels meet groups of tiles in which no slot has
work -- after field changes, at the end of a CTA's range, in the sparse
later rounds.  The padding tiles hold no samples, so the rendered bits must
not change, whatever the padding and however often the render repeats.
Cases: single widths 32, 64 and 128 (the four- and two-tile kernels) with
extra padding, and the mixed-width sets 64+128 and 32+128, 1000 renders
each (plain and graph-replayed), every render equal to the first bit for
bit, composited-sample counts included."""
import dataclasses

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


@pytest.fixture(scope="module")
def floor8():
    return F.floor384(specs=F.multiview_specs()[:8])


def _ctx(roam, wl, widths):
    r = roam.Roam(0)
    r.load_grid(wl.scene.bits, wl.scene.dims, wl.scene.origin, wl.scene.vox)
    r.load_fields(wl.part.field_of_rank, wl.affine)
    if len(set(widths.tolist())) == 1:
        W = int(widths[0])
        r.load_weights(F.xavier_weights(4, F.ROLE_TEACHER, wl.part.n_fields, W, wl.H), W, wl.H, wl.sigma_scale)
    else:
        r.load_weights_mixed(F.xavier_weights_mixed(4, F.ROLE_TEACHER, widths, wl.H), widths, wl.H, wl.sigma_scale)
    return r


def _repeat(roam, r, wl, n, pad=None, ref=None, prec=None):
    prec = roam.ROAM_BF16 if prec is None else prec
    opts = roam.render_opts(wl.delta, wl.n_max, precision=prec)
    gopts = roam.render_opts(wl.delta, wl.n_max, precision=prec, use_graph=True)
    if pad is not None:
        r.set_tile_padding(pad)
    if ref is None:
        ref = [x.clone() for x in r.render(wl.cams, opts)]
        torch.cuda.synchronize()
        ref.append(r.get_stats().n_used)
    bad = []
    for it in range(n):
        out = r.render(wl.cams, gopts if it % 2 else opts)
        torch.cuda.synchronize()
        same = all(torch.equal(a, b) for a, b in zip(ref[:3], out)) and r.get_stats().n_used == ref[3]
        if not same:
            bad.append(it)
    r.check()
    return ref, bad


@pytest.mark.parametrize("W,prec,pads,n", [(128, "bf16", (4, 8, 16), 300), (64, "bf16", (8, 16), 150),
                                           (32, "bf16", (8, 16), 150), (128, "fp8", (4, 8), 100),
                                           (64, "fp8", (8,), 100)])
def test_tile_padding_changes_no_bit(roam, floor8, W, prec, pads, n):
    """Padding 8 at W = 128 (three all-empty groups after every field's
    single tile in the sparse later rounds, CTA ranges starting inside
    them) once let about one render in a hundred differ: a slot read the
    weight image of a field change before it had landed."""
    p = roam.ROAM_BF16 if prec == "bf16" else roam.ROAM_FP8
    r = _ctx(roam, floor8, np.full(floor8.part.n_fields, W, np.int32))
    ref, bad = _repeat(roam, r, floor8, 20, prec=p)
    assert not bad, bad
    for pad in pads:
        _, bad = _repeat(roam, r, floor8, n, pad=pad, ref=ref, prec=p)
        assert not bad, (pad, len(bad), bad[:10])
    r.set_tile_padding(0)
    r.close()


@pytest.mark.parametrize("widths", [(64, 128), (32, 128)])
def test_mixed_width_renders_repeat_bit_for_bit(roam, floor8, widths):
    w = F.mixed_widths(4, floor8.part.n_fields, widths)
    r = _ctx(roam, floor8, w)
    _, bad = _repeat(roam, r, floor8, 1000)
    assert not bad, (len(bad), bad[:10])
    r.close()

"""Host planning on the CPU (rtc_plan_slices, rtc_plan_ingest): the slice cut of
the asymmetric allocation and the persistent loop's per-block ingest table,
checked against their definitions by brute force."""
import numpy as np
import pytest

import synth
from paper_1805_07254_gb300.rtc import RtcError, RTC_EINVAL, plan_ingest, plan_slices


def _cfg(name):
    return {"tiny": synth.tiny_scao, "elt": synth.elt_scao}[name]()


@pytest.mark.parametrize("name", ["tiny", "elt"])
@pytest.mark.parametrize("bands", [0, 1])
def test_without_a_readout_the_slices_are_equal(name, bands):
    cfg = _cfg(name)
    nt = cfg.n_valid
    g0 = plan_slices(cfg.subaps, cfg.nsub, cfg.npx, cfg.nact, "f32", 152, bands, 10.0)
    S = min(152, nt)
    assert np.array_equal(g0, (nt * np.arange(S + 1)) // S)


@pytest.mark.parametrize("store", ["f32", "bf16", "fp8"])
def test_cut_for_a_rolling_readout(store):
    """ELT, 74 bands of one subaperture row each, 10 us apart: valid bounds, at
    most 152 slices, none wider than twice the mean, the subapertures of the last
    band in slices of their own, and the early rows in wider slices than the late."""
    cfg = _cfg("elt")
    nt, S = cfg.n_valid, 152
    g0 = plan_slices(cfg.subaps, cfg.nsub, cfg.npx, cfg.nact, store, S, 74, 10.0)
    w = np.diff(g0)
    assert g0[0] == 0 and g0[-1] == nt and len(w) <= S and np.all(w >= 1)
    assert w.max() <= -(-2 * nt // S)
    last_row = cfg.subaps[:, 0].max()
    slice_of = np.repeat(np.arange(len(w)), w)
    for gi in np.nonzero(cfg.subaps[:, 0] == last_row)[0]:
        assert w[slice_of[gi]] == 1
    assert w[: len(w) // 2].mean() > 4 * w[-10:].mean()


def test_cut_rejects_bad_arguments():
    cfg = _cfg("tiny")
    for kw in ({"store": "f32", "bands": -1}, {"store": "f32", "bands": cfg.frame_side + 1},
               {"store": "f32", "band_interval_us": -1.0}):
        with pytest.raises(RtcError) as e:
            plan_slices(cfg.subaps, cfg.nsub, cfg.npx, cfg.nact, **kw)
        assert e.value.code == RTC_EINVAL
    bad = cfg.subaps.copy()
    bad[3, 1] = cfg.nsub
    with pytest.raises(RtcError):
        plan_slices(bad, cfg.nsub, cfg.npx, cfg.nact)


def _pixel_bytes(cfg, gis, n_wfs=1):
    """Byte offsets of every pixel of subapertures gis (w * n_valid + i) in the
    uint16 frame [n_wfs][H][W]."""
    H = cfg.frame_side
    nv = cfg.n_valid
    out = []
    for gi in gis:
        w, i = divmod(int(gi), nv)
        r, c = cfg.subaps[i]
        y = w * H + r * cfg.npx + np.arange(cfg.npx)
        x = c * cfg.npx + np.arange(cfg.npx)
        out.append(((y[:, None] * H + x[None, :]) * 2).ravel())
    return np.concatenate(out) if out else np.zeros(0, np.int64)


@pytest.mark.parametrize("name,blocks,unit,bands", [
    ("elt", 152, 16, 74), ("elt", 40, 16, 7), ("tiny", 52, 4, 3), ("tiny", 13, 2, 64)])
def test_ingest_units_are_exactly_the_blocks_pixels(name, blocks, unit, bands):
    """Each block's units are sorted, distinct, and exactly the units that hold a
    pixel of its subapertures; its band is the one holding its last pixel row."""
    cfg = _cfg(name)
    g0 = plan_slices(cfg.subaps, cfg.nsub, cfg.npx, cfg.nact, "f32", 152, bands, 10.0 if name == "elt" else 0.0)
    S = len(g0) - 1
    blocks = min(blocks, S)                   # a launch has at most one block per slice
    blk, units = plan_ingest(cfg.subaps, cfg.nsub, cfg.npx, g0, blocks, unit, bands)
    H = cfg.frame_side
    assert blk[0, 0] == 0 and blk[-1, 1] == len(units)
    for b in range(blocks):
        u = units[blk[b, 0]:blk[b, 1]]
        assert np.all(np.diff(u.astype(np.int64)) > 0)
        gis = np.arange(g0[S * b // blocks], g0[S * (b + 1) // blocks])
        px = _pixel_bytes(cfg, gis)
        assert np.array_equal(u, np.unique(px // unit).astype(np.uint32))
        assert u.max() < H * H * 2 // unit
        last = max(cfg.subaps[gi % cfg.n_valid, 0] for gi in gis) * cfg.npx + cfg.npx - 1
        j = blk[b, 2]
        assert (H * j) // bands <= last < (H * (j + 1)) // bands


def test_ingest_with_two_wfs_and_a_cut():
    cfg = _cfg("tiny")
    g0 = plan_slices(cfg.subaps, cfg.nsub, cfg.npx, cfg.nact, "bf16", 40, 8, 5.0, n_wfs=2)
    assert g0[-1] == 2 * cfg.n_valid
    blk, units = plan_ingest(cfg.subaps, cfg.nsub, cfg.npx, g0, len(g0) - 1, 16, 8, n_wfs=2)
    covered = np.concatenate([units[blk[b, 0]:blk[b, 1]] for b in range(len(g0) - 1)])
    px = _pixel_bytes(cfg, np.arange(2 * cfg.n_valid), n_wfs=2)
    assert set(np.unique(px // 16).tolist()) <= set(covered.tolist())


def test_ingest_rejects_bad_slices():
    cfg = _cfg("tiny")
    nt = cfg.n_valid
    for g0 in (np.array([0, 10, 10, nt]), np.array([0, 20, nt - 1]), np.array([1, 20, nt])):
        with pytest.raises(RtcError) as e:
            plan_ingest(cfg.subaps, cfg.nsub, cfg.npx, g0, 2, 16, 1)
        assert e.value.code == RTC_EINVAL
    with pytest.raises(RtcError):
        plan_ingest(cfg.subaps, cfg.nsub, cfg.npx, np.array([0, nt]), 1, 8, 1)   # unit 8 is not offered

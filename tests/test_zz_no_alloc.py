"""The allocation-free reconstruction entry point against the handle-based one.

Some users of this library cannot call cudaMalloc: a hard-real-time control
thread must not enter the CUDA allocator (which may synchronise the device and
block for an unbounded time) inside its loop, and a plugin inside a larger RTC
framework may receive every device buffer from that framework.  For them
rtc_mvm_integrate_noalloc runs the reconstruction + leaky integrator with its
split-K scratch in a static device array.  These tests check, through the C ABI,
that it gives the same DM commands as rtc_reconstruct_async (within the 1e-5
relative-RMS tolerance of the FP32 path) on two calls in a row, and that it
rejects sizes beyond its fixed scratch.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

import synth
from helpers import rel_rms

pytestmark = pytest.mark.gpu

DM_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_noalloc_matches_handle_path_on_two_calls(store):
    from paper_1805_07254_gb300 import Rtc
    from paper_1805_07254_gb300.rtc import mvm_integrate_noalloc

    cfg = synth.elt_scao()
    nact, ns = cfg.nact, cfg.nslopes
    kpad = (ns + 15) // 16 * 16
    ksplit = 4
    M = synth.control_matrix(cfg).numpy()
    rng = np.random.default_rng(0)
    slopes = [(0.3 * rng.standard_normal(ns)).astype(np.float32) for _ in range(2)]
    dev = torch.device("cuda:0")

    r = Rtc(cfg.nsub, cfg.npx, nact, obs=cfg.obs, gain=cfg.gain, leak=cfg.leak)
    r.load_cmat(M, store=store)

    # caller-owned buffers in the stored layout: [nact][kpad], zero padded
    Mp = torch.zeros((nact, kpad), dtype=torch.float32)
    Mp[:, :ns] = torch.from_numpy(M)
    Md = Mp.to(dev) if store == "f32" else Mp.to(dev).to(torch.bfloat16)
    d_s = torch.zeros(kpad, dtype=torch.float32, device=dev)
    d_a = torch.zeros(nact, dtype=torch.float32, device=dev)
    d_dm = torch.empty(nact, dtype=torch.float32, device=dev)
    d_ref = torch.empty(nact, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    for s in slopes:
        d_s[:ns] = torch.from_numpy(s).to(dev)
        r.reconstruct_async(d_s, d_ref, stream=st)
        mvm_integrate_noalloc(Md, store, None, nact, kpad, d_s, d_a, d_dm, cfg.gain, cfg.leak,
                              ksplit, stream=st)
        torch.cuda.synchronize()
        ref = d_ref.cpu().numpy()
        got = d_dm.cpu().numpy()
        assert rel_rms(got, ref) <= DM_TOL
        np.testing.assert_array_equal(d_a.cpu().numpy(), got)
    r.close()


def _stored_codes(M, store, kpad):
    """The caller's buffers for a stored type: [nact][kpad] codes (zero padded) and row
    scales (FP8 and INT8), from the oracle's quantisers."""
    from oracle import quant as Q
    nact, ns = M.shape
    scales = None
    if store == "f32":
        codes = torch.zeros((nact, kpad), dtype=torch.float32)
        codes[:, :ns] = torch.from_numpy(M)
    elif store == "fp8":
        q, scales = Q.fp8_row_quantise(M)
        codes = torch.zeros((nact, kpad), dtype=torch.float8_e4m3fn)
        codes[:, :ns] = torch.from_numpy(q).float().to(torch.float8_e4m3fn)
    else:
        q, scales = Q.int8_row_quantise(M)
        codes = torch.zeros((nact, kpad), dtype=torch.int8)
        codes[:, :ns] = torch.from_numpy(q.astype(np.int8))
    return codes, scales


@pytest.mark.parametrize("store", ["f32", "fp8", "int8"])
@pytest.mark.parametrize("ksplit", [1, 16])
def test_noalloc_matches_oracle_on_two_calls(store, ksplit):
    """Every stored type with its row scales, no split (no partials written) and the
    largest split the scratch holds, an odd actuator count (69): DM commands of two
    calls in a row against the FP64 oracle on the stored matrix."""
    from oracle import pipeline as P
    from oracle import quant as Q
    from paper_1805_07254_gb300.rtc import mvm_integrate_noalloc

    cfg = synth.tiny_scao()
    nact, ns = cfg.nact, cfg.nslopes
    kpad = (ns + 15) // 16 * 16
    M = synth.control_matrix(cfg).numpy()
    dev = torch.device("cuda:0")
    codes, scales = _stored_codes(M, store, kpad)
    d_M = codes.to(dev)
    d_sc = torch.from_numpy(scales).to(dev) if scales is not None else None
    Ms = Q.stored_matrix(M, store)
    rng = np.random.default_rng(1)
    d_s = torch.zeros(kpad, dtype=torch.float32, device=dev)
    d_a = torch.zeros(nact, dtype=torch.float32, device=dev)
    d_dm = torch.full((nact,), np.nan, dtype=torch.float32, device=dev)
    a_ref = np.zeros(nact)
    st = torch.cuda.current_stream()
    for _ in range(2):
        s = (0.3 * rng.standard_normal(ns)).astype(np.float32)
        d_s[:ns] = torch.from_numpy(s).to(dev)
        mvm_integrate_noalloc(d_M, store, d_sc, nact, kpad, d_s, d_a, d_dm, cfg.gain, cfg.leak,
                              ksplit, stream=st)
        torch.cuda.synchronize()
        a_ref = P.integrate(a_ref, P.reconstruct(Ms, s), cfg.gain, cfg.leak)
        got = d_dm.cpu().numpy()
        assert rel_rms(got, a_ref) <= DM_TOL, rel_rms(got, a_ref)
        np.testing.assert_array_equal(d_a.cpu().numpy(), got)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1805_07254_gb300.rtc import RtcError, RTC_EINVAL, mvm_integrate_noalloc
    dev = torch.device("cuda:0")
    big = 8193
    M = torch.zeros((big, 16), dtype=torch.float32, device=dev)
    s = torch.zeros(16, dtype=torch.float32, device=dev)
    a = torch.zeros(big, dtype=torch.float32, device=dev)
    with pytest.raises(RtcError) as e:
        mvm_integrate_noalloc(M, "f32", None, big, 16, s, a, None, 0.4, 0.99, 1)
    assert e.value.code == RTC_EINVAL and "8192" in str(e.value)
    with pytest.raises(RtcError) as e:
        mvm_integrate_noalloc(M, "f32", None, 100, 16, s, a, None, 0.4, 0.99, 17)
    assert e.value.code == RTC_EINVAL
    assert np.all(a.cpu().numpy() == 0)

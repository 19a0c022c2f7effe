"""Host-side helpers of bench.py that shape the JSON line: the e2e object's choice
between the resident and the per-call launch figure (the timing rule: no L2 flush is
possible while the kernel is resident, so that figure may lead only when the step's
inputs are larger than L2), the loop entries' L2 labels, and the recorded DRAM
traffic, which is reported only for the kernel sources it was captured from."""
import bench


class _Cfg:
    nact = 4421


def _stats(p50):
    return {"p50": p50, "p99": p50 + 2.0, "rms_jitter": 0.5}


INFO = {"frame_bytes": 1_095_200}


def test_resident_figure_leads_when_inputs_exceed_l2():
    e = bench.e2e_entry(_stats(49.0), _stats(37.4), True, INFO, _Cfg, 2000, 144_821_640, 126 << 20)
    assert e["value"] == 37.4 and e["mode"] == "resident kernel"
    assert e["launch_per_call"]["p50_us"] == 49.0 and e["resident"]["p50_us"] == 37.4
    assert e["h2d_bytes_per_step"] == 1_095_200 and e["d2h_bytes_per_step"] == 4 * 4421
    assert "not flushed" in e["resident"]["l2"] and "flushed" in e["launch_per_call"]["l2"]


def test_launch_figure_leads_when_inputs_fit_in_l2():
    e = bench.e2e_entry(_stats(33.0), _stats(30.0), False, INFO, _Cfg, 2000, 74_580_792, 126 << 20)
    assert e["value"] == 33.0 and e["mode"] == "one launch per call"
    assert e["resident"]["p50_us"] == 30.0


def test_loop_l2_labels():
    assert bench.matrix_l2_label(70 << 20, 0) == "resident"
    assert bench.matrix_l2_label(140 << 20, 0).startswith("streamed")
    assert bench.matrix_l2_label(35 << 20, 1).startswith("streamed (evict_first")


def test_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    dig = bench.kernel_source_digest()
    (prof / "dram_traffic.txt").write_text(
        "# comment\n"
        f"frame elt_f32 {dig} 148601344\n"
        "frame elt_bf16 0000000000000000 75821824\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the digest is taken over the package sources, which live under ROOT too
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: dig)
    assert bench.recorded_traffic("elt_f32") == 148601344.0
    assert bench.recorded_traffic("elt_bf16") is None      # captured from other sources
    assert bench.recorded_traffic("elt_fp8") is None       # never captured

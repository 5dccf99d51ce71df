"""Host logic of bench.py (no GPU): the ncu traffic lines it accepts, the algorithmic byte
model of the PCG kernels, and the roofline object built from per-kernel event times."""

import math

import pytest

import bench


def test_traffic_lines_need_the_current_fingerprint(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "a.md").write_text(
        "text\n"
        "```\n"
        "traffic: workload=w1 kernel=fft_lines loads=3 dram_bytes=1000 sources=cafe\n"
        "traffic: workload=w1 kernel=apply_K loads=3 dram_bytes=2000 sources=old0\n"
        "traffic: workload=w2 kernel=apply_K loads=1 dram_bytes=3000 sources=cafe\n"
        "```\n")
    (prof / "b.txt").write_text("`traffic: workload=w1 kernel=cg_p loads=3 dram_bytes=500 sources=cafe`\n")
    (prof / "c.ncu-rep").write_text("traffic: workload=w1 kernel=x loads=1 dram_bytes=1 sources=cafe\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_fingerprint", lambda: "cafe")
    got = bench.ncu_traffic("w1")
    assert got == {"fft_lines": (1000.0, 3, "a.md"), "cg_p": (500.0, 3, "b.txt")}
    assert bench.ncu_traffic("w2") == {"apply_K": (3000.0, 1, "a.md")}
    assert bench.ncu_traffic("w3") == {}


def test_traffic_lines_of_declared_equivalent_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "a.md").write_text("traffic: workload=w1 kernel=fft_lines loads=3 dram_bytes=1000 sources=old1\n"
                               "traffic: workload=w1 kernel=cg_p loads=3 dram_bytes=700 sources=old2\n")
    (prof / "eq.md").write_text("equivalent: sources=new0 captured=old1 reason=host-only\n"
                                "equivalent: sources=other captured=old2 reason=not-this-tree\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_fingerprint", lambda: "new0")
    assert bench.ncu_traffic("w1") == {"fft_lines": (1000.0, 3, "a.md")}
    monkeypatch.setattr(bench, "source_fingerprint", lambda: "new1")
    assert bench.ncu_traffic("w1") == {}


def test_fingerprint_changes_with_a_kernel_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2508_02613_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "include").mkdir()
    (tmp_path / "include" / "jfft.h").write_text("h")
    (tmp_path / "paper_2508_02613_gb300" / "build.py").write_text("b")
    (csrc / "k.cu").write_text("kernel 1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    a = bench.source_fingerprint()
    (csrc / "k.cu").write_text("kernel 2")
    b = bench.source_fingerprint()
    (csrc / "notes.txt").write_text("not a source")
    assert a != b and bench.source_fingerprint() == b and len(a) == 16


@pytest.mark.parametrize("shape", [(8, 16), (4, 8, 16)])
def test_byte_model_per_load(shape):
    """Compulsory bytes of one load: V = d N s per field, F = N / n_last (n_last / 2 + 1)
    complex frequencies, the J^1/2 factors N s."""
    d, N = len(shape), math.prod(shape)
    F = N // shape[-1] * (shape[-1] // 2 + 1)
    for s, sfx in ((8, ""), (4, "_f32")):
        V = d * N * s
        spec = d * F * 2 * s
        assert bench.traffic_bytes_per_unit("fft_rows_real_fwd" + sfx, shape) == V + spec + N * s
        assert bench.traffic_bytes_per_unit("fft_rows_real_fwd_xr" + sfx, shape) == 6 * V + spec + N * s
        assert bench.traffic_bytes_per_unit("fft_cols_real_inv" + sfx, shape) == spec + 2 * V + N * s
        assert bench.traffic_bytes_per_unit("cg_xr" + sfx, shape) == 6 * V
        assert bench.traffic_bytes_per_unit("cg_p" + sfx, shape) == 3 * V
        assert bench.traffic_bytes_per_unit("apply_K" + sfx, shape) == 2 * V + N * s
    assert bench.traffic_bytes_per_unit("apply_K_f32", shape, material_bytes=2) == 2 * d * N * 4 + 2 * N
    assert bench.traffic_bytes_per_unit("no_such_kernel", shape) is None


def test_roofline_picks_the_dominant_kernel(monkeypatch):
    monkeypatch.setattr(bench, "ncu_traffic", lambda w: {"fft_lines_f32": (123.0, 3, "p.md")})
    monkeypatch.setattr(bench, "hbm_peak_gbs", lambda: (5000.0, "measured"))
    shape = (64, 64)
    prof = {"apply_K_f32": (10, 2.0), "fft_lines_f32": (10, 3.0), "cg_p_f32": (10, 1.0), "stress": (1, 9.0)}
    r = bench.roofline(prof, 30, shape, False, "w")
    # "stress" has no byte model, so the FFT pass is the dominant modelled kernel
    assert r["kernel"] == "fft_lines_f32" and r["launches"] == 10 and r["traffic"] == 123.0
    byt = bench.traffic_bytes_per_unit("fft_lines_f32", shape)
    assert r["achieved"] == pytest.approx(30 * byt / 3.0e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0) and r["bound"] == "hbm"
    assert r["share"] == pytest.approx(3.0 / 15.0)
    alu = bench.roofline({"apply_K": (4, 2.0)}, 12, shape, True, "w")
    assert alu["bound"] == "alu" and alu["traffic"] is None
    assert alu["achieved"] == pytest.approx(12 * bench.flops_per_unit("apply_K", shape) / 2.0e-3 / 1e12)
    assert alu["frac"] == pytest.approx(alu["achieved"] / bench.FP64_PEAK_TFLOPS)
    every = bench.roofline(dict(prof, fft_rows_real_fwd_f32=(1, 0.5)), 30, shape, False, "w", every=True)
    # once-per-solve kernels (one launch here) are left out of the per-iteration list
    assert [r["kernel"] for r in every] == ["fft_lines_f32", "apply_K_f32", "cg_p_f32"]
    assert every[0]["frac"] == pytest.approx(r["frac"]) and all(0 < x["frac"] for x in every)

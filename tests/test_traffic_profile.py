"""The traffic profile that bench.py reads for roofline.traffic: its converter from the
raw page of an ncu report (units, per-launch means, per-pixel scaling, kernel names)
and the staleness rule (a profile whose source hash differs gives no figure)."""
import csv
import json

import bench

METRICS = ["dram__bytes_read.sum", "dram__bytes_write.sum", "gpu__time_duration.sum",
           "sm__pipe_alu_cycles_active.avg.pct_of_peak_sustained_active",
           "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active",
           "sm__issue_active.avg.pct_of_peak_sustained_elapsed",
           "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed",
           "sm__warps_active.avg.pct_of_peak_sustained_active", "launch__registers_per_thread",
           "smsp__inst_executed.sum", "smsp__inst_executed_pipe_alu.sum",
           "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active"]
UNITS = ["Mbyte", "Kbyte", "us", "%", "%", "%", "%", "%", "register/thread", "inst", "inst", "%"]


def _write_csv(path, rows, preamble=()):
    with open(path, "w", newline="") as f:
        for line in preamble:                 # ncu's log lines before the table
            f.write(line + "\n")
        w = csv.writer(f)
        w.writerow(["ID", "Kernel Name"] + METRICS)
        w.writerow(["", ""] + UNITS)
        for r in rows:
            w.writerow(r)


def test_converter_merges_captures_scales_and_averages(tmp_path):
    a, b = tmp_path / "raw_a.csv", tmp_path / "raw_b.csv"
    _write_csv(a, [
        ["0", "void rdhei::k_pass1<0, 0, 0>(rdhei::Batch)", "100", "500", "160", "84", "27", "75", "21", "53", "56",
         "4000", "3000", "0"],
        ["1", "void rdhei::k_pass1<0, 0, 0>(rdhei::Batch)", "300", "700", "170", "86", "27", "75", "21", "53", "56",
         "4000", "3000", "0"],
        ["3", "void rdhei::k_zero(uint4 *, unsigned int)", "1", "1", "5", "1", "1", "1", "1", "1", "30", "10", "1",
         "0"],
    ], preamble=["==PROF== Connected to process 1"])
    _write_csv(b, [
        ["0", "void rdhei::k_enc_fused<1, 0>(rdhei::Batch)", "20", "10", "150", "64", "15", "63", "38", "70", "64",
         "800", "500", "0"],
    ])
    out = tmp_path / "t.json"
    doc = bench.traffic_from_csv([str(a), str(b)], str(out), images=2, size=10)
    px = 2 * 10 * 10
    k = doc["kernels"]
    assert set(k) == {"pass1_keystream_hist", "enc_gather_embed"}        # uncaptured kernels ignored
    p = k["pass1_keystream_hist"]
    assert p["launches_captured"] == 2 and p["kernel"] == "k_pass1<0, 0, 0>"
    assert p["read_per_px"] == 200e6 / px and p["write_per_px"] == 600e3 / px    # Mbyte, Kbyte
    assert p["dram_bytes_per_px"] == (200e6 + 600e3) / px
    assert p["us_600"] == 165.0 and p["regs"] == 56
    assert p["inst_per_px"] == 4000 * 32 / px and p["alu_inst_per_px"] == 3000 * 32 / px   # warp -> thread
    assert k["enc_gather_embed"]["kernel"] == "k_enc_fused<1, 0>"
    assert doc["source_hash"] == bench.kernel_source_hash()
    assert json.loads(out.read_text()) == doc


def test_capture_recipe_is_one_small_capture_per_kernel():
    for kernel, cmd in bench.TRAFFIC_CAPTURE.items():
        assert "--clock-control none" in cmd and " -c 1 " in cmd and " -s " in cmd and "--set full" not in cmd
        assert kernel.split("<")[0] in cmd and "--kernels-only" in cmd and "--images 600" in cmd


def test_stale_profile_gives_no_traffic(tmp_path, monkeypatch):
    doc = {"source_hash": "0" * 16, "kernels": {"pass1_keystream_hist": {"dram_bytes_per_px": 2.0}}}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic_batch600x512.json").write_text(json.dumps(doc))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.measured_traffic("pass1_keystream_hist", 1000) == 2000.0
    assert bench.measured_traffic("enc_gather", 1000) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "1" * 16)
    assert bench.measured_traffic("pass1_keystream_hist", 1000) is None


def test_committed_profile_covers_the_captured_kernels():
    # (a stale hash is allowed here: bench.py then reports no traffic figure)
    with open(bench.os.path.join(bench.ROOT, "profiles", "dram_traffic_batch600x512.json")) as f:
        doc = json.load(f)
    assert set(doc["kernels"]) == set(bench.TRAFFIC_KERNELS.values())
    assert all(v["dram_bytes_per_px"] > 0 for v in doc["kernels"].values())

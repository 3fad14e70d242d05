"""Host-side helpers of the benchmark (no GPU): the kernel-code hash that ties the
reported DRAM traffic to the sources it was captured on, and the clock summary
that rejects throttled runs."""
import os
import shutil

import bench


def _copy_sources(tmp_path):
    dst = tmp_path / "paper_1801_06263_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_1801_06263_gb300", "csrc", f), dst / f)
    return dst


def test_code_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    dst = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._source_sha()
    f = dst / bench.KERNEL_SOURCES[0]
    text = f.read_text()
    f.write_text("// a new comment line\n\n/* and a block\n   comment */\n" + text.replace("\n", "  // trailing\n", 3))
    assert bench._source_sha() == h0
    f.write_text(text.replace("kDFold = 16", "kDFold = 17", 1))
    assert bench._source_sha() != h0


def test_clock_summary_flags_throttling(tmp_path):
    # nvidia-smi --format=csv,noheader,nounits rows of the query in Clocks.Q
    rows = ["0, 2070, 2070, 900.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1500, 2070, 1400.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 900.00, 0x0000000000000008, Active, Not Active, Not Active, Not Active"]
    c = bench.Clocks.__new__(bench.Clocks)
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    c.path = str(path)
    s = c.summary()
    assert s["sm_max_mhz"] == 2070.0 and s["sm_mhz"] == 2070.0 and s["samples"] == 3
    assert set(s["reasons"]) == {"sw_power_cap", "hw_slowdown"}


def test_roofs_come_from_the_device_and_the_sampled_clock(monkeypatch):
    import types

    import torch
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev: types.SimpleNamespace(multi_processor_count=76))
    r = bench.device_roofs(0, 1500.0)
    assert r["sms"] == 76 and r["sm_mhz"] == 1500.0
    assert abs(r["fp32_tflops"] - 76 * 128 * 2 * 1.5e9 / 1e12) < 1e-9
    assert abs(r["issue_per_s"] - 76 * 4 * 1.5e9) < 1.0
    assert abs(r["l1_tbps"] - 76 * 128 * 1.5e9 / 1e12) < 1e-9
    assert abs(r["l1_wavefronts_per_s"] - 76 * 1.5e9) < 1.0
    assert "76 SMs" in r["source"] and "1500 MHz" in r["source"]


def test_kept_ncu_counts_are_complete():
    """Every kept ncu figure names the kernel code it was taken on (the bench drops
    the figures whose source hash no longer matches)."""
    for k, v in bench.NCU_COUNTS.items():
        assert len(v["source_sha"]) == 16, k
        assert v["dram_bytes"] > 0 and v["warp_instructions"] > 0 and v["l1_wavefronts"] > 0

"""bench.py's output contract, on CPU: the reference arm (the oracle on a bounded sample) prints
one JSON line with the keys the driver reads, and the roofline bookkeeping (the 40-op count,
the derived integer-issue peak, the traffic record gated on the kernel sources) is consistent."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line(olib):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--workload", "flat16", "--ref-sweeps", "20"],
                         cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "attempts/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("flat16")


def test_roofline_bookkeeping():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.OPS_PER_ATTEMPT == 40 and bench.LANES_PER_SM == 128
    for name, rec in bench.NCU_RECORDS.items():
        assert set(rec) == {"sources", "sources_sha256", "bytes_per_launch", "inst_per_attempt", "pipes"}
        assert 0 < rec["pipes"]["issue_active"] <= 1 and 0 < rec["pipes"]["alu_pipe"] <= 1
        if rec["sources_sha256"] is not None:
            assert len(rec["sources_sha256"]) == 64
        valid = rec["sources_sha256"] == bench.kernel_sources_sha256(rec["sources"])
        assert bench.load_traffic(name) == (rec["bytes_per_launch"] if valid else None)
        assert bench.ncu_record(name, "inst_per_attempt") == (rec["inst_per_attempt"] if valid else None)
    # the roofline divides the 40-op algorithmic rate by 40 x the measured arithmetic-only attempt rate
    peaks = {"lop3_lane_ops_per_s": 40e12, "mix_lane_ops_per_s": 32e12, "philox_blocks_per_s": 1e12,
             "attempts_per_s_arithmetic": 2e12}
    r = bench.roofline(1e12, 2.0, peaks, 152, 2070.0, "k", {}, None, 27.0)
    assert r["bound"] == "alu" and r["unit"] == "Tops/s"
    assert abs(r["achieved"] - 40 * 0.5e12 / 1e12) < 1e-12
    assert abs(r["peak"] - 80.0) < 1e-12 and abs(r["frac"] - 20.0 / 80.0) < 1e-12
    c = r["ceilings"]
    assert abs(c["lane_issue_derived_Tops"] - 152 * 128 * 2070e6 / 1e12) < 1e-9
    assert abs(c["frac_of_philox_ceiling"] - 0.5e12 / 4e12) < 1e-12
    assert abs(c["frac_of_arithmetic_ceiling"] - 0.25) < 1e-12
    assert abs(c["frac_of_lop3_issue_by_instructions"] - 27.0 * 0.5e12 / 40e12) < 1e-12
    # a film on one 16-CTA cluster is also set against the ceiling of the 16 SMs it can use
    r = bench.roofline(1e12, 2.0, peaks, 152, 2070.0, "k", {"path": "resident", "ctas": 16}, None, None)
    c = r["ceilings"]
    assert c["sms_in_use"] == 16
    assert abs(c["frac_of_arithmetic_ceiling_of_sms_in_use"] - 0.25 * 152 / 16) < 1e-12
    assert "sms_in_use" not in bench.roofline(1e12, 2.0, peaks, 152, 2070.0, "k", {"path": "global", "ctas": 152},
                                              None, None)["ceilings"]
    # with the ncu pipe record: the attempts/s the kernel's own ALU work allows at a full ALU pipe
    r = bench.roofline(1e12, 2.0, peaks, 152, 2070.0, "k", {}, None, None, {"issue_active": 0.5, "alu_pipe": 0.4})
    c = r["ceilings"]
    assert c["ncu_alu_pipe_busy"] == 0.4 and abs(c["attempts_per_s_at_full_alu_pipe"] - 0.5e12 / 0.4) < 1e-3

"""Host logic of bench.py that needs no GPU: the ALU peak per SM clock, and the rule that the committed ncu
traffic is reported only while the kernel source still matches the hash recorded with it."""
import bench


def test_alu_peak_takes_the_binding_unit():
    """min(rsqrt rate / 2 per pair-eval, FP32 rate / 14 ops per pair-eval): with 28 rsqrt and 225 FP32 operations per
    SM clock (the rates measured at 64 warps per SM on GB300) the MUFU binds at 14 pair-evals per clock; a slower
    FP32 pipe takes over."""
    assert bench.peak_pairs_per_clk_sm(28.0, 225.0) == 14.0
    assert bench.peak_pairs_per_clk_sm(32.0, 140.0) == 10.0


def test_traffic_only_for_the_source_it_was_measured_on(monkeypatch):
    line = next(l for l in open(bench.os.path.join(bench.ROOT, "profiles", "sweep_kernel_plain_n16383.md"))
                if l.startswith("traffic_bytes_per_step:"))
    recorded_bytes, recorded_hash = int(line.split()[1]), line.split()[3]
    monkeypatch.setattr(bench, "source_hash", lambda: recorded_hash)
    assert bench.measured_traffic("plain_n16383") == recorded_bytes
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.measured_traffic("plain_n16383") is None
    assert bench.measured_traffic("no_such_workload") is None

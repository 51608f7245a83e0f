"""bench.py's profile bookkeeping (no GPU): the source fingerprint ignores comments and blank
lines but not code, and a profile's DRAM traffic is used only while its fingerprint matches."""
import os
import shutil

import bench

FILES = bench.SOURCE_FILES


def copy_tree(tmp_path):
    src = os.path.join(bench.ROOT, "paper_0908_4421_gb300", "csrc")
    dst = tmp_path / "paper_0908_4421_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in FILES:
        shutil.copy(os.path.join(src, f), dst / f)
    (tmp_path / "profiles").mkdir()
    return dst


def test_fingerprint_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    k = csrc / "kernels.cu"
    text = k.read_text()
    k.write_text("// a new comment line\n\n" + text.replace("\n", "  \n", 3) + "\n/* a block\n comment */\n")
    assert bench.kernel_source_hash() == h0
    k.write_text(text + "\nconstexpr int kUnusedProbe = 1;\n")
    assert bench.kernel_source_hash() != h0


def test_profiled_traffic_only_for_the_current_source(tmp_path, monkeypatch):
    copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    prof = tmp_path / "profiles" / "k_forward_w.md"
    assert bench.profiled_traffic("k_forward", "w") is None  # no summary
    prof.write_text(f"source_sha256_16: {bench.kernel_source_hash()}\ntraffic_bytes_per_launch: 12345\n")
    assert bench.profiled_traffic("k_forward", "w") == 12345
    prof.write_text("source_sha256_16: 0123456789abcdef\ntraffic_bytes_per_launch: 12345\n")
    assert bench.profiled_traffic("k_forward", "w") is None  # stale


def test_clock_summary_reports_throttle_reasons():
    """nvidia-smi rows (clocks, power, event-reason flags): median SM clock, max clock, and every
    reason seen Active; malformed lines are skipped."""
    cs = bench.ClockSampler(0)
    cs.lines = ["2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
                "1980, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
                "2010, 2070, 1400.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
                "[N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbage", ""]
    s = cs.summary()
    assert (s["samples"], s["sm_mhz"], s["sm_max_mhz"]) == (3, 2010.0, 2070.0)
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"],
                                               "samples": 0}


def test_cpu_oracle_solve_times_a_complete_solve():
    """The CPU baseline times one complete oracle solve (no extrapolation): the iteration count is
    the oracle's own for the same cap and stop rule."""
    from paper_0908_4421_gb300 import phantom
    import oracle
    case = phantom.make_case(phantom.TINY_5MM_5BEAM)
    lam0 = oracle.get().lambda0_rule(case, threads=1)
    t, iters, cores = bench.cpu_oracle_solve(case, lam0, max_iter=30, threads=1)
    ref = oracle.get().solve(case, lambda0=lam0, max_iter=30, delta=1e-6, threads=1, trace=False)
    assert cores == 1 and iters == ref.iterations and t > 0


def test_both_arms_print_the_same_config():
    from paper_0908_4421_gb300 import phantom
    case = phantom.make_case(phantom.TINY_5MM_5BEAM)
    a = bench.common_config("tiny-40x40x30-5mm-5beam", case, 200, 1)
    b = bench.common_config("tiny-40x40x30-5mm-5beam", case, 200, 1)
    assert a == b and set(a) >= {"workload", "m", "n", "nnz", "l2", "parallelism"}


def test_gc_paused_restores_the_collector():
    """The timed regions run with the cyclic garbage collector off and turn it back on, also
    when the region raises."""
    import gc

    assert gc.isenabled()
    with bench.gc_paused():
        assert not gc.isenabled()
    assert gc.isenabled()
    try:
        with bench.gc_paused():
            raise RuntimeError("inside the timed region")
    except RuntimeError:
        pass
    assert gc.isenabled()

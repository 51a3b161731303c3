"""Host logic of bench.py that needs no GPU: the kernel labels that tie the
stored ncu traffic to the timed launch, the source-hash gate on that traffic,
and the per-sweep spin-error measure."""
import numpy as np
import pytest

import bench


def test_kernel_labels():
    base = dict(kernel=1, vec_width=4, prefetch=3)
    assert bench.kernel_label(base) == "sc_pass_kernel<1, 4, 1, 2, 0, 1, 0>"
    assert bench.kernel_label(dict(base, prefetch=1)) == "sc_pass_kernel<1, 4, 1, 1, 0, 1, 0>"
    assert bench.kernel_label(dict(base, prefetch=2)) == "sc_pass_kernel<1, 4, 1, 0, 0, 1, 0>"
    # the S.e = S_z variant: FP32, V = 4, no prefetch, e = (0, 0, 1)
    assert bench.kernel_label(dict(base, prefetch=2), zaxis=True) == "sc_pass_kernel<1, 4, 1, 0, 0, 1, 1>"
    assert bench.kernel_label(dict(base, prefetch=3), zaxis=True) == "sc_pass_kernel<1, 4, 1, 2, 0, 1, 0>"
    assert bench.kernel_label(dict(base, prefetch=2), precision_code=0, zaxis=True) == \
        "sc_pass_kernel<0, 4, 1, 0, 0, 1, 0>"
    assert bench.kernel_label(dict(kernel=5, vec_width=8, prefetch=0)) == "sc_pipe_kernel"
    assert bench.kernel_label(dict(kernel=3, vec_width=1, prefetch=1)) == "table_pass_kernel"


def test_traffic_only_for_the_captured_sources_and_kernel(tmp_path, monkeypatch):
    f = tmp_path / "traffic.txt"
    f.write_text(f"kernel: sc_pass_kernel<1, 4, 1, 2, 0>\nsources_sha: {bench.kernels_sha()}\n"
                 "order: ascending\ndram_bytes_per_launch: 123\ncold_dram_bytes_per_launch: 456\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.read_traffic("sc_pass_kernel<1, 4, 1, 2, 0>") == 123.0
    assert bench.read_traffic("sc_pass_kernel<1, 4, 1, 2, 0>", 1) == 123.0
    assert bench.read_traffic("sc_pass_kernel<1, 4, 1, 2, 0>", 1, "cold_dram_bytes_per_launch") == 456.0
    assert bench.read_traffic("sc_pass_kernel<1, 4, 1, 2, 0>", 2) is None     # captured in the other order
    assert bench.read_traffic("sc_pass_kernel<1, 4, 1, 0, 0>") is None
    f.write_text("kernel: sc_pass_kernel<1, 4, 1, 2, 0>\nsources_sha: 0000\ndram_bytes_per_launch: 123\n")
    assert bench.read_traffic("sc_pass_kernel<1, 4, 1, 2, 0>") is None


def test_committed_traffic_matches_the_sources():
    """The stored capture belongs to the current kernel sources (else the bench
    reports no traffic)."""
    assert bench.read_traffic("sc_pass_kernel<1, 4, 1, 0, 0, 1, 1>", 2) is not None


def test_fp64_ops_only_for_the_captured_sources_and_kernel(tmp_path, monkeypatch):
    f = tmp_path / "ops.txt"
    f.write_text(f"kernel: sc_pass_kernel<0, 2, 1, 0, 0, 1>\nsources_sha: {bench.kernels_sha()}\n"
                 "fp64_inst_per_attempt: 60.5\nfp64_flop_per_attempt: 80\nfp64_pipe_inst_per_attempt: 66\n")
    monkeypatch.setattr(bench, "FP64_OPS_FILE", str(f))
    ops = bench.read_fp64_ops("sc_pass_kernel<0, 2, 1, 0, 0, 1>")
    assert ops["inst"] == 60.5 and ops["flop"] == 80.0 and ops["pipe_inst"] == 66.0
    assert bench.read_fp64_ops("sc_pass_kernel<0, 1, 1, 0, 0, 1>") is None   # another kernel
    f.write_text("kernel: sc_pass_kernel<0, 2, 1, 0, 0, 1>\nsources_sha: 0000\nfp64_inst_per_attempt: 60.5\n"
                 "fp64_flop_per_attempt: 80\n")
    assert bench.read_fp64_ops("sc_pass_kernel<0, 2, 1, 0, 0, 1>") is None   # other sources


def test_committed_fp64_ops_match_the_sources():
    """The stored FP64 instruction counts belong to the current kernel sources
    and to the kernel the bench's FP64 form runs (the automatic launch)."""
    assert bench.read_fp64_ops("sc_pass_kernel<0, 2, 1, 0, 0, 1, 0>") is not None


def test_spin_error_measure():
    rng = np.random.default_rng(3)
    S0 = rng.normal(size=(100, 3))
    G, O = S0.copy(), S0.copy()
    G[:40] += 1.0                 # both accept sites 0..39, O slightly differently
    O[:40] += 1.0 + 1e-6
    G[40:45] += 1.0               # the GPU alone accepts five sites
    out = bench._spin_error(S0, G, O)
    assert out["decision_mismatch_frac"] == pytest.approx(0.05)
    assert out["err_max"] == pytest.approx(np.sqrt(3) * 1e-6, rel=1e-6)
    assert out["accept_rate"] == pytest.approx(0.40)

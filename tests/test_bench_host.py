"""Host logic of bench.py that needs no GPU: the DRAM-traffic table keyed by
kernel source hash, the measured peaks, the preconditioner labels and the
argument defaults the driver relies on."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _sha(name):
    p = os.path.join(ROOT, "paper_2007_10411_gb300", "csrc", name + ".cu")
    return hashlib.sha1(open(p, "rb").read()).hexdigest()


def test_traffic_table_lists_every_family_with_sane_ratios():
    """profiles/ncu_traffic.txt lists every kernel family bench.py reports; the
    ratios whose source hash still matches (bench.ncu_traffic) are plausible
    DRAM-per-algorithmic-byte figures.  A stale entry is not an error: bench.py
    then reports the roofline's traffic as null until the counters are re-taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    fams = {l.split()[0] for l in open(path) if l.strip() and not l.startswith("#")}
    # the right-preconditioned step runs passes CA (family arnoldi_a) and B
    assert {"jv", "precond", "arnoldi_a", "arnoldi_b", "fp64_pipe_jv"} <= fams
    for fam, r in bench.ncu_traffic().items():
        assert 0.2 < r < 1.5, (fam, r)
    pipe = bench.ncu_fp64_pipe()
    if pipe is not None:
        assert 0.0 < pipe[0] <= 1.0 and pipe[1] > 0.0


def test_traffic_table_ignores_stale_hashes(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.txt").write_text(
        "# comment\n"
        "jv 0.5 stencil %s\n"
        "arnoldi_a 1.0 krylov 0000000000000000000000000000000000000000\n" % _sha("stencil"))
    csrc = tmp_path / "paper_2007_10411_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in ("stencil", "krylov"):
        (csrc / (name + ".cu")).write_bytes(
            open(os.path.join(ROOT, "paper_2007_10411_gb300", "csrc", name + ".cu"), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic() == {"jv": 0.5}


def test_measured_peaks_have_denominators():
    p = bench.measured_peaks()
    assert p["hbm_gbs"] > 1000.0
    assert p["source"]


def test_pc_labels_name_the_preconditioner():
    case = {"opts": {"pc_sweeps": 2}}
    assert "field-block" in bench.pc_label("block", case)
    assert "Schur" in bench.pc_label("schur", case)
    assert "nonlinear" in bench.pc_label("nonlinear", case)


def test_default_arguments(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1
    assert a.precond == "block" and a.impl == "ours"
    assert a.schur_sweeps == 32 and a.nonlinear_steps > 0


@pytest.mark.parametrize("world", [1, 2, 4])
def test_job_throughput_sums_over_ranks(world):
    one = bench.job_throughput(524288, 10, 1, 1000.0)
    assert bench.job_throughput(524288, 10, world, 1000.0) == pytest.approx(world * one)


def test_metric_label_names_the_precision():
    # the headline label is fixed; another workload or a float64 step says so in its label
    assert bench.metric_name(bench.WORKLOAD) == bench.METRICS[bench.WORKLOAD]
    assert "mixed FP32/FP64" in bench.metric_name(bench.WORKLOAD)
    assert "FP64 JFNK" in bench.metric_name(bench.WORKLOAD, fp64=True)
    assert "mixed" not in bench.metric_name(bench.WORKLOAD, fp64=True)
    assert bench.metric_name("thermal_neutral_128x64", fp64=True).endswith("(thermal_neutral_128x64, FP64 JFNK)")

"""Host logic of bench.py's evidence (no GPU): the measured-traffic lines under
profiles/ and the stage-kernel labels.

`roofline.traffic` is read from a `bench-traffic:` line of an ncu summary and
reported only while the kernel's source has the hash recorded with the counters;
these tests check that every such line is well formed and names a known kernel,
that a matching hash yields the figure and a changed source yields none, and the
label of a mask of stage kernels.
"""
import os
import re

import bench


def _traffic_lines():
    out = []
    pdir = os.path.join(bench.ROOT, "profiles")
    for name in sorted(os.listdir(pdir)):
        with open(os.path.join(pdir, name)) as fh:
            for line in fh:
                if "bench-traffic:" in line:
                    out.append((name, line.strip()))
    return out


def test_every_traffic_line_is_well_formed_and_names_a_known_kernel():
    lines = _traffic_lines()
    assert lines, "no measured-traffic line under profiles/"
    for name, line in lines:
        m = re.match(r"bench-traffic: kernel=(\S+) workload=(\S+) source_sha256=([0-9a-f]{16}) "
                     r"bytes_per_launch=([0-9.eE+]+)$", line)
        assert m, (name, line)
        assert m.group(1) in bench.KERNEL_SOURCES, (name, m.group(1))
        assert float(m.group(4)) > 0, (name, line)


def test_traffic_is_reported_only_for_the_source_it_was_measured_on(tmp_path, monkeypatch):
    src = tmp_path / "paper_1603_05211_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "fv.cuh").write_text("// kernel source as captured\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.kernel_source_sha("k_fvp")
    (tmp_path / "profiles" / "k.md").write_text(
        f"bench-traffic: kernel=k_fvp workload=w source_sha256={sha} bytes_per_launch=1234\n")
    assert bench.profiled_traffic("k_fvp (pencil on staged primitives)", "w") == (1234.0, "k.md")
    assert bench.profiled_traffic("k_fvp (pencil on staged primitives)", "other")[0] is None
    (src / "fv.cuh").write_text("// kernel source changed since\n")
    value, why = bench.profiled_traffic("k_fvp (pencil on staged primitives)", "w")
    assert value is None and "changed" in why


def test_stage_kernel_labels():
    assert bench.stage_kernel_names(0) == "stage kernel"
    assert bench.stage_kernel_names(8) == "k_fvp (pencil on staged primitives)"
    assert bench.stage_kernel_names(1 | 32) == "k_fv (pencil) + k_fvt (TMA-staged, packed x/y lines)"

"""The committed ncu summaries that bench.py reads: every traffic line parses,
names a kernel the library defines, and the tensor-core kernels' lines were
taken on the current kernel code (else bench.py would report null)."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import pytest  # noqa: E402

from paper_2310_16668_gb300 import workloads as W  # noqa: E402

PAT = re.compile(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+kernel:\s*(\S+)\s+precision:\s*(\S+)\s+"
                 r"source_sha:\s*([0-9a-f]+)\s+workload:\s*(\S+)")


def _lines():
    d = os.path.join(ROOT, "profiles")
    out = []
    for f in sorted(os.listdir(d)):
        if f.endswith((".md", ".txt")):
            out += [(f, m) for m in PAT.finditer(open(os.path.join(d, f)).read())]
    return out


def test_traffic_lines_parse_and_name_library_kernels():
    src = "".join(open(os.path.join(ROOT, "paper_2310_16668_gb300", "csrc", f)).read()
                  for f in ("tc_kernels.cuh", "tc_complex.cuh", "skel_kernels.cuh"))
    lines = _lines()
    assert lines
    for f, m in lines:
        assert float(m.group(1)) > 0, f
        assert re.search(r"\b" + m.group(2) + r"\b", src), (f, m.group(2))
        assert m.group(3) in ("fp64", "fp32", "fp32_tc"), f
        assert m.group(5) in set(W.WORKLOADS) | {W.CurveSets().name}, (f, m.group(5))


def test_tensor_core_traffic_is_current():
    # a kernel change makes the committed figure stale until it is captured
    # again; that is reported as a skip, not a failure
    for kernel, workload in (("tc_stored_kernel", "laplace3d_uniform_n1048576"),
                             ("tc_cnear_kernel", "helmholtz3d_k25_uniform_n1048576")):
        t = bench.ncu_traffic(kernel, "fp32_tc", workload)
        if t is None:
            pytest.skip(f"{kernel}: no traffic line for the current kernel code {bench.kernel_source_sha(kernel)}")
        assert t > 0


def test_profile_commands_run_committed_files_only():
    # every summary gives the command that made it, and the command names no
    # scratch file
    d = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(d)):
        text = open(os.path.join(d, f)).read()
        assert "```" in text, f
        assert "_work/" not in text, f

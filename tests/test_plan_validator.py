"""The host check of a plan's lists (validate_plan, run on every plan before
it is uploaded): a real plan passes, and each corruption of an index the
device kernels use is reported.  The check is compiled from the library's
own plan source with the host compiler and linked against the built
library (for the parameter defaults)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2312_00005_gb300 import bemfmm, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plan_check_accepts_plans_and_rejects_corruptions(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    bemfmm.lib()                                  # the built library, for bem_params_default
    so = os.path.join(ROOT, "paper_2312_00005_gb300", "_bemfmm.so")
    exe = str(tmp_path / "plan_validator_check")
    cmd = [cxx, "-O1", "-std=c++17", "-I/usr/local/cuda/include", os.path.join(ROOT, "tests", "plan_validator_check.cpp"),
           os.path.join(ROOT, "paper_2312_00005_gb300", "csrc", "bem_plan.cpp"), so,
           "-Wl,-rpath," + os.path.dirname(so), "-lpthread", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    nodes, tris = inputs.icosphere(3, 0.1)
    fn, ft = str(tmp_path / "nodes.bin"), str(tmp_path / "tris.bin")
    np.ascontiguousarray(nodes, np.float64).tofile(fn)
    np.ascontiguousarray(tris, np.int32).tofile(ft)
    r = subprocess.run([exe, fn, ft], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    res = dict(line.split(": ", 1) for line in r.stdout.strip().splitlines())
    assert res.pop("valid") == "ok"
    assert set(res) == {"near_leaf_out_of_range", "near_pointers_not_monotone", "entry_count", "cluster_out_of_range",
                        "translation_row_out_of_range"}
    for case, msg in res.items():
        assert msg != "ok", case

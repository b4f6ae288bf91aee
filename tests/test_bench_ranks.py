"""Replica bookkeeping of bench.py across processes (gloo, world size 2, CPU):
times are the maximum over ranks and product counts the sum, as the
whole-job throughput of independent replicas requires."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    # rank r: 10 + r ms timed, 20 + 3 r ms end to end, 50 + r and 40 + r products
    res = bench.combine_ranks(10.0 + rank, 20.0 + 3 * rank, 50.0 + rank, 40.0 + rank)
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_two_processes():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn", join=True)
    for r in range(ws):
        t, e, mv, emv = out[r]
        assert t == 11.0 and e == 23.0
        assert mv == 101.0 and emv == 81.0


def test_combine_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(1.5, 2.5, 3.0, 4.0) == (1.5, 2.5, 3.0, 4.0)


@pytest.mark.parametrize("workload", ["head_bands_c3", "head_adjoint_c4"])
def test_extra_workloads_reference_arm_reports_unavailable(workload):
    """The batched-frequency and adjoint workloads have no bounded oracle
    sample: their reference arm prints one JSON line with "unavailable" and
    exits 0."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        workload], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line

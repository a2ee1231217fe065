"""Multi-rank host logic of bench.py on CPU: two gloo ranks on 127.0.0.1 (no GPU).
The max over ranks that the timed region uses, and the reference arm under
torchrun-style launch: rank 0 alone prints one JSON line, the other rank exits 0
without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
mode = sys.argv[1]
if mode == "max":
    args = bench.parse_args([])
    world, rank, local, pg = bench.dist_setup(args)
    got = bench.max_over_ranks(pg, 1.5 + rank, "cpu")
    print(json.dumps({{"rank": rank, "world": world, "max": got}}), flush=True)
    pg.destroy_process_group()
else:
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-stride", "62"]
    sys.exit(bench.main())
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _run_two(mode, timeout):
    port = _free_port()
    code = _WORKER.format(root=ROOT)
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code, mode], env=env, cwd=ROOT, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        outs.append((p.returncode, out, err))
    return outs


def test_max_over_ranks_gloo():
    outs = _run_two("max", 120)
    for rc, out, err in outs:
        assert rc == 0, err
    vals = [json.loads(o.strip().splitlines()[-1]) for _, o, _ in outs]
    assert sorted(v["rank"] for v in vals) == [0, 1]
    assert all(v["world"] == 2 and v["max"] == 2.5 for v in vals)


def test_reference_arm_rank0_only():
    pytest.importorskip("numpy")
    outs = _run_two("reference", 600)
    (rc0, out0, err0), (rc1, out1, err1) = outs
    assert rc0 == 0 and rc1 == 0, (err0, err1)
    assert out1.strip() == ""
    line = json.loads(out0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0

"""Host-side pieces of bench.py: the multi-rank plumbing (world size 2 over
gloo, one process per rank as torchrun would start them) and the reference
arm (the FP64 oracle timed on the host) with its JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
d = bench.Dist(backend="gloo")
d.barrier()
m = d.max(float(d.rank) + 0.5)
d.barrier()
print(json.dumps({{"rank": d.rank, "world": d.world, "max": m}}), flush=True)
d.close()
"""


def test_two_rank_barrier_and_max_over_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    assert all(o["world"] == 2 and o["max"] == 1.5 for o in outs)


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--nx", "96",
                        "--steps", "2", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "cell-updates/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True


def test_reference_arm_second_rank_exits_quietly():
    port = _free_port()
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    # rank 1 of the reference arm does no work and prints nothing; it must not
    # wait for rank 0 (the reference arm creates no process group)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--nx", "64",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_cpu_baseline_legs_on_a_small_grid():
    """The one-core and the OpenMP baseline legs time the oracle on a bounded
    sample and report what they ran on."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2006_01748_gb300 import inputs
    p = inputs.hetero_8192(nx=96)
    one = bench.cpu_baseline_leg(p)
    assert one["kind"] == "oracle" and one["cores"] == 1 and one["value"] > 0
    omp = bench.cpu_openmp_leg(p)
    if omp is None:
        pytest.skip("the compiler has no OpenMP")
    assert omp["kind"] == "oracle (OpenMP build)" and omp["cores"] >= 1 and omp["value"] > 0
    assert "explicit steps of the 96x96 grid" in omp["sample"]

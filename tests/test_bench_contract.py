"""The bench's CPU-side contract (no GPU): the reference arm's JSON line,
quiet non-zero ranks, and the max-over-ranks time of N replicas with two
gloo processes."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = dict(os.environ, OMP_NUM_THREADS="2")
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                          env=env, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def _worker(rank, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=2)
    ms = bench.max_over_ranks(torch, [3.5, 7.25][rank], "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms))


def test_max_over_ranks_with_two_gloo_processes():
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 7.25), (1, 7.25)]


class _FakeSim:
    npatch = 1024

    def stats(self):
        return {"live_bytes": 1343488}


def test_roofline_bytes_count_the_ghost_sources_of_each_kernel():
    sys.path.insert(0, ROOT)
    import bench
    tables_sums = 2 * 1024 * 8 + 1024 * 9 * 8
    # ring-free D2Q9 on BL5/3: own record read and written are compulsory;
    # the eight neighbour records it reads for its ghosts mostly hit L2
    ringfree = bench.roofline_bytes(_FakeSim(), {"scheme": "d2q9", "wavelet": "bl53", "P": 64})
    assert ringfree["compulsory"] == 2 * 1343488 + tables_sums
    assert ringfree["with_l2_reuse"] == 10 * 1343488 + tables_sums
    # kernels with a ghost ring (Haar): the ring of 12 (P+1) + 4 FP32 values read and written per patch
    ring = bench.roofline_bytes(_FakeSim(), {"scheme": "d2q9", "wavelet": "haar", "P": 64})
    assert ring["compulsory"] == ring["with_l2_reuse"] == 2 * 1343488 + 2 * 1024 * (12 * 65 + 4) * 4 + tables_sums


@pytest.mark.parametrize("P,L", [(64, 4), (32, 3)])
def test_roofline_numerator_is_the_oracles_operation_count(P, L):
    """The ALU roofline's numerator (algorithmic FP32 operations per lattice
    update) against what the oracle executes, counted by a number type whose
    +, -, * and / count one each: a forward and an inverse 2-D transform per
    field, one BGK collision per node; the threshold's |d| and compare per
    coefficient are the formula's own (two per coefficient)."""
    import bench
    import oracle as O
    fwd, inv, coll = O.count_ops(P, L)
    assert coll == 135
    assert fwd == inv == 2 * (P + 1) * bench.lifting_flops_per_line(P, L)
    E, F = P + 1, 9
    want = F * (fwd + inv) / (P * P) + coll + 2 * F * E * E / (P * P)
    assert abs(bench.algorithmic_flops_per_lu(P, L) - want) < 1e-9

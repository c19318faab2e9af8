"""The benchmark's multi-rank host logic on CPU: two gloo ranks, no GPU.

With N replicas (one seeded problem per rank, no data-path collective) the
benchmark reports the slowest rank's time; a rank that missed the tolerance
makes the whole job's value None.  The reference arm runs on rank 0 only.
"""

import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    try:
        got = [bench.max_over_ranks(v[rank], dist, "cpu") for v in values]
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    values = [(0.5, 0.25), (0.1, 0.9), (None, 0.3), (0.2, None), (None, None)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [0.5, 0.9, None, None, None]
    assert res[0] == want and res[1] == want


def test_max_over_ranks_single_process():
    import bench

    assert bench.max_over_ranks(0.3) == 0.3
    assert bench.max_over_ranks(None) is None


@pytest.mark.parametrize("rank", ["1", "3"])
def test_reference_arm_other_ranks_exit_without_work(rank):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="4", LOCAL_RANK=rank)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "4"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_line_contract(monkeypatch, capsys):
    """Rank 0 prints one JSON line with the contract's keys; each timed step is one whole oracle solve to
    the tolerance and each warm-up step a one-subiteration solve (the oracle solve itself is replaced by
    a stub here: it takes tens of seconds of CPU work)."""
    import bench

    calls = []

    def fake(cfg, data, alpha, M, xstar, tol_hu, x0="fbp", max_iter=60, stop_after_sub=None):
        calls.append(stop_after_sub)
        return {"seconds": 1.5, "fbp_s": 0.1, "dl_s": 0.2, "cores": 1, "iters_to_tol": 6,
                "rmsd_trace_hu": [3.0, 0.9]}

    monkeypatch.setattr(bench, "oracle_solve_to_tol", fake)
    monkeypatch.setattr(bench, "oracle_xstar", lambda cfg: (object(), {"recipe": "stub", "kkt_rms_hu": 0.0}))
    monkeypatch.setattr(bench, "make_problem", lambda args, rank: (type("C", (), {"name": "fan2d_512"})(), 1.999,
                                                                     20, 30, None))
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"])
    args = bench.parse()
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] == 1.5 and line["unit"] == "s"
    assert line["higher_is_better"] is False and line["steps"] == 2 and line["warmup"] == 3
    assert line["ms_per_step"] == 1500.0
    assert line["e2e"] == {"value": 1.5, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == 1.5
    assert calls == [1, 1, 1, None, None]


def test_reference_arm_without_stored_xstar(monkeypatch, capsys):
    import bench

    monkeypatch.setattr(bench, "oracle_xstar", lambda cfg: (None, None))
    monkeypatch.setattr(bench, "make_problem", lambda args, rank: (type("C", (), {"name": "fan2d_x"})(), 1.999,
                                                                     20, 30, None))
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    assert bench.run_reference(bench.parse()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line


def test_kernel_digest_ignores_comments_only(tmp_path):
    """The DRAM-traffic record is reported only while the profiled kernels' code is unchanged: a comment
    edit keeps the digest, a code edit in the forward or back projector changes it."""
    import shutil

    import bench

    src = os.path.join(ROOT, "paper_1512_04564_gb300", "csrc")
    for f in ("projectors.cu", "ct_internal.cuh"):
        shutil.copy(os.path.join(src, f), tmp_path / f)
    d0 = bench._source_digest(str(tmp_path))
    assert d0 == bench._source_digest()
    p = tmp_path / "projectors.cu"
    text = p.read_text()
    p.write_text(text.replace("fp_csr_kernel(FanDev G", "fp_csr_kernel(FanDev G /* a comment */", 1))
    assert bench._source_digest(str(tmp_path)) == d0
    for old, new in (("8 * __ldg(&G.ray_order[rank])", "8 * __ldg(&G.ray_order[rank + 0])"),  # forward
                     ("const int slot = chunk * kRecGroup + lane;", "const int slot = lane + chunk * kRecGroup;")):  # back
        assert text.count(old) == 1
        p.write_text(text.replace(old, new))
        assert bench._source_digest(str(tmp_path)) != d0

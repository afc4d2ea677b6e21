"""bench.py's N > 1 path on the CPU: two ranks over gloo on 127.0.0.1.

The GPU arm runs one independent replica per rank (no collective on the data path) and reports
the whole-job rate over the slowest rank; the reference arm runs on rank 0 only.  Checked here:
the timing reduction hands every rank the per-entry maximum over the ranks, the whole-job rate
counts every replica's units, and `bench.py --impl reference` launched by torchrun with two ranks
prints exactly one JSON line (rank 0) while rank 1 exits 0 without work."""
import json
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, nproc=2, timeout=600):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)


def test_timings_reduce_to_the_slowest_rank(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent(f"""
        import json, sys
        sys.path.insert(0, {ROOT!r})
        import torch.distributed as dist
        import bench
        dist.init_process_group("gloo")
        r, w = dist.get_rank(), dist.get_world_size()
        got = bench.max_over_ranks([1.0 + r, 5.0 - r, 2.5], w, "cpu")
        dist.barrier()
        out = json.dumps({{"vals": got, "rate": bench.whole_job_rate(1000, w, got[0])}})
        # one write per line (shorter than PIPE_BUF): the two ranks share the pipe
        sys.stdout.write("RANK %d %s\\n" % (r, out))
        sys.stdout.flush()
        dist.destroy_process_group()
    """))
    p = _torchrun([str(script)])
    assert p.returncode == 0, p.stderr[-3000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("RANK")]
    assert sorted(int(l.split(" ", 2)[1]) for l in lines) == [0, 1]
    for l in lines:
        d = json.loads(l.split(" ", 2)[2])
        assert d["vals"] == [2.0, 5.0, 2.5]           # per-entry maximum over the two ranks
        assert d["rate"] == 2 * 1000 / 2.0e-3         # both replicas' units over the slowest time


def test_one_rank_timing_is_unchanged():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(500, 1, 2.0) == 500 / 2.0e-3


def test_reference_arm_prints_once_under_two_ranks():
    p = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                  timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout[-3000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "DoF/s"
    assert d["config"]["n_cells"] == 64 ** 3 and d["e2e"]["h2d_bytes_per_step"] == 0

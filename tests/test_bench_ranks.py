"""bench.py's multi-rank plumbing on the CPU: two gloo ranks launched the way
torchrun launches them (RANK / WORLD_SIZE / MASTER_* in the environment)."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import io, contextlib, json, os, sys
sys.path.insert(0, os.getcwd())
import bench
rank, world, dist = bench.dist_init(2)
assert dist is not None and dist.get_backend() == "gloo"
# each rank reports its own step time; the job's time is the slowest rank's
mine = [10.0 + rank, 5.0 - rank]
both = bench.max_over_ranks(dist, mine)
out = io.StringIO()
class A: steps = 1; warmup = 0; gpus = world
with contextlib.redirect_stdout(out):
    if rank != 0:
        bench.run_reference(A, rank, world)      # other ranks exit without work
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "world": world, "max": both, "ref_out": out.getvalue()}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_max_and_only_rank0_reports():
    import json
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], cwd=ROOT, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for r in outs:
        assert r["world"] == 2
        assert r["max"] == [11.0, 5.0]
    assert outs[1]["ref_out"] == ""


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host and prints
    one JSON line with the keys of the bench line contract."""
    import json
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_kernel_fingerprint_ignores_comments_and_sees_code(tmp_path):
    """The traffic figure of a committed ncu summary is used only while the
    kernel code it was taken on is unchanged: the fingerprint must not move
    when only comments or blank lines change, and must move with the code."""
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_1609_03170_gb300", "csrc")
    for f in ("grape_kernels.cuh", "grape_num.cuh", "grape_internal.h"):
        shutil.copy(os.path.join(src, f), tmp_path / f)
    base = bench.kernel_source_sha(str(tmp_path))
    assert base == bench.kernel_source_sha()
    k = tmp_path / "grape_kernels.cuh"
    text = k.read_text()
    k.write_text("// a new comment line\n\n" + text.replace("\n", "   \n", 3) + "/* block\n comment */\n")
    assert bench.kernel_source_sha(str(tmp_path)) == base
    k.write_text(text.replace("mbar_init(mbar_sa, 1u + (uint32_t)blockDim.x);",
                              "mbar_init(mbar_sa, 2u + (uint32_t)blockDim.x);", 1))
    assert bench.kernel_source_sha(str(tmp_path)) != base

"""bench.py's launcher logic on the CPU: the world size it runs under must
match --gpus, and --gpus N without a launcher re-runs the command as N ranks."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_world_size_must_match_gpus():
    env = dict(os.environ, WORLD_SIZE="3", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--steps", "1"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 2 and "WORLD_SIZE=3 but --gpus 2" in r.stderr


def test_spawn_command_line(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    seen = {}

    def fake_call(cmd):
        seen["cmd"] = cmd
        return 0

    monkeypatch.setattr(bench.subprocess, "call", fake_call)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--gpus", "4", "--parallelism", "strips"])
    assert bench.spawn_ranks(4) == 0
    cmd = seen["cmd"]
    assert cmd[1:4] == ["-m", "torch.distributed.run", "--nnodes=1"]
    assert cmd[cmd.index("--nproc-per-node") + 1] == "4"
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[-4:] == ["--gpus", "4", "--parallelism", "strips"]


def test_cpu_list_helpers(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    assert bench.compact_cpus({0, 1, 2, 3, 8, 10, 11}) == "0-3,8,10-11"
    assert bench.compact_cpus(set()) == ""

    # a GPU whose PCI device lists CPUs 2-3: the helper returns them (within
    # the process's own affinity); anything missing gives None
    class R:
        stdout = "00000009:01:00.0\n"

    monkeypatch.setattr(bench.subprocess, "run", lambda *a, **k: R())
    real_open = open

    def fake_open(path, *a, **k):
        if path == "/sys/bus/pci/devices/0009:01:00.0/local_cpulist":
            import io
            return io.StringIO("2-3\n")
        return real_open(path, *a, **k)

    monkeypatch.setattr("builtins.open", fake_open)
    mine = os.sched_getaffinity(0)
    got = bench.gpu_local_cpus(0)
    assert got == ({2, 3} & mine or None)
    monkeypatch.setattr("builtins.open", real_open)
    assert bench.gpu_local_cpus(0) is None

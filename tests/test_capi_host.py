"""CPU-only checks of the boundary: the shared library exports every function include/ufg.h
declares, the Python binding covers them, and the multi-rank bench logic (per-rank problem
ownership, max-over-ranks timing) under a 2-rank gloo group."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ufg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[a-z_ ]+\*?\s*\**(ufg_[a-zA-Z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1008_3647_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    return B.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ufg_apply_M", "ufg_apply_Mdag", "ufg_solve_cg_normal",
                 "ufg_solve_bicgstab_two_step", "ufg_set_preconditioner", "ufg_hmc_force",
                 "ufg_lattice_create", "ufg_field_create", "ufg_solve_batch"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    import ctypes
    lib = ctypes.CDLL(lib_path)  # loading needs no GPU
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True)
    exported = set(re.findall(r" T (ufg_\w+)", out.stdout))
    assert set(_declared()) <= exported


def test_binding_covers_the_header():
    from paper_1008_3647_gb300 import ufg
    assert set(_declared()) == set(ufg.EXPORTED)


def test_binding_fails_loudly_without_library(tmp_path):
    code = ("import paper_1008_3647_gb300.ufg as u\n"
            "try:\n    u.load(%r)\nexcept RuntimeError as e:\n    print('raised')\n"
            % str(tmp_path / "missing.so"))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert "raised" in r.stdout


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    t = bench.max_over_ranks(1.0 + rank, world)
    q.put((rank, t, bench.seeds_for_rank(rank)))
    dist.destroy_process_group()


def test_bench_multirank_logic_gloo():
    import multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert [r[1] for r in res] == [2.0, 2.0]  # every rank reports the slowest rank's time
    assert not set(res[0][2]) & set(res[1][2])  # disjoint problems per rank


def test_bench_clock_summary_keeps_the_timed_window():
    # nvidia-smi lines (timestamp first): only samples inside the marked window count; the
    # throttle reasons and the median clock come from those
    import datetime
    sys.path.insert(0, ROOT)
    import bench
    lines = [
        "2026/12/03 18:11:05.100, 0, 1200, 2070, 250.5, 0x0, Not Active, Not Active, Not Active, "
        "Not Active",
        "2026/12/03 18:11:05.200, 0, 2070, 2070, 900.1, 0x4, Not Active, Not Active, Not Active, "
        "Active",
        "2026/12/03 18:11:05.300, 0, 2055, 2070, 880.0, 0x0, Not Active, Not Active, Not Active, "
        "Not Active",
        "2026/12/03 18:11:06.300, 0, 2070, 2070, 260.0, 0x0, Active, Not Active, Not Active, "
        "Not Active",
        "not a sample line",
    ]
    rows = bench.ClockSampler.parse(lines)
    assert len(rows) == 4
    t0 = datetime.datetime(2026, 12, 3, 18, 11, 5, 150000)
    t1 = datetime.datetime(2026, 12, 3, 18, 11, 6)
    s = bench.ClockSampler.summarise(rows, t0, t1)
    assert s["samples"] == 2 and s["window"] == "timed region"
    assert s["sm_mhz"] == (2070 + 2055) / 2 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["power_w_max"] == 900.1
    # no sample inside the window: all samples, said so
    s = bench.ClockSampler.summarise(rows, t1, t1)
    assert s["samples"] == 4 and s["window"].startswith("whole run")
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler.summarise([], None, None)["reasons"] == ["unsampled"]

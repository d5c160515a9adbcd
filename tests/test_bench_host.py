"""Host logic of bench.py, without a GPU: the algorithmic bytes of the
roofline, the matching of a committed ncu traffic record to the kernel
sources and launch plan, the clock-record summary and the FLOP count."""
import importlib.util
import os
import re
import types

import numpy as np
import pytest

from paper_2005_05899_b300 import meshgen as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_count_each_referenced_node_once(bench):
    m = mg.tgv_mesh(3)
    conn = m.conn[0]
    b, e, n = bench.tet_algorithmic_bytes(m)
    assert e == conn.shape[0] == 6 * 27
    assert n == np.unique(conn).size
    assert b == 16 * e + 52 * n
    # a mesh whose elements reference only some of the nodes
    sub = mg.Mesh(xyz=m.xyz, conn={0: conn[:5]})
    b5, e5, n5 = bench.tet_algorithmic_bytes(sub)
    assert (e5, n5) == (5, np.unique(conn[:5]).size) and b5 == 16 * 5 + 52 * n5


def test_traffic_record_needs_matching_sources_and_plan(bench, monkeypatch):
    import json
    recs = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))["tet04_mixed_assembly"]
    rec = recs[0]
    plan = dict(rec["plan"])
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["source_hash"])
    assert bench.ncu_traffic("tet04_mixed_assembly", plan) == rec["dram_bytes_per_launch"]
    # every recorded plan finds its own record
    for r in recs:
        assert bench.ncu_traffic("tet04_mixed_assembly", dict(r["plan"])) == r["dram_bytes_per_launch"]
    # the generic chunk size does not change the TET04 kernel's launch
    assert bench.ncu_traffic("tet04_mixed_assembly", dict(plan, chunk_elems=96)) == rec["dram_bytes_per_launch"]
    # a configuration that was not captured, another kernel key, changed sources: no traffic figure
    captured = {bench.tet_kernel_config(r["plan"])["compute_warps"] for r in recs}
    missing = [t for t, w in ((128, 4), (256, 8), (384, 12)) if w not in captured]
    if missing:
        assert bench.ncu_traffic("tet04_mixed_assembly", dict(plan, threads_per_block=missing[0])) is None
    assert bench.ncu_traffic("tet04_mixed_assembly", dict(plan, chunk_acc=1)) is None
    assert bench.ncu_traffic("no_such_kernel", plan) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.ncu_traffic("tet04_mixed_assembly", plan) is None


def test_clock_summary(bench, tmp_path, monkeypatch):
    monkeypatch.setenv("FEA_BENCH_CLOCKS_DIR", str(tmp_path))
    cs = bench.ClockSampler(0)
    rows = [
        "0, 2032, 2032, 800.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1990, 2032, 1100.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2032, 1050.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2032, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    with open(cs.path, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    # stand-ins for the sampling process and its output file
    cs.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: 0, kill=lambda: None)
    cs.f = open(os.devnull, "w")
    s = cs.stop()
    assert s == {"sm_mhz": 2010.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"], "samples": 3}
    # without a sampling process there is no record
    assert bench.ClockSampler(0).stop() is None


def test_tet_flop_count_matches_its_itemisation(bench):
    src = open(os.path.join(ROOT, "bench.py")).read()
    block = src[src.index("# FP32 operations of one TET04"):src.index("TET_FLOPS =")]
    # each part's count ends its item (before a comma, a period or the line's end)
    items = [int(x) for x in re.findall(r"\b(\d+)(?:,|\.|\s*$)", block, flags=re.M)]
    assert len(items) == 14
    assert sum(items) == bench.TET_FLOPS == 411


def test_a_failed_secondary_leg_is_reported_in_its_place(bench):
    assert bench.run_leg("ok", lambda: {"v": 1}) == {"v": 1}

    def boom():
        raise RuntimeError("device lost")
    assert bench.run_leg("bad", boom) == {"error": "RuntimeError: device lost"}


def test_mesh_flops_sum_the_per_type_counts(bench):
    # per Gauss point 90 nen + 147 operations, plus 5 per element
    assert bench.ELEM_FLOPS == {"TET04": 4 * 507 + 5, "PYR05": 8 * 597 + 5, "PEN06": 6 * 687 + 5,
                                "HEX08": 8 * 867 + 5}
    counts = {"TET04": 3, "PYR05": 0, "PEN06": 2, "HEX08": 1}
    assert bench.mesh_flops(counts) == 3 * 2033 + 2 * 4127 + 6941
    assert bench.mesh_flops({}) == 0
    # the batch's meshes (channel-like) by their own counts
    m = mg.channel_mesh(nx=6, ny=10, nz=4, seed=1, n_layers=2, split_frac=0.3)
    assert bench.mesh_flops(m.counts()) == sum(bench.ELEM_FLOPS[t] * n for t, n in m.counts().items())


def _max_rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = importlib.util.spec_from_file_location("bench_rank", os.path.join(ROOT, "bench.py"))
        bench = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(bench)
        # each rank's step time and end-to-end times; the slowest rank differs per entry
        got = bench.max_over_ranks([10.0 + rank, 5.0 - rank, 7.0 * (rank == 1)], world, device="cpu")
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_times_are_the_maximum_over_two_gloo_ranks(bench):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = mp.get_context("spawn").SimpleQueue()
    mp.start_processes(_max_rank_main, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    res = sorted(q.get() for _ in range(2))
    assert [r for r, _ in res] == [0, 1]
    for _, got in res:
        assert got == [11.0, 5.0, 7.0]
    # one rank: the values unchanged
    assert bench.max_over_ranks([3.5, 1.0], 1, device="cpu") == [3.5, 1.0]


def test_reference_arm_prints_its_json_line(bench):
    """`bench.py --impl reference` (the oracle on the host cores, no GPU) on
    a small airplane-like mesh: one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--n-axis", "40"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "RHS assembly Melem/s" and d["unit"] == "Melem/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
    # the same workload description as the GPU arm's line
    assert set(d["config"]) == {"workload", "elements", "nodes", "counts", "l2", "parallelism"}
    assert d["config"]["workload"] == bench.WORKLOAD and d["config"]["elements"] == sum(
        d["config"]["counts"].values())
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["serial_value"] > 0 and cb["cpu_model"] and "TET04" in cb["sample"]

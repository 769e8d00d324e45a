"""Host-side logic of bench.py (no GPU): the multi-rank timing aggregation with
two gloo ranks on the CPU, the reference arm's non-zero ranks, and the served
request stream (every request inside the forward-Euler bound, the configured mix)."""
import os
import socket

import numpy as np
import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


PORT = _free_port()


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r+1) ms in total and 10*(world-r) ms in its kernels
        got = bench.reduce_max_over_ranks([rank + 1.0, 10.0 * (world - rank)])
        out.put((rank, got, bench.replica_glups(1e9, world, got[0] * 1e-3)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, PORT, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, glups in res:
        assert got == [2.0, 20.0]                      # both ranks see the slowest rank's times
        assert glups == pytest.approx(2 * 1e9 / 2e-3 / 1e9)  # all ranks' work over the slowest time



def test_replica_glups_is_whole_job():
    assert bench.replica_glups(4e9, 4, 2.0) == pytest.approx(8.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, steps, warmup = bench.DEFAULT, 3, 3

    assert bench.run_reference(A()) == 0


def test_served_request_stream():
    import paper_2511_10508_gb300 as sp

    reqs = bench.served_requests(400, 4)
    assert len(reqs) == 400
    models = [m for m, *_ in reqs]
    dims = [len(sh) for _, sh, *_ in reqs]
    assert set(models) == {0, 1, 2} and set(dims) == {2, 3}
    for m, sh, dt, n, kw in reqs:
        lo, hi = (64, 2048) if len(sh) == 2 else (32, 256)
        assert lo <= sh[0] <= hi and 100 <= n <= 5000 and kw["dtype"] in (0, 1)
        p = sp.params(m, len(sh), **{k: v for k, v in kw.items()})
        ok, f = sp.check_stability(m, len(sh), 1.0, dt, p)
        assert ok, (m, sh, dt, kw, f)
    # log-uniform sides: the median 2D side is near sqrt(64*2048) = 362
    s2 = np.array([sh[0] for _, sh, *_ in reqs if len(sh) == 2])
    assert 250 < np.median(s2) < 520
    assert bench.served_requests(400, 4) == reqs  # seeded


@pytest.mark.parametrize("workload", sorted(bench.WORKLOADS))
def test_roofline_object_of_every_workload(workload):
    """The roofline object of every bench workload (host arithmetic only): FP64 lines
    are bound by the FP64 pipe against the derived peak, FP32/BF16 lines by HBM
    against the measured copy bandwidth; achieved = algorithmic work / time."""
    w = bench.WORKLOADS[workload]
    model, dims, shape, st, dtype = w[0], w[1], w[2], w[4], w[5]
    order = int(workload.split("-gen", 1)[1].split("-")[0]) if "-gen" in workload else 0
    spectral = "spectral" in workload
    npts = int(np.prod(shape))
    roof = bench.roofline(model, dims, st, dtype, order, spectral, npts, 1.0, 1, None, {"hbm_gbs": 6800.0})
    assert set(("bound", "achieved", "peak", "unit", "frac", "traffic")) <= set(roof)
    if dtype == 0:
        assert roof["bound"] == "alu" and roof["unit"] == "FP64 Gop/s" and roof["peak"] == bench.FP64_PEAK_GOPS
    else:
        assert roof["bound"] == "hbm" and roof["unit"] == "GB/s" and roof["peak"] == 6800.0
        if not spectral:
            # bytes per update: one read and one write of every field
            assert roof["achieved"] == pytest.approx(bench.hbm_bytes_per_lup(model, dtype, dims) * npts / 1e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])


def test_reference_arm_line():
    """The reference arm (the oracle timed on the host cores) prints the benchmark
    line with the same metric and config as the GPU arm, an e2e equal to its value
    with no host transfers, and a cpu_baseline describing the run."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                        "ac2d-256-f64-lap5", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "GLUPS" and line["unit"] == "GLUPS"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["warmup"] >= 3
    assert line["config"]["workload"].startswith("Allen-Cahn 2D 256x256 f64")
    assert line["e2e"] == {"value": line["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]


def test_workload_table_is_well_formed():
    """Every bench workload names a model, dims and stencil that fit together,
    a storage type, a positive step count, and (where given) a steps-per-launch
    and kernel-family pair from the library's documented values; the per-config
    entries name existing workloads."""
    models = {0, 1, 2, 3, 4}
    for name, spec in bench.WORKLOADS.items():
        assert 7 <= len(spec) <= 9, name
        model, dims, shape, dt, st, dtype, sub = spec[:7]
        assert model in models and dims in (2, 3) and len(shape) == dims, name
        assert all(int(n) >= 1 for n in shape) and dt > 0 and sub >= 1, name
        assert dtype in (0, 1, 2), name
        if st != 6:  # fixed stencils: 0-2 are 2D, 3-5 are 3D
            assert (st < 3) == (dims == 2), name
        if len(spec) > 7:
            assert spec[7] in (1, 2, 4), name
        if len(spec) > 8:
            assert spec[8] in (0, 1, 2, 3, 4, 5, 6), name
    for entry in bench.PER_CONFIG:
        assert entry[1] in bench.WORKLOADS, entry

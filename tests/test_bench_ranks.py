"""Host logic of the bench on the CPU: the multi-replica path on two gloo ranks (the whole-job
time is the slowest rank's, the work summed over ranks), the request-stream statistics,
and the placement of each kernel on the roof its intensity selects."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [1.5, 2.5][rank]
    work = [1.0e6, 3.0e6][rank]
    t, w = bench.aggregate_over_ranks(dist, elapsed, work, "cpu")
    out[rank] = (t, w)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        assert out[r] == (2.5, 4.0e6)
    assert bench_value(out[0]) == pytest.approx(1.6e6)


def bench_value(res):
    t, w = res
    return w / t


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(None, 3.0, 7.0, "cpu") == (3.0, 7.0)


def test_request_stream_statistics():
    import bench
    assert bench.percentile([], 0.5) is None
    v = list(range(1, 101))  # 1 .. 100
    # nearest rank: p50 of 1..100 is the 50th value, p99 the 99th, p100 the maximum
    assert bench.percentile(v, 0.5) == 50 and bench.percentile(v, 0.99) == 99 and bench.percentile(v, 0.0) == 1
    assert bench.percentile(v, 1.0) == 100 and bench.percentile(v, 0.505) == 51
    assert bench.percentile([7.0], 0.99) == 7.0
    res = [{"t_submit": 0.0, "t_done": 0.010 * (k + 1), "status": 0 if k % 4 else -4,
            "stats": {"newton_its": 3}} for k in range(8)]
    st = bench.stream_stats(res, [1000] * 8, 2.0, {-4: "RICH_ENOTCONV_LIN"})
    assert st["failed"] == {"RICH_ENOTCONV_LIN": 2}
    assert st["dof_newton_per_s"] == 6 * 1000 * 3 / 2.0          # converged work only
    assert abs(st["latency_ms_all"]["max"] - 80.0) < 1e-9 and abs(st["latency_ms_all"]["mean"] - 45.0) < 1e-9
    assert st["converged"] == 6 and st["failure_rate"] == 0.25 and st["converged_per_s"] == 3.0
    assert abs(st["latency_ms_converged"]["p50"] - 40.0) < 1e-9  # 20,30,40,60,70,80 -> nearest rank 3


def test_serving_run_end_to_end_against_a_fake_server(monkeypatch):
    # the request-stream driver with a stand-in for the request server (no GPU):
    # every request "converges" in 2 Newton iterations, 5 ms after submission
    import types
    import numpy as np
    import bench
    from paper_2112_05051_gb300 import synth

    class FakeServer:
        def __init__(self, slots=8, **kw):
            self.t = 0.0
            self.out = {}

        def submit(self, grid, soil, bc, kmean, dt, p0=None, ks=None, precision=1, opts=None, session=0):
            rid = len(self.out) + 1
            self.t += 0.001
            self.out[rid] = {"status": 0 if kmean != 2 else -4, "stats": {"newton_its": 2}, "t_submit": self.t,
                             "t_done": self.t + 0.005, "p": np.full(grid.n, -61.5)}
            return rid

        def wait(self, rid):
            return self.out.pop(rid)

        def counters(self):
            return {"admitted": 0, "max_in_flight": 3, "reserved_bytes": 0.0}

        def close(self):
            pass

    fake = types.SimpleNamespace(Server=FakeServer, PREC_MIXED=1, KRYLOV_FCG=0, ERRORS={-4: "RICH_ENOTCONV_LIN"},
                                 default_newton_opts=lambda **kw: None)
    monkeypatch.setattr(synth, "ks_field", lambda grid, seed, sigma, *a, **k: np.ones(grid.n))
    args = types.SimpleNamespace(serving_requests=12, serving_slots=3, serving_lists=1, serving_coarse_max=500,
                                 serving_aggregation=0)
    out = bench.serving_run(args, fake)
    assert out["requests"] == 12 and out["max_in_flight"] == 3
    assert out["capacity_rps"] > 0 and out["latency_ms_converged"]["p50"] == pytest.approx(5.0, abs=1e-6)
    assert 0.0 < out["failure_rate"] < 1.0
    assert set(out["failed"]) <= {"RICH_ENOTCONV_LIN"}
    assert out["mix_vs_alone_max_rel_dev"] == 0.0


def test_kernels_are_placed_on_the_roof_their_intensity_selects():
    # the bound follows from algorithmic flops/byte against the FP64 balance point:
    # FP64 kernels above it are FP64-FMA-bound, below it and every FP32 kernel HBM-bound
    sys.path.insert(0, ROOT)
    import bench
    peak_gbs, fp64_tf = 6761.6, 1.0544
    bal = bench.fp64_balance(peak_gbs, fp64_tf)
    assert abs(bal - 0.15594) < 1e-4
    n, nv, ms = 2097152, 20, 0.1
    # CGS dots over nv basis vectors: 2 n nv flops on 8 n (nv + 1) bytes, intensity 0.238
    r = bench.roofline_of("multidot", ms, 1, 8.0 * n * (nv + 1), 2.0 * n * nv, True, peak_gbs, fp64_tf, None)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["peak"] == fp64_tf
    assert abs(r["achieved"] - 2.0 * n * nv / 1e-4 / 1e12) < 1e-9 and abs(r["frac"] - r["achieved"] / fp64_tf) < 1e-12
    # a prolongation: 2 flops per entry on 12 B per entry plus the vectors, intensity < 0.156
    nnz = 3.4 * n
    r = bench.roofline_of("prolong", ms, 1, 12.0 * nnz + 20.0 * n, 2.0 * nnz, True, peak_gbs, fp64_tf, None)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == peak_gbs
    assert abs(r["frac"] - (12.0 * nnz + 20.0 * n) / 1e-4 / 1e9 / peak_gbs) < 1e-12
    # the same CGS intensity in an FP32 kernel is HBM-bound (no FP64 pipe involved)
    r = bench.roofline_of("l1jacobi", ms, 1, 8.0 * n * (nv + 1), 2.0 * n * nv, False, peak_gbs, fp64_tf, None)
    assert r["bound"] == "hbm" and r["fp64_frac"] is None
    # launch averages
    r = bench.roofline_of("restrict", 2.0, 4, 4e8, 1e7, True, peak_gbs, fp64_tf, 1.1e8)
    assert r["avg_launch_us"] == 500.0 and r["algorithmic_bytes_per_launch"] == 1e8 and r["traffic"] == 1.1e8

"""Multi-rank bench logic on CPU (gloo, world size 2): every rank times its own
replica, rank 0 reports the steps of all ranks over the slowest rank's time,
and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 * (rank + 1)
        m = bench.max_over_ranks(ms, world, "cpu")
        v = bench.whole_job_value(10, world, m)

        class A:
            steps, warmup, workload, cpu_budget = 1, 3, "tg2d_32", 1.0
        ref = bench.run_reference(A, rank, world)
        out.put((rank, m, v, ref is None))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_value():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v, ref_none in res:
        assert m == 200.0                      # the slowest rank's time on every rank
        assert v == pytest.approx(2 * 10 / 0.2)
        assert ref_none == (rank != 0)         # reference arm: rank 0 only


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_value(4, 1, 500.0) == pytest.approx(8.0)


def test_family_bytes_model_on_a_small_mesh():
    """The algorithmic-byte model of the bench's roofline, on a mesh whose sizes are
    known: each family's per-launch bytes follow its stated formula."""
    sys.path.insert(0, ROOT)
    import bench
    from workloads import problems as WP
    pb = WP.stress_cube(4)
    N, T = pb.mesh.n_dofs, pb.mesh.n_cells
    Z = 1000
    tuning = {"candidates": [{"col16": 1, "us": 1.0}]}
    amg = {"levels": 3, "rows": [N, 20, 3], "nnz": [Z, 200, 9], "p_nnz": [300, 40]}
    f = bench.family_bytes(pb, Z, None, tuning, amg)
    ns = (N + 31) // 32
    assert f["pcg_spmv"][1] == 6 * Z + 12 * N + 8 * ns
    assert f["amg_fine"][1] == 4 * Z + 16 * N + 8 * ns
    assert f["bicg_spmm"][1] == 8 * Z + 4 * (N + 1) + 36 * N
    want_t = (12 * 300 + 16 * N + 12 * 20) + (12 * 40 + 16 * 20 + 12 * 3)
    assert abs(f["amg_transfer"][1] - want_t / 4) < 1e-9
    want_c = 2 * (6 * 200 + 20 * 20) + 4 * 3 * 4 + 8 * 3
    assert abs(f["amg_coarse"][1] - want_c / 3) < 1e-9
    assert f["assemble"][1] == 128 * T + 28 * Z + 204 * N
    assert f["outer"][1] == 10 * Z + 84 * N
    assert f["pcg_update"][1] == 40 * N
    # without 16-bit columns the column bytes are 4 per entry
    f32 = bench.family_bytes(pb, Z, None, {"candidates": [{"col16": 0, "us": 1.0}]}, amg)
    assert f32["pcg_spmv"][1] - f["pcg_spmv"][1] == 2 * Z
    # pair-packed level-1 matrix and level-0 transfers: 4 bytes per entry, slice headers
    fp = bench.family_bytes(pb, Z, None, tuning, dict(amg, packed=[6, 1]))
    want_tp = (8 * 300 + 12.5 * N + 8.5 * 20) + (12 * 40 + 16 * 20 + 12 * 3)
    assert abs(fp["amg_transfer"][1] - want_tp / 4) < 1e-9
    want_cp = 2 * (4 * 200 + 16.5 * 20) + 4 * 3 * 4 + 8 * 3
    assert abs(fp["amg_coarse"][1] - want_cp / 3) < 1e-9
    # a packed restriction that keeps 32-bit columns: 6 bytes per entry
    fw = bench.family_bytes(pb, Z, None, tuning, dict(amg, packed=[6 | 16, 1]))
    assert abs((fw["amg_transfer"][1] - fp["amg_transfer"][1]) * 4 - 2 * 300) < 1e-9
    # a BiCGStab product shape with 16-bit column offsets: 6 bytes per entry
    t16 = dict(tuning, bicg_chosen=2, bicg_candidates=[{"lanes": 0, "col16": 0},
                                                       {"lanes": 2, "rows": 4, "min_blocks": 1, "col16": 1}])
    f16 = bench.family_bytes(pb, Z, None, t16, amg)
    assert f16["bicg_spmm"][1] == 6 * Z + 4 * (N + 1) + 36 * N

"""The allocation-free entry point against the allocating one.

oasis_spmv_dot_f64_noalloc serves callers that cannot allocate device memory
(code running under a caller-owned memory pool or inside an allocator, or on a
device that is already full): its reduction scratch is a static device array.
It must give the same product and dot as oasis_spmv_dot_f64, call after call,
and must not change the device's free memory.  This file is collected last so
that a failure here never hides the other GPU tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03643_gb300 import build
    build.build()
    from paper_1602_03643_gb300 import capi as c
    from workloads import meshes as WM

    m = WM.jitter_interior(WM.box_mesh_3d(12, 11, 10), 0.2, 1 / 12, seed=9)
    h = c.oasis_mesh_create(m.dim, m.coords, m.cells, m.dof_of_vertex, m.n_dofs)
    try:
        c.oasis_assemble_constant(h)
        rng = np.random.default_rng(11)
        for which in (c.OASIS_MAT_K, c.OASIS_MAT_M):
            x = torch.tensor(rng.normal(size=m.n_dofs), device="cuda")
            y_ref = torch.empty_like(x)
            xy_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
            c.oasis_spmv_dot_f64(h, which, x, y_ref, xy_ref)
            torch.cuda.synchronize()
            y = torch.full_like(x, float("nan"))
            xy = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            free_before = torch.cuda.mem_get_info()[0]
            for _ in range(2):                                 # two calls in a row
                y.fill_(float("nan"))
                xy.fill_(float("nan"))
                c.oasis_spmv_dot_f64_noalloc(h, which, x, y, xy)
                torch.cuda.synchronize()
                yn, yr = y.cpu().numpy(), y_ref.cpu().numpy()
                np.testing.assert_allclose(yn, yr, rtol=0, atol=1e-13 * np.abs(yr).max())
                assert abs(xy.item() - xy_ref.item()) <= 1e-12 * abs(xy_ref.item())
            assert torch.cuda.mem_get_info()[0] == free_before
    finally:
        c.oasis_mesh_destroy(h)

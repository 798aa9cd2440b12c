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


def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_03643_gb300 import build
    build.build()
    from paper_1602_03643_gb300 import capi as c
    return torch, c


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    torch, c = _lib()
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


def test_noalloc_alternating_meshes_on_a_user_stream_bitwise():
    """Two meshes of different sizes, calls alternating on one user stream, the
    larger mesh with more 256-row tiles (1,073) than the kernel's grid (at most
    4 blocks per SM), so each block walks several tiles.  The shared scratch
    and its ticket carry over from call to call; every result must equal the
    allocating entry point's bit for bit (same kernel, same grid, same order)."""
    torch, c = _lib()
    from workloads import meshes as WM

    meshes = [WM.box_mesh_3d(64, 64, 64),                               # 274,625 dofs
              WM.jitter_interior(WM.box_mesh_3d(9, 7, 8), 0.2, 1 / 9, seed=4)]
    stream = torch.cuda.Stream()
    handles, refs = [], []
    rng = np.random.default_rng(5)
    try:
        for m in meshes:
            h = c.oasis_mesh_create(m.dim, m.coords, m.cells, m.dof_of_vertex, m.n_dofs)
            handles.append(h)
            c.oasis_assemble_constant(h, stream)
        with torch.cuda.stream(stream):
            for h, m in zip(handles, meshes):
                x = torch.tensor(rng.normal(size=m.n_dofs), device="cuda")
                y = torch.empty_like(x)
                xy = torch.zeros(1, dtype=torch.float64, device="cuda")
                c.oasis_spmv_dot_f64(h, c.OASIS_MAT_K, x, y, xy, stream)
                refs.append((x, y, xy))
            outs = [(torch.empty_like(x), torch.empty(1, dtype=torch.float64, device="cuda")) for x, _, _ in refs]
        stream.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        for rep in range(3):
            for k in (0, 1):
                y, xy = outs[k]
                with torch.cuda.stream(stream):
                    y.fill_(float("nan"))
                    xy.fill_(float("nan"))
                c.oasis_spmv_dot_f64_noalloc(handles[k], c.OASIS_MAT_K, refs[k][0], y, xy, stream)
                stream.synchronize()
                assert torch.equal(y, refs[k][1]), (rep, k)
                assert xy.item() == refs[k][2].item(), (rep, k, xy.item(), refs[k][2].item())
        assert torch.cuda.mem_get_info()[0] == free_before
    finally:
        for h in handles:
            c.oasis_mesh_destroy(h)


def test_noalloc_rejects_a_mesh_beyond_its_scratch_on_the_host():
    """The static scratch holds one partial per 256-row tile, 65,536 tiles: a
    mesh with 16,777,217 dofs is refused with OASIS_EINVAL before any launch.
    The mesh has one cell (the other vertices carry isolated dofs) and is not
    assembled: the bound depends on its size alone."""
    torch, c = _lib()
    n = 65536 * 256 + 1
    coords = np.zeros((n, 3))
    coords[1, 0] = coords[2, 1] = coords[3, 2] = 1.0
    cells = np.array([[0, 1, 2, 3]], dtype=np.int32)
    h = c.oasis_mesh_create(3, coords, cells)
    try:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        xy = torch.zeros(1, dtype=torch.float64, device="cuda")
        with pytest.raises(c.OasisError) as e:
            c.oasis_spmv_dot_f64_noalloc(h, c.OASIS_MAT_K, x, y, xy)
        assert e.value.code == c.OASIS_EINVAL
        assert "static scratch" in str(e.value)
        torch.cuda.synchronize()
    finally:
        c.oasis_mesh_destroy(h)

"""Edge and degenerate cases of the boundary.

CPU: malformed meshes and arguments are rejected by aimx_setup on the host
before any device work (degenerate triangle, edge shared by three triangles,
inconsistent orientation, vertex id out of range, no interior edge, stencil
order and grid-size limits).  GPU: the smallest problem (two triangles, one
RWG function, open surface) against the oracle, and argument errors of the
product and solve calls (no right-hand sides, null buffers, non-positive
frequency).
"""

import ctypes

import numpy as np
import pytest

C0 = 299792458.0
E_ARG, E_MESH, E_GRID = -1, -2, -3


def _setup_rc(xyz, tri, grid=(8, 8, 8), order=2):
    from paper_2009_02281_gb300 import aimx
    lib = aimx.load(build_if_missing=True)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    mesh = aimx._Mesh(len(xyz), len(tri), xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    mat = aimx._Material(0, 1.0, 1.0, 1.0, 1.0, 0.0)
    g = aimx._Grid()
    for a in range(3):
        g.n[a] = grid[a]
    g.near_radius = 3
    out = ctypes.c_void_p()
    rc = lib.aimx_setup(ctypes.byref(mesh), ctypes.byref(mat), ctypes.byref(g), order, ctypes.byref(out))
    if rc == 0:
        lib.aimx_destroy(out)
    return rc


def _tet():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    tri = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2]])
    return xyz, tri


def test_degenerate_triangle_rejected():
    xyz, tri = _tet()
    xyz = np.vstack([xyz, [[2, 0, 0]]])
    tri = np.vstack([tri, [[0, 1, 4]]])          # collinear vertices 0, 1, 4
    assert _setup_rc(xyz, tri) == E_MESH


def test_edge_shared_by_three_triangles_rejected():
    xyz, tri = _tet()
    xyz = np.vstack([xyz, [[0.5, -1, 0.3]]])
    tri = np.vstack([tri, [[0, 1, 4]]])          # third triangle on edge (0, 1)
    assert _setup_rc(xyz, tri) == E_MESH


def test_inconsistent_orientation_rejected():
    xyz, tri = _tet()
    tri = tri.copy()
    tri[1] = tri[1][[0, 2, 1]]
    assert _setup_rc(xyz, tri) == E_MESH


def test_vertex_id_out_of_range_rejected():
    xyz, tri = _tet()
    tri = tri.copy()
    tri[2, 1] = 7
    assert _setup_rc(xyz, tri) == E_MESH


def test_single_triangle_has_no_basis():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float)
    assert _setup_rc(xyz, np.array([[0, 1, 2]])) == E_MESH


def test_order_and_grid_limits():
    xyz, tri = _tet()
    assert _setup_rc(xyz, tri, order=0) == E_ARG
    assert _setup_rc(xyz, tri, order=4) == E_ARG
    assert _setup_rc(xyz, tri, grid=(3, 8, 8), order=2) == E_ARG


# ------------------------------------------------------------------ GPU

@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_02281_gb300 import build
    build.build()
    return torch


@pytest.mark.gpu
def test_two_triangle_plate_matches_oracle(torch_cuda):
    """The smallest problem: one RWG function on an open two-triangle plate."""
    torch = torch_cuda
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, EFIE
    xyz = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [0.1, 0.1, 0.0]])
    tri = np.array([[0, 1, 2], [1, 3, 2]])
    ctx = Context(xyz, tri, (8, 8, 8), formulation=EFIE)
    assert ctx.N == 1
    prob = op.setup(xyz, tri, 2, (8, 8, 8), radius=3)
    f = 3e8
    x = np.array([[1.0 - 0.5j]])
    ref = op.matvec_efie(prob, f, x[0])
    for dt, tol in ((torch.complex128, 1e-9), (torch.complex64, 1e-5)):
        y = ctx.matvec(f, torch.tensor(x, dtype=dt, device="cuda")).cpu().numpy()[0]
        assert np.abs(y - ref).max() <= tol * np.abs(ref).max()
    ctx.close()


@pytest.mark.gpu
def test_product_and_solve_argument_errors(torch_cuda):
    torch = torch_cuda
    from synth import icosphere
    from paper_2009_02281_gb300 import Context, EFIE, aimx
    xyz, tri = icosphere(1)
    ctx = Context(xyz, tri, (8, 8, 8), formulation=EFIE)
    lib = aimx.load()
    x = torch.zeros((1, ctx.nunk), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    xp, yp = ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())
    assert lib.aimx_matvec(ctx._ctx, 1e8, 0, xp, yp, 0, None) == E_ARG            # no right-hand side
    assert lib.aimx_matvec(ctx._ctx, 1e8, 1, None, yp, 0, None) == E_ARG          # null input
    assert lib.aimx_matvec(ctx._ctx, 0.0, 1, xp, yp, 0, None) == E_ARG            # frequency <= 0
    assert lib.aimx_matvec(ctx._ctx, 1e8, 1, xp, yp, 7, None) == E_ARG            # unknown precision
    b = torch.zeros((1, ctx.nunk), dtype=torch.complex128, device="cuda")
    xs = torch.empty_like(b)
    assert lib.aimx_solve(ctx._ctx, 1e8, 0, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(xs.data_ptr()),
                          None, None, None) == E_ARG
    # a zero right-hand side is solved exactly by x = 0
    xz, st, rc = ctx.solve(1e8, b)
    assert rc == 0 and np.all(xz.cpu().numpy() == 0) and st[0]["rel_residual"] == 0.0
    ctx.close()

"""The allocation-free Poisson entry point, for callers that cannot allocate
device memory when they need a solve (they hand the library raw pointers and
own every allocation themselves).  Its output must match the handle-based
fsei_poisson_solve on the same right-hand side, on two calls in a row (the
second call reuses the shared static scratch the first one left behind, with
a narrower spectrum row than the first call's, so stale padding would show).
In mixed precision the entry point solves its near-zero modes in double from
factors formed on the fly, where a grid handle uses factors made at grid
creation: both are also held to the FP64 oracle.  This file is collected
last on purpose."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12          # FP64: the two entry points against each other
TOL_MIXED = 1e-5     # FSEI_MIXED: against each other and against the oracle


def _rhs(shape, dz, seed):
    rng = np.random.default_rng(seed)
    s = rng.standard_normal(shape)
    w = dz[:, None, None] * np.ones(shape)
    return s - (s * w).sum() / w.sum()


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
@pytest.mark.parametrize("zbc,stretch", [(1, 2.0), (0, 0.0)])
def test_noalloc_poisson_matches_handle_solve_twice(zbc, stretch, prec_name):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15187_gb300 import fsei
    from paper_2103_15187_gb300.inputs import z_faces
    from oracle.grid import Grid as OGrid
    from oracle.poisson import oracle_poisson
    lib = fsei.load()
    prec = fsei.FSEI_FP64 if prec_name == "fp64" else fsei.FSEI_MIXED
    dtype = torch.float64 if prec_name == "fp64" else torch.float32
    tol = TOL if prec_name == "fp64" else TOL_MIXED
    fn = lib.fsei_poisson_solve_noalloc
    fn.argtypes = [ctypes.POINTER(fsei.GridDesc), ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    stream = torch.cuda.current_stream()
    # spectrum rows of 64 then 32 complex values (nx/2 + 1 rounded up to 16)
    for call, (nx, ny, nz) in enumerate([(96, 36, 20), (32, 24, 40)]):
        d = fsei.GridDesc()
        d.nx, d.ny, d.nz = nx, ny, nz
        d.lx, d.ly, d.zbc, d.lz, d.stretch = 2 * np.pi, np.pi, zbc, 2.0, stretch
        d.prec = prec
        d.near_zero_tau = 0.0
        zf = z_faces(nz, zbc, 2.0, stretch)
        s = _rhs((nz, ny, nx), zf[1:] - zf[:-1], 100 + call)
        rhs = torch.tensor(s, dtype=dtype, device="cuda")
        phi_static = torch.full_like(rhs, float("nan"))
        st = fn(ctypes.byref(d), ctypes.c_void_p(rhs.data_ptr()),
                ctypes.c_void_p(phi_static.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, st
        grid = fsei.Grid(nx, ny, nz, 2 * np.pi, np.pi, zbc=zbc, lz=2.0, stretch=stretch,
                         prec=prec)
        phi_ref = torch.empty_like(rhs)
        fsei.poisson_solve(grid, rhs, phi_ref)
        torch.cuda.synchronize()
        a = phi_static.double().cpu().numpy()
        b = phi_ref.double().cpu().numpy()
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= tol, (call, err)
        if prec_name == "mixed":
            g = OGrid(nx, ny, nz, 2 * np.pi, np.pi, zbc, lz=2.0, stretch=stretch)
            ref = oracle_poisson(g, rhs.double().cpu().numpy())
            err_o = np.linalg.norm(a - ref) / np.linalg.norm(ref)
            assert err_o <= TOL_MIXED, (call, err_o)


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    from paper_2103_15187_gb300 import fsei
    lib = fsei.load()
    fn = lib.fsei_poisson_solve_noalloc
    fn.argtypes = [ctypes.POINTER(fsei.GridDesc), ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    d = fsei.GridDesc()
    d.nx, d.ny, d.nz = 512, 512, 512
    d.lx, d.ly, d.zbc, d.lz, d.stretch = 1.0, 1.0, 1, 2.0, 2.0
    d.prec = fsei.FSEI_FP64
    # 16-byte aligned non-null stand-ins: the size check comes before any
    # device work, so nothing is read or written through them
    assert fn(ctypes.byref(d), ctypes.c_void_p(256), ctypes.c_void_p(256), None) == 2


def test_noalloc_refuses_stream_capture():
    """A call on a stream being captured is refused (its copies from the
    static host buffer would replay after later calls rewrote it)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15187_gb300 import fsei
    lib = fsei.load()
    fn = lib.fsei_poisson_solve_noalloc
    fn.argtypes = [ctypes.POINTER(fsei.GridDesc), ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    d = fsei.GridDesc()
    d.nx, d.ny, d.nz = 32, 24, 40
    d.lx, d.ly, d.zbc, d.lz, d.stretch = 2 * np.pi, np.pi, 1, 2.0, 2.0
    d.prec = fsei.FSEI_FP64
    rhs = torch.zeros((40, 24, 32), dtype=torch.float64, device="cuda")
    phi = torch.zeros_like(rhs)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            st = fn(ctypes.byref(d), ctypes.c_void_p(rhs.data_ptr()),
                    ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(side.cuda_stream))
    assert st == 1

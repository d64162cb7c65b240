"""The allocation-free FP32 product agrees with aimx_matvec (collected last on purpose).

aimx_matvec_noalloc serves callers that cannot allocate device memory when
they need the product (a fixed memory budget, an allocator owned by another
framework): its work buffers live in one static device array of the library.
This test calls it through the C ABI on two calls in a row and compares each
result with the ordinary entry point's, within the FP32 tolerance of the
parity tests.  It works both alone in a fresh process and after the other
tests, because it builds its own context and makes the one ordinary FP32 call
that the no-alloc entry point requires first.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0
TOL32 = 1e-5


def test_noalloc_matches_matvec_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from synth import icosphere, random_complex
    from paper_2009_02281_gb300 import Context, PMCHWT, F32, build, aimx
    build.build()
    lib = aimx.load()
    xyz, tri = icosphere(2)
    ctx = Context(xyz, tri, (16, 16, 16), order=2, formulation=PMCHWT, eps_out=1.0, eps_in=4.0)
    assert ctx.matvec_path(F32) == 0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (seed, kfac) in enumerate(((41, 1.2), (42, 0.8))):
        freq = kfac * C0 / (2 * np.pi)
        x = torch.tensor(random_complex((3, ctx.nunk), seed=seed), dtype=torch.complex64, device="cuda")
        y_ref = ctx.matvec(freq, x)                       # ordinary entry point (allocates on first use)
        y = torch.full_like(x, complex(float("nan"), float("nan")))
        rc = lib.aimx_matvec_noalloc(ctx._ctx, freq, x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()), stream)
        assert rc == 0, lib.aimx_last_error(ctx._ctx)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL32, call
    # requests beyond the static array are refused with a clear message
    big = 1 << 20
    rc = lib.aimx_matvec_noalloc(ctx._ctx, 1e8, big, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 stream)
    assert rc == -1
    assert b"static limit" in lib.aimx_last_error(ctx._ctx)
    ctx.close()

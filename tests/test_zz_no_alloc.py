"""The allocation-free FP32 product agrees with aimx_matvec (collected last on purpose).

aimx_matvec_noalloc serves callers that cannot allocate device memory when
they need the product (a fixed memory budget, an allocator owned by another
framework): its work buffers live in one static device array of the library.
This test calls it through the C ABI on calls in a row and compares each
result with the ordinary entry point's, within the FP32 tolerance of the
parity tests.  One call is at a frequency the context has not seen, so the
entry point regenerates the kernel spectra itself; that result is also
checked against the FP64 oracle.  Device memory in use (the context's own
book-keeping and the device's free memory) must not change across the
allocation-free calls, with the default z-pass and with the TMA-pipelined
one; the only change allowed is on the very first call, when the library's
fixed static array becomes resident on the device.  It works both alone in a fresh process and after the other tests,
because it builds its own context and makes the one ordinary FP32 call that
the no-alloc entry point requires first.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0
TOL32 = 1e-5


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_matvec_and_allocates_nothing():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from synth import icosphere, random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import Context, PMCHWT, F32, build, aimx, wait_timeouts
    build.build()
    lib = aimx.load()
    xyz, tri = icosphere(2)
    grid = (16, 16, 16)
    ctx = Context(xyz, tri, grid, order=2, formulation=PMCHWT, eps_out=1.0, eps_in=4.0)
    assert ctx.matvec_path(F32) == 0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    nrhs = 3
    kfacs = (1.2, 0.8, 1.05, 0.95)            # one frequency per call (k a / pi)
    xs = [torch.tensor(random_complex((nrhs, ctx.nunk), seed=41 + i), dtype=torch.complex64, device="cuda")
          for i in range(len(kfacs))]
    ys = [torch.full_like(x, complex(float("nan"), float("nan"))) for x in xs]

    def noalloc(i):
        freq = kfacs[i] * C0 / (2 * np.pi)
        rc = lib.aimx_matvec_noalloc(ctx._ctx, freq, nrhs, ctypes.c_void_p(xs[i].data_ptr()),
                                     ctypes.c_void_p(ys[i].data_ptr()), stream)
        assert rc == 0, lib.aimx_last_error(ctx._ctx)

    def memory_state():
        torch.cuda.synchronize()
        return ctx._info()["device_bytes"], torch.cuda.mem_get_info()[0]

    # the one ordinary FP32 call the entry point requires (allocates the context's buffers)
    f0 = kfacs[0] * C0 / (2 * np.pi)
    y_ref0 = ctx.matvec(f0, xs[0])
    first = memory_state()
    noalloc(0)                                  # same frequency as the ordinary call
    before = memory_state()
    # The first call resolves the static array's device address, which makes the library's
    # fixed 64 MiB array resident on this device (once per process); nothing else may appear.
    assert before[0] == first[0]
    assert 0 <= first[1] - before[1] <= (64 + 2) << 20, (first, before)
    noalloc(1)                                  # a new frequency: spectra regenerated in place
    after = memory_state()
    assert after == before, "device memory changed across aimx_matvec_noalloc: %s -> %s" % (before, after)
    f1 = kfacs[1] * C0 / (2 * np.pi)
    y_ref1 = ctx.matvec(f1, xs[1])              # ordinary entry point at the new frequency, afterwards
    torch.cuda.synchronize()
    for y, yr in ((ys[0], y_ref0), (ys[1], y_ref1)):
        a, b = y.cpu().numpy(), yr.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert _rel(a, b) <= TOL32
    # the regenerating call against the FP64 oracle
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    x1 = xs[1].cpu().numpy().astype(np.complex128)
    ref1 = np.stack([op.matvec_pmchwt(prob, f1, xi, 1.0, 4.0) for xi in x1])
    assert _rel(ys[1].cpu().numpy(), ref1) <= TOL32

    # the TMA-pipelined z-pass (schedule variant 3) on the static array
    ctx.set_schedule(3)
    assert ctx.matvec_path(F32) == 0
    f2 = kfacs[2] * C0 / (2 * np.pi)
    ctx.matvec(f2, xs[2])                       # loads the variant's kernels before measuring
    before = memory_state()
    noalloc(2)                                  # spectra of f2 are current
    noalloc(3)                                  # a new frequency again
    after = memory_state()
    assert after == before, "device memory changed across aimx_matvec_noalloc (variant 3)"
    assert wait_timeouts() == 0
    f3 = kfacs[3] * C0 / (2 * np.pi)
    y_ref2 = ctx.matvec(f2, xs[2])
    y_ref3 = ctx.matvec(f3, xs[3])
    torch.cuda.synchronize()
    for y, yr in ((ys[2], y_ref2), (ys[3], y_ref3)):
        a, b = y.cpu().numpy(), yr.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert _rel(a, b) <= TOL32
    ctx.set_schedule(0)

    # requests beyond the static array are refused with a clear message
    big = 1 << 20
    rc = lib.aimx_matvec_noalloc(ctx._ctx, 1e8, big, ctypes.c_void_p(xs[0].data_ptr()),
                                 ctypes.c_void_p(ys[0].data_ptr()), stream)
    assert rc == -1
    assert b"static limit" in lib.aimx_last_error(ctx._ctx)
    # a context whose FP32 products are routed to the generic path is refused
    ctx.set_path(1)
    rc = lib.aimx_matvec_noalloc(ctx._ctx, f0, nrhs, ctypes.c_void_p(xs[0].data_ptr()),
                                 ctypes.c_void_p(ys[0].data_ptr()), stream)
    assert rc == -7
    ctx.close()

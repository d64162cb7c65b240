"""The bounded copy wait of the TMA-pipelined z-pass runs out and is reported.

The per-tile wait's limit is shortened through the test hook (aimx_set_wait_limit) so that it
gives up before the copy completes: the product then reports the timeouts through
aimx_wait_timeouts, and after the default limit is restored the same context computes correct
products again (oracle tolerance), with no further timeouts.  No GPU fault is involved: a block
whose wait ran out drains its one copy in flight with the full bound and returns.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C0 = 299792458.0


def test_tile_wait_runs_out_and_context_recovers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from synth import icosphere, random_complex
    from oracle import operator as op
    from paper_2009_02281_gb300 import build, Context, PMCHWT, F32, wait_timeouts
    from paper_2009_02281_gb300.aimx import set_wait_limit
    build.build()
    xyz, tri = icosphere(2)
    grid = (16, 16, 16)
    ctx = Context(xyz, tri, grid, order=2, formulation=PMCHWT, eps_out=1.0, eps_in=4.0)
    ctx.set_schedule(3)
    assert ctx.matvec_path(F32) == 0
    f = 1.1 * C0 / (2 * np.pi)
    x = torch.tensor(random_complex((4, ctx.nunk), seed=81), dtype=torch.complex64, device="cuda")
    ctx.matvec(f, x)
    torch.cuda.synchronize()
    assert wait_timeouts() == 0
    try:
        set_wait_limit(1)                 # one cycle: the first poll of each block gives up
        ctx.matvec(f, x)
        torch.cuda.synchronize()
        n = wait_timeouts()
    finally:
        set_wait_limit(0)
    assert n >= 1
    y = ctx.matvec(f, x).cpu().numpy()
    torch.cuda.synchronize()
    assert wait_timeouts() == 0
    prob = op.setup(xyz, tri, 2, grid, radius=3)
    xh = x.cpu().numpy().astype(np.complex128)
    ref = np.stack([op.matvec_pmchwt(prob, f, xi, 1.0, 4.0) for xi in xh])
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-5
    ctx.close()

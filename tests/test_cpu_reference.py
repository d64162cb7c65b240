"""The benchmark's host-side timing baselines (CPU only).

The FFT-based FP64 CPU product that the benchmark times beside the GPU (a
timing baseline, not the oracle) must compute the same AIMx operator as the
oracle's direct grid summation: on a small sphere, with the exact near rows,
it reproduces every output row of the oracle's EFIE and two-region products
to rounding.  Also: the single-thread oracle run in a fresh interpreter, and
the host description.
"""

import numpy as np
import pytest

C0 = 299792458.0


def _small(formulation):
    from synth.meshes import icosphere
    xyz, tri = icosphere(2)
    wl = dict(name="small", xyz=xyz, tri=tri, formulation=formulation, eps_out=1.0,
              eps_in=4.0 if formulation == "pmchwt" else None, grid_n=(10, 10, 10), order=2, radius=2,
              freq=0.4 * C0)
    return wl


@pytest.mark.parametrize("formulation", ["efie", "pmchwt"])
def test_fft_product_matches_oracle_on_every_row(formulation):
    import bench
    wl = _small(formulation)
    nb = len(wl["tri"]) * 3 // 2
    s = bench.OracleSample(wl, nb)            # 997 is prime: the sampled rows cover every basis
    assert len(np.unique(s.rows)) == nb
    s.run(s.rows)
    fc = bench.FastCpuAIMx(s, workers=2)
    y = s.sampled(fc.far(s.x)) + fc.near_exact_rows(s.x)
    assert np.linalg.norm(y - s.y) <= 1e-12 * np.linalg.norm(s.y)
    # the far part alone differs from the oracle's product by the near correction, which is not small
    yf = s.sampled(fc.far(s.x))
    assert np.linalg.norm(yf - s.y) > 1e-3 * np.linalg.norm(s.y)


def test_fast_reference_record():
    import bench
    wl = _small("efie")
    s = bench.OracleSample(wl, 8)
    s.run(s.rows)
    r = bench.fast_cpu_reference(s, reps=1)
    assert r["rel_err_vs_oracle_on_sample"] < 1e-12
    assert r["value"] > 0 and r["cores"] >= 1
    assert "timing baseline" in r["kind"]


def test_single_thread_oracle_and_host():
    import bench
    from synth import workloads
    r = bench.oracle_single_thread(workloads.pec_sphere_1920(), 2)
    assert "error" not in r, r
    assert r["cores"] == 1 and r["value"] > 0
    h = bench.host_cpu()
    assert h["nproc"] >= 1 and h["machine"]

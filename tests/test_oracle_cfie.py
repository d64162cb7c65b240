"""Pins of the CFIE oracle for closed PEC bodies (Sec. III-B, Eqs. MFIEout, CFIEout, KAIMx, CFIEAIMx).

* RCS of the CFIE solution against the PEC Mie series, and the CFIE current
  against the EFIE current (same physics, different equation),
* the MFIE part is second-kind: the CFIE stays well conditioned where the
  EFIE passes through the sphere's first interior (TM) resonance,
* the static K_g part is exactly zero (principal value) on a flat plate,
* the rotated weights integrate n x f exactly (partition of unity),
* with alpha = 1 the CFIE is the EFIE.
"""

import numpy as np
import pytest

from oracle import cfie, excitation, farfield, mie, solve
from oracle import operator as op
from oracle.constants import MU0
from oracle.rwg import rwg_arrays
from synth import icosphere

C0 = 299792458.0


@pytest.fixture(scope="module")
def sphere_l1():
    xyz, tri = icosphere(1)
    return cfie.setup_cfie(op.setup(xyz, tri, 2, (8, 8, 8), radius=3))


@pytest.fixture(scope="module")
def sphere_l2():
    xyz, tri = icosphere(2)
    return cfie.setup_cfie(op.setup(xyz, tri, 2, (12, 12, 12), radius=3))


def test_rcs_vs_mie_and_efie(sphere_l2):
    k = 1.0
    f = k * C0 / (2 * np.pi)
    prob = sphere_l2
    Jc = solve.lu_solve(cfie.dense_cfie(prob, f), cfie.planewave_rhs_cfie(prob["rwg"], k, [0, 0, 1], [1, 0, 0]))
    VE, _ = excitation.planewave_rhs(prob["rwg"], k, [0, 0, 1], [1, 0, 0])
    Je = solve.lu_solve(op.dense_efie(prob, f), VE)
    th = np.linspace(0.2, np.pi - 0.2, 9)
    for phi in (0.0, np.pi / 2):
        dirs = np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)], 1)
        s = farfield.rcs(farfield.far_field(prob["rwg"], Jc, k, 2 * np.pi * f, MU0, dirs))
        ref = mie.bistatic_rcs(k, 1.0, th, phi)
        assert np.max(np.abs(s - ref) / ref.max()) < 0.06
    assert np.linalg.norm(Jc - Je) / np.linalg.norm(Je) < 0.05


def test_cfie_removes_interior_resonance(sphere_l1):
    """Across ka = 2.5..3.1 the EFIE's condition number peaks (first TM cavity mode); the CFIE's does not."""
    ce, cc = [], []
    for ka in np.linspace(2.5, 3.1, 7):
        f = ka * C0 / (2 * np.pi)
        se = np.linalg.svd(op.dense_efie(sphere_l1, f), compute_uv=False)
        sc = np.linalg.svd(cfie.dense_cfie(sphere_l1, f), compute_uv=False)
        ce.append(se[0] / se[-1])
        cc.append(sc[0] / sc[-1])
    assert max(ce) > 5 * min(ce)
    assert max(cc) < 1.2 * min(cc)
    assert max(cc) < min(ce)


def test_static_kg_vanishes_between_coplanar_bases():
    """Principal value: on one flat face grad G_s x f is normal and g = n x f tangential."""
    from synth import box
    from oracle.rwg import build_rwg
    xyz, tri = box([0, 0, 0], [1.0, 1.0, 1.0], [3, 3, 3])
    rwg = build_rwg(xyz, tri)
    T, _, _, _ = rwg_arrays(rwg)
    flat = [m for m in range(rwg["n"]) if np.all(np.abs(rwg["xyz"][rwg["tri"][T[m]]][..., 2]) < 1e-12)]
    assert len(flat) >= 10
    rows = np.repeat(flat, len(flat))
    cols = np.tile(flat, len(flat))
    kg = cfie.static_kg(rwg, rows, cols)
    other = [m for m in range(rwg["n"]) if m not in flat][:10]
    assert np.abs(kg).max() <= 1e-14 * np.abs(cfie.static_kg(rwg, np.repeat(flat[:10], 10), np.tile(other, 10))).max()


def test_rotated_weights_partition_of_unity(sphere_l1):
    prob = sphere_l1
    rwg = prob["rwg"]
    T, P, C, S = rwg_arrays(rwg)
    nrm = cfie.normals(rwg)
    cen = rwg["centroid"]
    ref = np.zeros((prob["N"], 3))
    for side in range(2):
        t = T[:, side]
        ref += np.cross(nrm[t], (S[side] * C[:, side] * rwg["area"][t])[:, None] * (cen[t] - P[:, side]))
    assert np.abs(prob["lam_g"].sum(axis=1) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_alpha_one_is_the_efie(sphere_l1):
    from synth import random_complex
    f = 0.7 * C0 / (2 * np.pi)
    x = random_complex((sphere_l1["N"],), seed=9)
    assert np.allclose(cfie.matvec_cfie(sphere_l1, f, x, alpha=1.0), op.matvec_efie(sphere_l1, f, x), rtol=0,
                       atol=1e-13 * np.abs(op.matvec_efie(sphere_l1, f, x)).max())
    V1 = cfie.planewave_rhs_cfie(sphere_l1["rwg"], 0.7, [0, 0, 1], [1, 0, 0], alpha=1.0)
    VE, _ = excitation.planewave_rhs(sphere_l1["rwg"], 0.7, [0, 0, 1], [1, 0, 0])
    assert np.allclose(V1, VE, rtol=1e-14, atol=0)

"""Pins of the conventional-AIM oracle (Sec. II-B), the comparison method of the paper.

* near entries equal the dense MoM entries (computed by an independent path:
  per-triangle potential tables),
* far entries equal the AIMx grid entries,
* the per-frequency precorrection tends to the static one as k -> 0,
* G_d against its definition and its R -> 0 limit,
* AIM's own accuracy is no worse than AIMx's (the paper's comparison).
"""

import numpy as np
import pytest

from oracle import aim, mom, static
from oracle import operator as op
from synth import icosphere

C0 = 299792458.0


@pytest.fixture(scope="module")
def sphere():
    xyz, tri = icosphere(1)
    return op.setup(xyz, tri, 2, (8, 8, 8), radius=3)


def _near_mask(prob):
    m = np.zeros((prob["N"], prob["N"]), dtype=bool)
    m[prob["near"]["rows"], prob["cols"]] = True
    return m


@pytest.mark.parametrize("ka", [0.5, 1.5])
def test_near_entries_equal_mom_and_far_entries_equal_aimx(sphere, ka):
    f = ka * C0 / (2 * np.pi)
    Za = aim.dense_efie_aim(sphere, f)
    Zm = mom.dense_efie_mom(sphere["rwg"], f)[0]
    Zx = op.dense_efie(sphere, f)
    near = _near_mask(sphere)
    assert near.any() and (~near).any()
    assert np.abs(Za - Zm)[near].max() <= 1e-12 * np.abs(Zm).max()
    assert np.abs(Za - Zx)[~near].max() <= 1e-14 * np.abs(Zm).max()


def test_precorrection_tends_to_static(sphere):
    rows, cols = sphere["near"]["rows"], sphere["cols"]
    k = 1e-5
    PA, PP = aim.precorrection_k(sphere["lam"], sphere["anc"], sphere["grid"], rows, cols, k)
    SA, SP, _ = static.precorrection(sphere["lam"], sphere["anc"], sphere["grid"], rows, cols, 3)
    assert np.abs(PA.real - SA).max() <= 1e-9 * np.abs(SA).max()
    assert np.abs(PP.real - SP).max() <= 1e-9 * np.abs(SP).max()
    # the imaginary part is -k/(4 pi) times the product of the stencil sums, to O(k^3)
    lam = sphere["lam"]
    s = lam.sum(axis=1)
    ref = -k / (4 * np.pi) * np.einsum("bc,bc->b", s[rows][:, :3], s[cols][:, :3])
    assert np.abs(PA.imag - ref).max() <= 1e-6 * np.abs(ref).max() + 1e-20


def test_Gd_definition_and_limit():
    k = 2.3
    R = np.array([1e-3, 0.1, 1.0, 7.5])
    ref = (np.exp(-1j * k * R) - 1.0) / (4 * np.pi * R)
    assert np.allclose(aim.G_d(k, R), ref, rtol=1e-10, atol=0)
    assert aim.G_d(k, 0.0) == -1j * k / (4 * np.pi)
    assert abs(aim.G_d(k, 1e-9) - aim.G_d(k, 0.0)) <= 1e-8 * k


def test_matvec_matches_dense(sphere):
    from synth import random_complex
    f = 0.8 * C0 / (2 * np.pi)
    k = 0.8
    near = aim.near_aim(sphere, k)
    x = random_complex((sphere["N"],), seed=2)
    y = aim.matvec_efie_aim(sphere, f, x, near=near)
    Z = aim.dense_efie_aim(sphere, f, near=near)
    assert np.linalg.norm(y - Z @ x) <= 1e-12 * np.linalg.norm(y)


def test_aim_accuracy_no_worse_than_aimx(sphere):
    """Against the dense MoM, AIM's error is at most AIMx's (the paper reports comparable accuracy)."""
    f = 1.5 * C0 / (2 * np.pi)
    Zm = mom.dense_efie_mom(sphere["rwg"], f)[0]
    ea = np.linalg.norm(aim.dense_efie_aim(sphere, f) - Zm)
    ex = np.linalg.norm(op.dense_efie(sphere, f) - Zm)
    assert ea <= ex

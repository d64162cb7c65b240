"""Synthetic workloads shaped like the paper's examples (inputs only).

Each workload is a dict of mesh, materials, grid, stencil order, frequency and
right-hand-side batch size; the meshes are procedural (icosphere), seeded, and
stand in for the paper's geometries, which are not available.

* ``pec_sphere_1920``: PEC sphere, radius 1 m, icosphere level 3 (1280
  triangles, 1920 RWG), diameter = 1 free-space wavelength (f = c/2 Hz),
  24^3 grid (order 2, near radius 3), one x-polarised plane wave along +z,
  FP64.
* ``dielectric_sphere_61440``: eps_r = 4 sphere, radius 1 m, icosphere level 5
  (20480 triangles, 30720 RWG, two-region formulation with 61440 unknowns),
  diameter = 3 free-space wavelengths (f = 1.5 c Hz, about 449.7 MHz), 64^3 grid padded to
  128^3, order 2, near radius 3, 64 right-hand sides, FP32 matvec.
* ``conductor_bars``: 8 parallel copper bars (sigma = 5.8e7 S/m, surface
  impedance) of 1000 x 10 x 5 um with 10 um gaps in eps_r = 3.5, structured
  mesh with 3.2 um cells along the bars (75k unknowns), one delta-gap port at
  the middle of each bar, a 256 x 16 x 8 grid (padded 512 x 32 x 16), 100
  log-spaced frequencies from 1 MHz to 100 GHz.
* ``copper_blocks``: seeded layouts of 2-12 rectangular copper blocks (1-6 mm
  footprint, 0.2-1 mm thick, surface impedance) on a 20 mm square, structured
  meshes of ~0.4 mm cells: the learned preconditioner's training and held-out
  evaluation layouts.
* ``uneven_batch``: seeded mix of PEC (EFIE) and dielectric (eps_r ~ U[2, 6],
  two-region) spheres, boxes and tori of size U[0.5, 4] free-space wavelengths
  at f = c (wavelength 1 m), meshed for a log-uniform 2k-60k unknowns, each
  with a power-of-two grid per axis (8..64 nodes) chosen for a spacing of
  min(0.1 interior wavelength, mean mesh edge) and capped at 64 nodes, 4
  right-hand sides, FP32.
"""

import numpy as np

from .meshes import box, icosphere, torus

C0 = 299792458.0


def pec_sphere_1920():
    xyz, tri = icosphere(3)
    return dict(name="pec_sphere_1920", xyz=xyz, tri=tri, formulation="efie", eps_out=1.0, eps_in=None,
                grid_n=(24, 24, 24), order=2, radius=3, freq=C0 / 2.0, nrhs=1, precision="f64")


def dielectric_sphere_61440(nrhs=64):
    xyz, tri = icosphere(5)
    return dict(name="dielectric_sphere_61440", xyz=xyz, tri=tri, formulation="pmchwt", eps_out=1.0,
                eps_in=4.0, grid_n=(64, 64, 64), order=2, radius=3, freq=1.5 * C0, nrhs=nrhs,
                precision="f32")


def conductor_bars(nbars=8, length=1000e-6, width=10e-6, thickness=5e-6, gap=10e-6, divisions=(312, 3, 2)):
    """Parallel copper bars in a dielectric: the sweep workload (inputs only).

    Bars along x, side by side in y with ``gap`` between them, meshed as
    structured boxes (an even x division puts a vertex line at the middle,
    where each bar's delta-gap port sits).  Returns the merged mesh, the port
    definitions (point, normal, box_lo, box_hi) and the sweep settings."""
    from .meshes import merge_meshes
    parts, ports = [], []
    for i in range(nbars):
        y0 = i * (width + gap)
        parts.append(box([0.0, y0, 0.0], [length, y0 + width, thickness], list(divisions)))
        eps = 0.25 * gap
        ports.append(([0.5 * length, 0.0, 0.0], [1.0, 0.0, 0.0], [-eps, y0 - eps, -eps],
                      [length + eps, y0 + width + eps, thickness + eps]))
    xyz, tri, _ = merge_meshes(parts)
    return dict(name="conductor_bars_%d" % nbars, xyz=xyz, tri=tri, formulation="efie", eps_out=3.5, eps_in=None,
                sigma=5.8e7, grid_n=(256, 16, 8), order=2, radius=3, ports=ports,
                freqs=np.logspace(6, 11, 100), precision="f32")


def copper_blocks(seed, nblocks=None, edge=0.4e-3, region=20e-3, footprint=(1e-3, 6e-3)):
    """A seeded layout of rectangular copper blocks on a plane (inputs only).

    ``nblocks`` (default U{2..12}) boxes of 1-6 mm footprint and 0.2-1 mm
    height placed without overlap in a ``region`` x ``region`` square, meshed as
    structured boxes with cells of about ``edge``; sigma = 5.8e7 S/m, free
    space around them.  Returns a workload dict (EFIE with surface impedance)."""
    from .meshes import merge_meshes
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 13)) if nblocks is None else int(nblocks)
    placed, parts = [], []
    tries = 0
    while len(placed) < n and tries < 2000:
        tries += 1
        w, d = rng.uniform(footprint[0], footprint[1], size=2)
        t = rng.uniform(0.2e-3, 1e-3)
        x0, y0 = rng.uniform(0, region - w), rng.uniform(0, region - d)
        gap = 0.5e-3
        if any(x0 < bx + bw + gap and bx < x0 + w + gap and y0 < by + bd + gap and by < y0 + d + gap
               for bx, by, bw, bd in placed):
            continue
        placed.append((x0, y0, w, d))
        div = [max(1, int(round(w / edge))), max(1, int(round(d / edge))), max(1, int(round(t / edge)))]
        parts.append(box([x0, y0, 0.0], [x0 + w, y0 + d, t], div))
    xyz, tri, _ = merge_meshes(parts)
    ext = xyz.max(0) - xyz.min(0)
    grid = tuple(_pow2_nodes(e, edge) for e in ext)
    return dict(name="copper_blocks_%d" % seed, xyz=xyz, tri=tri, formulation="efie", eps_out=1.0, eps_in=None,
                sigma=5.8e7, grid_n=grid, order=2, radius=3, precision="f32")


def _pow2_nodes(extent, h, order=2):
    m = (order + 1) // 2
    need = int(np.ceil(extent / h)) + 1 + 2 * m
    n = 8
    while n < need and n < 64:
        n *= 2
    return n


def uneven_batch(n=48, seed=0, nrhs=4):
    """Members of an uneven batch of meshes (list of workload dicts)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = ("sphere", "box", "torus")[int(rng.integers(3))]
        dielectric = bool(rng.integers(2))
        eps = float(rng.uniform(2.0, 6.0)) if dielectric else None
        size = float(rng.uniform(0.5, 4.0))             # free-space wavelengths (1 m)
        target = float(np.exp(rng.uniform(np.log(2000.0), np.log(60000.0))))
        edges = target / (2 if dielectric else 1)
        if kind == "sphere":
            level = int(np.clip(np.round(np.log(edges / 30.0) / np.log(4.0)), 2, 5))
            xyz, tri = icosphere(level, radius=0.5 * size)
        elif kind == "box":
            d = max(2, int(np.round(np.sqrt(edges / 18.0))))
            a = 0.5 * size / np.sqrt(3.0)
            xyz, tri = box([-a, -a, -a], [a, a, a], [d, d, d])
        else:
            nm = max(4, int(np.round(np.sqrt(edges / 6.0))))
            xyz, tri = torus(0.35 * size, 0.15 * size, 2 * nm, nm)
        lam_in = 1.0 / np.sqrt(eps) if dielectric else 1.0
        ext = xyz.max(0) - xyz.min(0)
        t = xyz[tri]
        edge = np.mean(np.linalg.norm(t - np.roll(t, 1, axis=1), axis=2))
        h = min(0.1 * lam_in, edge)       # resolve the wavelength and the mesh
        grid = tuple(_pow2_nodes(e, h) for e in ext)
        out.append(dict(name="%s_%s_%d" % (kind, "diel" if dielectric else "pec", i), xyz=xyz, tri=tri,
                        formulation="pmchwt" if dielectric else "efie", eps_out=1.0, eps_in=eps,
                        grid_n=grid, order=2, radius=3, freq=C0, nrhs=nrhs, precision="f32"))
    return out


WORKLOADS = {"pec_sphere_1920": pec_sphere_1920, "dielectric_sphere_61440": dielectric_sphere_61440}

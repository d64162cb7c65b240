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
"""

from .meshes import icosphere

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


WORKLOADS = {"pec_sphere_1920": pec_sphere_1920, "dielectric_sphere_61440": dielectric_sphere_61440}

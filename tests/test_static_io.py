"""Static-data files (aimx_save_static / aimx_load_static).

CPU tests: malformed files are rejected with AIMX_E_IO on the host, before any
device work (missing file, wrong magic, truncation, checksum mismatch).  GPU
test: a saved and reloaded context reproduces the setup products and both
products bit for bit.
"""

import ctypes
import struct

import numpy as np
import pytest

E_IO = -8


def _lib():
    from paper_2009_02281_gb300 import aimx, build
    if not __import__("os").path.exists(build.LIB):
        build.build()
    return aimx.load()


def _load_rc(path):
    lib = _lib()
    out = ctypes.c_void_p()
    return lib.aimx_load_static(str(path).encode(), ctypes.byref(out)), out


def _fnv(data):
    h = 1469598103934665603
    for c in data:
        h ^= c
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _tiny_file(good_sum=True):
    """A well-formed header for a one-triangle 'mesh' with consistent array sizes."""
    nv, nt, form, order, n, radius, N, nnz = 3, 1, 0, 1, (4, 4, 4), 3, 1, 1
    body = struct.pack("<8i", 1, nv, nt, form, order, *n) + struct.pack("<ii", radius, N) + struct.pack("<q", nnz)
    body += struct.pack("<5d", 1.0, 1.0, 1.0, 1.0, 0.0) + struct.pack("<6d", 1, 1, 1, 0, 0, 0)
    U = (order + 1) ** 3
    body += np.zeros(3 * nv).tobytes() + np.array([0, 1, 2], dtype=np.int32).tobytes()
    body += np.zeros(N * U * 4).tobytes() + np.zeros(3 * nnz).tobytes() + np.zeros(3 * N).tobytes()
    s = _fnv(body) if good_sum else _fnv(body) ^ 1
    return b"AIMXSTAT" + body + struct.pack("<Q", s)


def test_missing_file(tmp_path):
    rc, _ = _load_rc(tmp_path / "none.bin")
    assert rc == E_IO


def test_wrong_magic(tmp_path):
    p = tmp_path / "bad.bin"
    p.write_bytes(b"NOTAIMX!" + bytes(100))
    assert _load_rc(p)[0] == E_IO


def test_truncated(tmp_path):
    p = tmp_path / "trunc.bin"
    p.write_bytes(_tiny_file()[:60])
    assert _load_rc(p)[0] == E_IO


def test_checksum_mismatch(tmp_path):
    p = tmp_path / "sum.bin"
    p.write_bytes(_tiny_file(good_sum=False))
    assert _load_rc(p)[0] == E_IO


@pytest.mark.gpu
def test_save_load_roundtrip(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from synth import icosphere, random_complex
    from paper_2009_02281_gb300 import Context, PMCHWT, AimxError
    xyz, tri = icosphere(2)
    a = Context(xyz, tri, (16, 16, 16), order=2, formulation=PMCHWT, eps_out=1.0, eps_in=4.0)
    path = tmp_path / "sphere.aimx"
    a.save_static(path)
    b = Context.load_static(path)
    for k in ("n_basis", "n_unknowns", "near_nnz", "grid_n", "pad", "grid_h", "grid_origin", "order", "formulation"):
        assert a.info[k] == b.info[k], k
    ea, eb = a.export_setup(), b.export_setup()
    for k in ea:
        assert np.array_equal(ea[k], eb[k]), k
    f = 2.1e8
    x = random_complex((3, a.nunk), seed=5)
    for dt in (torch.complex64, torch.complex128):
        xt = torch.tensor(x, dtype=dt, device="cuda")
        ya = a.matvec(f, xt).cpu().numpy()
        yb = b.matvec(f, xt).cpu().numpy()
        assert np.array_equal(ya, yb)
    # a flipped byte in the stored arrays is caught by the checksum
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 0x40
    bad = tmp_path / "flipped.aimx"
    bad.write_bytes(bytes(raw))
    with pytest.raises(AimxError) as ei:
        Context.load_static(bad)
    assert ei.value.code == E_IO
    a.close()
    b.close()

"""The C-ABI library builds, loads and exports every symbol include/*.h
declares (no compute call: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(qmc_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for required in ("qmc_system_load", "qmc_walkers_eval", "qmc_logpsi_backward"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1209_6630_gb300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_error_path_without_gpu_call():
    from paper_1209_6630_gb300._lib import lib
    L = lib()
    # invalid arguments are rejected on the host before any device work
    rc = L.qmc_det_inverse(1, 0, None, None, None, None, None, None)
    assert rc == -1
    assert b"1 <= n <= 1024" in L.qmc_last_error()
    rc = L.qmc_system_load(None, 0, None)
    assert rc == -1


def test_oracle_and_library_share_no_code():
    import oracle
    for p in glob.glob(os.path.join(ROOT, "paper_1209_6630_gb300", "**", "*.py"), recursive=True):
        assert "import oracle" not in open(p).read() and "from oracle" not in open(p).read(), p
    osrc = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_1209_6630_gb300" not in osrc


def _header_enums():
    vals = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(QMC_[A-Z0-9_]+)\s*=\s*(-?\d+)u?\b", src):
            vals[m.group(1)] = int(m.group(2))
    return vals


def test_binding_constants_match_header_enums():
    from paper_1209_6630_gb300 import _lib as L
    e = _header_enums()
    assert {k: e["QMC_PREC_" + k.upper()] for k in L.PREC} == L.PREC
    assert {k: e["QMC_A4_" + k.upper()] for k in L.A4_MODE} == L.A4_MODE
    assert {k: e["QMC_C15_" + k.upper()] for k in L.C15_MODE} == L.C15_MODE
    assert {k: e["QMC_EXPIRE_" + k.upper()] for k in L.EXPIRE} == L.EXPIRE
    assert (L.STATUS_SINGULAR_UP, L.STATUS_SINGULAR_DN, L.STATUS_NONFINITE, L.STATUS_TIMEOUT) == (
        e["QMC_STATUS_SINGULAR_UP"], e["QMC_STATUS_SINGULAR_DN"], e["QMC_STATUS_NONFINITE"], e["QMC_STATUS_TIMEOUT"])
    assert (L.DTYPE_F64, L.DTYPE_F32) == (e["QMC_DTYPE_F64"], e["QMC_DTYPE_F32"])
    assert (L.QMC_OK, L.QMC_ERR_INVALID, L.QMC_ERR_CUDA, L.QMC_ERR_TIMEOUT, L.QMC_ERR_CAPACITY, L.QMC_ERR_NOMEM) == (
        e["QMC_OK"], e["QMC_ERR_INVALID"], e["QMC_ERR_CUDA"], e["QMC_ERR_TIMEOUT"], e["QMC_ERR_CAPACITY"],
        e["QMC_ERR_NOMEM"])


def test_crc32_key_checked_at_load():
    """Sec. V.C (error checking): the CRC-32 key of the critical data.  The
    binding computes it with zlib; the library recomputes it with its own
    table-driven CRC before any device call, so a corrupted byte is caught on
    the host (QMC_ERR_INVALID) and an intact description passes the check
    (then QMC_OK on a GPU, QMC_ERR_CUDA without one)."""
    import ctypes as C
    import zlib

    import numpy as np

    from paper_1209_6630_gb300._lib import lib
    from paper_1209_6630_gb300.api import desc_crc32, system_desc
    from synth import tiny_system

    L = lib()
    s = tiny_system("mini_chain")
    d, keep, _ = system_desc(s)
    # the key is zlib's CRC-32 of the arrays' bytes in declaration order, then eps
    blob = b"".join(a.tobytes() for a in keep) + np.array([s.eps]).tobytes()
    assert d.crc32 == zlib.crc32(blob) & 0xFFFFFFFF
    h = C.c_void_p()
    rc = L.qmc_system_load(C.byref(d), 0, C.byref(h))
    assert rc in (0, -2), L.qmc_last_error()         # passed the CRC check
    if rc == 0:
        L.qmc_system_free(h)
    # one flipped bit in an MO coefficient: rejected on the host, nothing loaded
    keep[11].view(np.uint8)[5] ^= 0x10
    rc = L.qmc_system_load(C.byref(d), 0, C.byref(h))
    assert rc == -1
    msg = L.qmc_last_error().decode()
    assert "CRC-32" in msg
    got = int(msg.split("description is ")[1].split(",")[0], 16)
    assert got == desc_crc32(keep, d.eps) != d.crc32      # the library's CRC = zlib's on the corrupted bytes
    # a wrong key with intact data is rejected the same way
    keep[11].view(np.uint8)[5] ^= 0x10
    d.crc32 ^= 1
    assert L.qmc_system_load(C.byref(d), 0, C.byref(h)) == -1

"""The C-ABI library builds, loads and exports every symbol its header declares.

CPU-only: argument validation is exercised (it runs before any CUDA call);
nothing here launches a kernel.
"""
import os
import re

import numpy as np
import pytest

from paper_1809_04352_gb300 import build as libbuild
from paper_1809_04352_gb300 import eses

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return eses.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "eses.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eses_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(eses.SYMBOLS) == names


def test_binding_names_match_abi():
    for n in _declared():
        assert callable(getattr(eses, n)), n


@pytest.mark.parametrize("bad", [
    dict(n=0), dict(r=-1.0), dict(r=0.0), dict(nan=True), dict(rp=-0.1), dict(rp=0.0), dict(h=0.0), dict(margin=0.1),
    dict(inf_rp=True),
])
def test_invalid_arguments_rejected(lib, bad):
    xyz = np.zeros((3, 3))
    xyz[1, 0] = 2.0
    xyz[2, 1] = 2.0
    r = np.full(3, 1.5)
    rp, h, margin = 1.4, 0.5, 1.0
    if "n" in bad:
        xyz, r = xyz[:0], r[:0]
    if "r" in bad:
        r[1] = bad["r"]
    if "nan" in bad:
        xyz[2, 2] = np.nan
    if "rp" in bad:
        rp = bad["rp"]
    if "inf_rp" in bad:
        rp = float("inf")
    if "h" in bad:
        h = bad["h"]
    if "margin" in bad:
        margin = bad["margin"]
    with pytest.raises(eses.EsesError) as ei:
        eses.eses_create(xyz, r, rp, h, margin)
    assert ei.value.code == eses.ESES_EINVAL
    assert eses.eses_last_error(None)


def test_null_context_calls_fail_cleanly(lib):
    import ctypes
    assert lib.eses_run(None) == eses.ESES_EINVAL
    assert lib.eses_set_option(None, 1, 64) == eses.ESES_EINVAL
    lib.eses_destroy(None)
    assert lib.eses_stats(None, None, 0) == eses.ESES_EINVAL
    assert isinstance(lib.eses_last_error(ctypes.c_void_p()), bytes)


def test_destroy_frees_every_device_buffer():
    """Every device buffer the context declares is released by eses_destroy
    (a source check: a buffer added without its release leaks device memory)."""
    src = open(os.path.join(ROOT, "paper_1809_04352_gb300", "csrc", "eses_api.cu")).read()
    names = []
    for decl in re.findall(r"^\s*DBuf ([A-Za-z0-9_\[\], ]+);", src, flags=re.M):
        names += [n.strip() for n in decl.split(",")]
    assert len(names) > 60
    body = src[src.index("void eses_destroy(eses_ctx *c)"):]
    body = body[:body.index("\n}\n")]
    for n in names:
        if n.endswith("[3]"):
            assert f"free_buf(c->{n[:-3]}[a])" in body, n
        else:
            assert f"&c->{n}" in body, n


def test_noalloc_rejects_tile_counts_that_wrap_32_bits(lib):
    """eses_crossing_edges_noalloc checks its size limit in 64 bits: an axis of
    8 * (2^32 + 1) points has 2^32 + 1 tiles, which a 32-bit tile count would
    wrap to 1 and let through.  The size check runs before any CUDA call, so
    placeholder pointers never reach the device."""
    import ctypes
    fake = ctypes.c_void_p(16)
    cap = np.zeros(3, np.int64)
    counts = np.zeros(3, np.int64)
    for dims in ([8 * (2 ** 32 + 1), 1, 1], [1, 8 * 2 ** 32, 1], [1, 1, 8 * (2 ** 31) + 8], [2 ** 62, 2, 2],
                 [512, 512, 264]):
        d = np.asarray(dims, np.int64)
        rc = lib.eses_crossing_edges_noalloc(fake, d.ctypes.data, fake, fake, fake, cap.ctypes.data,
                                             counts.ctypes.data, None)
        assert rc == eses.ESES_EINVAL, dims

"""The C-ABI library loads on a machine without a GPU and exports every entry
point its header declares; host-only argument checks behave (no GPU work)."""
import ctypes
import os
import re

import pytest

from paper_1107_5463_gb300 import build as lib_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]

_DECL = re.compile(r"^\s*(?:int|void|const\s+char\s*\*)\s*\**\s*(sl_\w+)\s*\(", re.M)


def declared():
    names = []
    for h in HEADERS:
        names += _DECL.findall(open(h).read())
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(lib_build.build())


def test_header_declares_the_boundary():
    names = declared()
    for required in ("sl_create", "sl_sweep", "sl_sweep_series", "sl_measure",
                     "sl_required_bytes", "sl_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_required_bytes_host_logic(lib):
    from paper_1107_5463_gb300 import spinmc
    nb = spinmc.sl_required_bytes(2, 16384, 1, spinmc.SL_J_UNIFORM, spinmc.SL_STORE_I8)
    assert nb >= 2 * 16384 * 16384  # spins + natural-order staging
    nb_bonds = spinmc.sl_required_bytes(3, 16, 1, spinmc.SL_J_BONDS, spinmc.SL_STORE_I8)
    nb_plain = spinmc.sl_required_bytes(3, 16, 1, spinmc.SL_J_UNIFORM, spinmc.SL_STORE_I8)
    assert nb_bonds >= nb_plain + 3 * 16**3
    for bad in ((4, 16, 1, 0, 0), (2, 15, 1, 0, 0), (2, 0, 1, 0, 0), (2, 16, 2, 0, 0),
                (2, 16, 1, 7, 0), (2, 16, 1, 0, 9)):
        with pytest.raises(spinmc.SpinMCError) as ei:
            spinmc.sl_required_bytes(*bad)
        assert ei.value.status == spinmc.SL_EINVAL
        assert str(ei.value)


def test_create_rejects_bad_geometry_before_any_device_work():
    from paper_1107_5463_gb300 import spinmc
    for d, L in ((1, 8), (2, 7)):
        with pytest.raises(spinmc.SpinMCError) as ei:
            spinmc.sl_create(d, L, 1, 0, 0, 1.0, None, 1, 0, None, 0, None)
        assert ei.value.status == spinmc.SL_EINVAL


def test_status_strings(lib):
    from paper_1107_5463_gb300 import spinmc
    for st in (0, -1, -2, -3, -4, -5):
        assert spinmc._lib.sl_strerror(st)
    buf = ctypes.create_string_buffer(4)
    n = spinmc._lib.sl_last_error(buf, 4)
    assert n >= len(buf.value)


def test_bit_storage_needs_L_multiple_of_64_and_uniform_J():
    from paper_1107_5463_gb300 import spinmc
    assert spinmc.sl_required_bytes(2, 128, 1, 0, spinmc.SL_STORE_BITS) > 0
    for bad in ((2, 96, 1, 0, spinmc.SL_STORE_BITS), (2, 128, 1, 1, spinmc.SL_STORE_BITS),
                (2, 128, 2, 0, spinmc.SL_STORE_BITS)):
        with pytest.raises(spinmc.SpinMCError):
            spinmc.sl_required_bytes(*bad)

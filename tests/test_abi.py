"""The C ABI: libdf builds for sm_103a, loads, and exports every declared symbol (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(df_[A-Za-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["df_create", "df_setup", "df_split_int8", "df_build_J", "df_build_K", "df_energy",
                     "df_destroy", "df_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2601_08077_gb300 import build
    path = build.build_library()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_pure_host_entry_points():
    """Functions that touch no device memory run without a GPU."""
    from paper_2601_08077_gb300 import build
    from oracle import df_oracle as O
    lib = ctypes.CDLL(build.build_library())
    lib.df_level_for.argtypes = [ctypes.c_double]
    lib.df_strerror.restype = ctypes.c_char_p
    for x in [1.0, 2e-6, 1.99e-6, 5e-9, 4.99e-9, 2e-11, 1.99e-11, 7e-14, 6.99e-14, 0.0]:
        assert lib.df_level_for(x) == O.level_for(x)
    for lv in range(5):
        assert lib.df_level_slices(lv) == O.slices_for_level(lv)
    assert lib.df_strerror(-5) == b"bounded device wait ran out"
    h = ctypes.c_void_p()
    assert lib.df_create(ctypes.byref(h), 0, 10, 2, 8) == -1      # rejected before any allocation
    assert lib.df_create(ctypes.byref(h), 10, 10, 2, 9) == -1


def test_crt_host_entry_points_match_the_oracle():
    from paper_2601_08077_gb300 import build
    from oracle import crt_oracle as CO
    lib = ctypes.CDLL(build.build_library())
    lib.df_crt_operand_bits.argtypes = [ctypes.c_longlong, ctypes.c_int]
    lib.df_crt_moduli_for_bits.argtypes = [ctypes.c_longlong, ctypes.c_int]
    assert [lib.df_crt_modulus(i) for i in range(CO.MAX_MODULI)] == CO.moduli(CO.MAX_MODULI)
    assert lib.df_crt_modulus(-1) == 0 and lib.df_crt_modulus(CO.MAX_MODULI) == 0
    for K in (1, 7, 64, 100, 600, 1200, 32000, 2 ** 20, 2 ** 26):
        for n in range(2, CO.MAX_MODULI + 1):
            assert lib.df_crt_operand_bits(K, n) == CO.operand_bits(K, n), (K, n)
        for bits in (23, 31, 39, 47, 52):
            assert lib.df_crt_moduli_for_bits(K, bits) == CO.moduli_for_bits(K, bits), (K, bits)
    assert lib.df_crt_operand_bits(2 ** 26 + 1, 8) == 0 and lib.df_crt_operand_bits(10, 17) == 0

"""CPU checks of the tables behind the library's table-driven exp / expm1 / log1p: every entry of
eec_tables.h against 200-bit mpmath values (double-double pairs to about 2^-100 relative), and the
Cody-Waite split of ln2/256."""
import os
import re

import mpmath
import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLES = os.path.join(ROOT, "paper_2604_03079_gb300", "csrc", "eec_tables.h")
mpmath.mp.prec = 200


def _parse():
    text = open(TABLES).read()
    arrays = {}
    for name, body in re.findall(r"(\w+)\[\d+\] = \{(.*?)\};", text, flags=re.S):
        arrays[name] = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-fp.+\-]+", body)]
    consts = {k: float.fromhex(v) for k, v in
              re.findall(r"constexpr double (\w+) = (-?0x[0-9a-fp.+\-]+);", text)}
    return arrays, consts


def test_exp_table_is_two_to_the_j_over_256():
    a, _ = _parse()
    assert len(a["kExp2Hi"]) == len(a["kExp2Lo"]) == 256
    for j in range(256):
        exact = mpmath.power(2, mpmath.mpf(j) / 256)
        assert float(exact) == a["kExp2Hi"][j]
        err = abs(mpmath.mpf(a["kExp2Hi"][j]) + mpmath.mpf(a["kExp2Lo"][j]) - exact) / exact
        assert err < mpmath.mpf(2) ** -100


def test_log_tables():
    a, _ = _parse()
    assert len(a["kF"]) == len(a["kInvF"]) == len(a["kLogFHi"]) == len(a["kLogFLo"]) == 257
    for j in range(257):
        F = 1 + mpmath.mpf(j) / 256
        assert a["kF"][j] == float(F)
        assert a["kInvF"][j] == float(1 / F)
        err = abs(mpmath.mpf(a["kLogFHi"][j]) + mpmath.mpf(a["kLogFLo"][j]) - mpmath.log(F))
        assert err < mpmath.mpf(2) ** -100


def test_reduction_constants():
    _, c = _parse()
    ln2oN = mpmath.log(2) / 256
    assert c["kLn2oNHi"] == float(ln2oN)
    assert abs(mpmath.mpf(c["kLn2oNHi"]) + mpmath.mpf(c["kLn2oNLo"]) - ln2oN) < mpmath.mpf(2) ** -110
    assert c["kInvLn2xN"] == float(256 / mpmath.log(2))


def test_bit_pattern_constants_match_their_values():
    # the comparisons on the integer pipe use these IEEE-754 patterns; each carries its value
    import re
    import struct
    src = open(os.path.join(ROOT, "paper_2604_03079_gb300", "csrc", "eec_fastmath.cuh")).read()
    found = re.findall(r"constexpr (?:unsigned )?long long (kBits\w+) = (0x[0-9A-Fa-f]+)(?:LL|ull);"
                       r"\s*// (\S+)", src)
    assert len(found) == 6
    for name, hexv, val in found:
        v = 2.0 ** int(val[2:]) if val.startswith("2^") else float(val)
        assert int(hexv, 16) == struct.unpack("<Q", struct.pack("<d", v))[0], name

"""Writes eec_tables.h: the tables of the table-driven FP64 exp / expm1 / log1p (eec_fastmath.cuh).

Values are computed with mpmath at 200-bit precision and rounded to double; double-double pairs
(hi, lo) keep the tables accurate well below one ulp. Run: python gen_tables.py (rewrites the
header beside this script).
"""
import os

import mpmath

mpmath.mp.prec = 200
HERE = os.path.dirname(os.path.abspath(__file__))


def dd(v):
    hi = float(v)
    lo = float(v - mpmath.mpf(hi))
    return hi, lo


def arr(name, vals):
    body = ",\n    ".join(", ".join(v.hex() for v in vals[i:i + 4]) for i in range(0, len(vals), 4))
    return f"static __device__ const double {name}[{len(vals)}] = {{\n    {body}}};\n"


def main():
    ln2 = mpmath.log(2)
    exp_hi, exp_lo = zip(*(dd(mpmath.power(2, mpmath.mpf(j) / 64)) for j in range(64)))
    F = [1 + mpmath.mpf(j) / 128 for j in range(129)]
    logF_hi, logF_lo = zip(*(dd(mpmath.log(f)) for f in F))
    invF = [float(1 / f) for f in F]
    Fd = [float(f) for f in F]
    l_hi, l_lo = dd(ln2 / 64)
    out = ["// Generated by gen_tables.py (mpmath, 200-bit precision); do not edit.",
           "// 2^(j/64) for the exponential, and F_j = 1 + j/128, 1/F_j, log(F_j) for the",
           "// logarithm, as used by the table-driven functions in eec_fastmath.cuh.",
           "#pragma once", "",
           f"constexpr double kInvLn2x64 = {float(64 / ln2).hex()};   // 64 / ln 2",
           f"constexpr double kLn2o64Hi = {l_hi.hex()};   // ln2/64, leading part",
           f"constexpr double kLn2o64Lo = {l_lo.hex()};   // ln2/64 - kLn2o64Hi", "",
           arr("kExp2Hi", list(exp_hi)), arr("kExp2Lo", list(exp_lo)),
           arr("kLogFHi", list(logF_hi)), arr("kLogFLo", list(logF_lo)),
           arr("kInvF", invF), arr("kF", Fd)]
    with open(os.path.join(HERE, "eec_tables.h"), "w") as fh:
        fh.write("\n".join(out))


if __name__ == "__main__":
    main()

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


NEXP = 256   # 2^(j/NEXP): exp and expm1 reduce to |r| <= ln2 / (2 NEXP)
NLOG = 256   # F_j = 1 + j/NLOG, j = 0..NLOG: log1p reduces to |u| <= 1 / (2 NLOG)


def main():
    ln2 = mpmath.log(2)
    exp_hi, exp_lo = zip(*(dd(mpmath.power(2, mpmath.mpf(j) / NEXP)) for j in range(NEXP)))
    F = [1 + mpmath.mpf(j) / NLOG for j in range(NLOG + 1)]
    logF_hi, logF_lo = zip(*(dd(mpmath.log(f)) for f in F))
    invF = [float(1 / f) for f in F]
    Fd = [float(f) for f in F]
    l_hi, l_lo = dd(ln2 / NEXP)
    out = ["// Generated by gen_tables.py (mpmath, 200-bit precision); do not edit.",
           f"// 2^(j/{NEXP}) for the exponential, and F_j = 1 + j/{NLOG}, 1/F_j, log(F_j) for the",
           "// logarithm, as used by the table-driven functions in eec_fastmath.cuh.",
           "#pragma once", "",
           f"constexpr int kExpN = {NEXP};   // entries of kExp2Hi / kExp2Lo",
           f"constexpr int kLogN = {NLOG};   // kF etc. hold kLogN + 1 entries",
           f"constexpr double kInvLn2xN = {float(NEXP / ln2).hex()};   // {NEXP} / ln 2",
           f"constexpr double kLn2oNHi = {l_hi.hex()};   // ln2/{NEXP}, leading part",
           f"constexpr double kLn2oNLo = {l_lo.hex()};   // ln2/{NEXP} - kLn2oNHi", "",
           arr("kExp2Hi", list(exp_hi)), arr("kExp2Lo", list(exp_lo)),
           arr("kLogFHi", list(logF_hi)), arr("kLogFLo", list(logF_lo)),
           arr("kInvF", invF), arr("kF", Fd)]
    with open(os.path.join(HERE, "eec_tables.h"), "w") as fh:
        fh.write("\n".join(out))


if __name__ == "__main__":
    main()

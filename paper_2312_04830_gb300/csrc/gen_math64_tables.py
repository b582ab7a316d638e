"""Writes math64_tables.h: the constant tables of the library's FP64 exp and
log (pr_math64.cuh), from 50-digit arithmetic (mpmath).

    python paper_2312_04830_gb300/csrc/gen_math64_tables.py

exp: 2^(j/64), j = 0..63, as a double-double (hi = the nearest double, lo =
the nearest double to the rest).  log: for F_j = 1 + j/128, j = 0..128, the
nearest double to 1/F_j and ln F_j as a double-double.  Also ln 2 / 64 and
ln 2 as double-doubles.
"""
import os

import mpmath

mpmath.mp.dps = 50
HERE = os.path.dirname(os.path.abspath(__file__))


def dd(v):
    hi = float(v)
    lo = float(v - mpmath.mpf(hi))
    return hi, lo


def main():
    lines = ["// Generated by gen_math64_tables.py (50-digit arithmetic); do not edit.",
             "#pragma once", ""]
    e = [dd(mpmath.power(2, mpmath.mpf(j) / 64)) for j in range(64)]
    lines.append("// 2^(j/64) = kExp2Hi[j] + kExp2Lo[j]")
    lines.append("__device__ const double kExp2Hi[64] = {" + ", ".join(repr(a) for a, _ in e) + "};")
    lines.append("__device__ const double kExp2Lo[64] = {" + ", ".join(repr(b) for _, b in e) + "};")
    inv = [float(1 / (1 + mpmath.mpf(j) / 128)) for j in range(129)]
    lg = [dd(mpmath.log(1 + mpmath.mpf(j) / 128)) for j in range(129)]
    lines.append("// F_j = 1 + j/128: 1/F_j rounded, and ln F_j = kLogFHi[j] + kLogFLo[j]")
    lines.append("__device__ const double kInvF[129] = {" + ", ".join(repr(a) for a in inv) + "};")
    lines.append("__device__ const double kLogFHi[129] = {" + ", ".join(repr(a) for a, _ in lg) + "};")
    lines.append("__device__ const double kLogFLo[129] = {" + ", ".join(repr(b) for _, b in lg) + "};")
    l64 = dd(mpmath.log(2) / 64)
    l2 = dd(mpmath.log(2))
    lines.append("constexpr double kLn2Over64Hi = %r, kLn2Over64Lo = %r;" % l64)
    lines.append("constexpr double kLn2Hi = %r, kLn2Lo = %r;" % l2)
    lines.append("constexpr double k64OverLn2 = %r;" % float(64 / mpmath.log(2)))
    with open(os.path.join(HERE, "math64_tables.h"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

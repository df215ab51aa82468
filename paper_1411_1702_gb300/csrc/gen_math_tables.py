"""Writes pf_mathtab.h: the tables of the table-driven logarithm and sine /
cosine of pf_math.cuh, each entry the double nearest the exact value
(computed with mpmath at 60 digits).

    python paper_1411_1702_gb300/csrc/gen_math_tables.py     # rewrites pf_mathtab.h

  kPfLogInvF[j] = 1 / F_j,  F_j = 1 + j/128, j = 0..128
  kPfLogF[j] = log F_j,  kPfLogF[129 + j] = log(F_j / 2)
  kPfSinPi64[j] = sin(pi j / 64),  kPfCosPi64[j] = cos(pi j / 64),  j = 0..128
"""
from __future__ import annotations

import os

import mpmath

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "pf_mathtab.h")
N_LOG = 128
N_TRIG = 64


def nearest(v) -> float:
    # the 60-digit value rounded to 53 bits: the nearest double unless the
    # exact value lies within 1e-60 (relative) of a midpoint between doubles
    with mpmath.workprec(53):
        return float(mpmath.mpf(v))


def table(name, vals):
    rows = []
    for i in range(0, len(vals), 3):
        rows.append("    " + ", ".join(float.hex(v) for v in vals[i:i + 3]) + ",")
    return f"PF_TABLE double {name}[{len(vals)}] = {{\n" + "\n".join(rows) + "\n};\n"


def main():
    mpmath.mp.dps = 60
    inv_f = [nearest(1 / (1 + mpmath.mpf(j) / N_LOG)) for j in range(N_LOG + 1)]
    log_f = [nearest(mpmath.log(1 + mpmath.mpf(j) / N_LOG)) for j in range(N_LOG + 1)]
    # log(F_j / 2) for x in [1/2, 1), where e log 2 + log F_j would cancel
    log_f += [nearest(mpmath.log((1 + mpmath.mpf(j) / N_LOG) / 2)) for j in range(N_LOG + 1)]
    sin_t = [nearest(mpmath.sin(mpmath.pi * j / N_TRIG)) for j in range(2 * N_TRIG + 1)]
    cos_t = [nearest(mpmath.cos(mpmath.pi * j / N_TRIG)) for j in range(2 * N_TRIG + 1)]
    # exact zeros where the exact value is zero
    for j in (0, N_TRIG, 2 * N_TRIG):
        sin_t[j] = 0.0
    for j in (N_TRIG // 2, 3 * N_TRIG // 2):
        cos_t[j] = 0.0
    text = (
        "// pf_mathtab.h -- tables of pf_math.cuh, written by gen_math_tables.py (do not edit):\n"
        "// each entry is the double nearest the exact value.\n"
        "#pragma once\n\n"
        "#ifdef __CUDACC__\n#define PF_TABLE __device__ const\n#else\n#define PF_TABLE static const\n#endif\n\n"
        "// 1 / F_j, and log F_j then log(F_j / 2), F_j = 1 + j/128\n"
        + table("kPfLogInvF", inv_f) + "\n" + table("kPfLogF", log_f) + "\n"
        "// sin(pi j/64) and cos(pi j/64)\n"
        + table("kPfSinPi64", sin_t) + "\n" + table("kPfCosPi64", cos_t)
    )
    with open(OUT, "w") as f:
        f.write(text)
    print(OUT)


if __name__ == "__main__":
    main()

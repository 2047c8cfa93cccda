"""Writes fastmath_tables.cuh: the tables and split constants of the table-driven exp and log
(fastmath.cuh), evaluated with mpmath at 60 digits.

    python paper_0908_2654_gb300/csrc/gen_fastmath_tables.py
"""
import os

import mpmath as mp

mp.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))
LOG_J0, LOG_J1 = 96, 192          # F = j/128 covers the reduced mantissa range [0.75, 1.5)


def split(v, keep_bits):
    """v = hi + lo with hi holding keep_bits significant bits (so small integer multiples of hi
    are exact) and lo = the double nearest v - hi."""
    e = int(mp.floor(mp.log(abs(v), 2)))
    q = mp.mpf(2) ** (e - keep_bits + 1)
    hi = mp.nint(v / q) * q
    return float(hi), float(v - hi)


def row(vals, per=4):
    out = []
    for i in range(0, len(vals), per):
        out.append("    " + " ".join(f"{v!r}," for v in vals[i:i + per]))
    return "\n".join(out)


def render():
    """The text of fastmath_tables.cuh."""
    ln2 = mp.log(2)
    exp_t = [float(mp.power(2, mp.mpf(j) / 64)) for j in range(64)]
    log_hi, log_lo, log_inv = [], [], []
    for j in range(LOG_J0, LOG_J1 + 1):
        F = mp.mpf(j) / 128
        v = mp.log(F)
        hi = float(v)
        log_hi.append(hi)
        log_lo.append(float(v - mp.mpf(hi)))
        log_inv.append(float(1 / F))
    ln2_64_hi, ln2_64_lo = split(ln2 / 64, 29)
    ln2_hi, ln2_lo = split(ln2, 29)
    n = LOG_J1 - LOG_J0 + 1
    src = f"""// Tables for the table-driven exp and log of fastmath.cuh, written by gen_fastmath_tables.py
// (mpmath, 60 digits, each entry rounded to the nearest double):
//   kExpTable[j] = 2^(j/64), j = 0..63
//   kLogHi[i] + kLogLo[i] = ln F, kLogInv[i] = 1/F, F = (i + {LOG_J0})/128, i = 0..{n - 1}
// The split constants hold 29 significant bits in their high parts, so integer multiples below
// 2^24 of them are exact.
#pragma once
constexpr int kLogJ0 = {LOG_J0};
__device__ const double kExpTable[64] = {{
{row(exp_t)}
}};
__device__ const double kLogHi[{n}] = {{
{row(log_hi)}
}};
__device__ const double kLogLo[{n}] = {{
{row(log_lo)}
}};
__device__ const double kLogInv[{n}] = {{
{row(log_inv)}
}};
constexpr double kInvLn2x64 = {float(64 / ln2)!r};
constexpr double kLn2By64Hi = {ln2_64_hi!r};
constexpr double kLn2By64Lo = {ln2_64_lo!r};
constexpr double kLn2Hi = {ln2_hi!r};
constexpr double kLn2Lo = {ln2_lo!r};
"""
    return src


def main():
    with open(os.path.join(HERE, "fastmath_tables.cuh"), "w") as f:
        f.write(render())


if __name__ == "__main__":
    main()

"""Writes emt_logtab.h: the reduction table of the integer-pipe natural
logarithm (emt_intlog.cuh), in exact integer arithmetic.

Interval j of X in [0.75, 1.5) is [0.75 + j 2^-8, 0.75 + (j + 1) 2^-8),
j = 0..191.  Its reduction factor is I_j 2^-15, I_j the integer nearest to
2^15 / (interval centre), except I_j = 2^15 for the two intervals next to 1
(so that r = X - 1 exactly there).  The table holds I_j and
ln(2^15 / I_j) rounded to a signed multiple of 2^-116, and ln 2 likewise.
Each logarithm is 2 atanh((a - b) / (a + b)) summed in rational arithmetic
until the terms fall below 2^-200.

Run: python gen_logtab.py  (rewrites emt_logtab.h beside this file)
"""
import os
from fractions import Fraction

Q = 116


def ln_ratio(a: int, b: int) -> int:
    """round(ln(a / b) 2^Q) for positive integers a, b with |a - b| < (a + b) / 4."""
    z = Fraction(a - b, a + b)
    z2 = z * z
    term, total, k = z, Fraction(0), 0
    while abs(term) > Fraction(1, 2 ** 200):
        total += term / (2 * k + 1)
        term *= z2
        k += 1
    v = 2 * total * 2 ** Q
    return round(v)


def table():
    inv, t = [], []
    for j in range(192):
        if j in (63, 64):
            i = 1 << 15
        else:
            i = round(Fraction(1 << 15) * 256 / Fraction(2 * (192 + j) + 1, 2))
        inv.append(i)
        t.append(ln_ratio(1 << 15, i))
    # ln 2 = 2 atanh(1/3)
    ln2 = ln_ratio(2, 1)
    return inv, t, ln2


def split(v: int):
    u = v & ((1 << 128) - 1)
    return u >> 64, u & ((1 << 64) - 1)


def main():
    inv, t, ln2 = table()
    hi = [split(v)[0] for v in t]
    lo = [split(v)[1] for v in t]
    out = ["// emt_logtab.h -- written by gen_logtab.py; do not edit.",
           "// Reduction table of the integer-pipe logarithm (emt_intlog.cuh):",
           "// I_j (Q1.15) and ln(2^15 / I_j) as signed 128-bit multiples of 2^-116",
           "// (high word, low word), j = 0..191; ln 2 in the same format.",
           "#pragma once",
           "#define EMT_LOGTAB_INV { \\"]
    for k in range(0, 192, 12):
        out.append("    " + ", ".join(f"{v}u" for v in inv[k:k + 12]) + (", \\" if k + 12 < 192 else " \\"))
    out.append("}")
    for name, arr in (("HI", hi), ("LO", lo)):
        out.append(f"#define EMT_LOGTAB_{name} {{ \\")
        for k in range(0, 192, 4):
            out.append("    " + ", ".join(f"0x{v:016X}ull" for v in arr[k:k + 4]) + (", \\" if k + 4 < 192 else " \\"))
        out.append("}")
    h, l = split(ln2)
    out.append(f"#define EMT_LN2_HI 0x{h:016X}ull")
    out.append(f"#define EMT_LN2_LO 0x{l:016X}ull")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "emt_logtab.h")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")
    return path


if __name__ == "__main__":
    print(main())

"""Generate trig_table.inc: the sin/cos table and constants of the float-float step math.

    python paper_1710_03462_b300/csrc/gen_trig_table.py

Entries, for k = 0..2047 and theta_k = 2 pi k / 2048 evaluated with 60-digit mpmath:
{hi(sin), lo(sin), hi(cos), lo(cos)} where hi = nearest float, lo = nearest float to the
remainder, so hi + lo carries about 48 bits.  Constants: round(2^63 * 4/pi) for the
fixed-point reduction of x to turns, and 2 pi / 2^64 as a float pair.  Floats are
written as C hexadecimal literals, so the compiler reads them exactly.
"""
import os

import mpmath
import numpy as np

mpmath.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))
M = 2048


def split(v):
    hi = np.float32(float(v))
    lo = np.float32(float(v - mpmath.mpf(float(hi))))
    return hi, lo


def hexf(f):
    f = float(np.float32(f))
    return "0.0f" if f == 0.0 else f.hex() + "f"


def main():
    lines = []
    for k in range(M):
        th = 2 * mpmath.pi * k / M
        sh, sl = split(mpmath.sin(th))
        ch, cl = split(mpmath.cos(th))
        lines.append(f"  {{{hexf(sh)}, {hexf(sl)}, {hexf(ch)}, {hexf(cl)}}},")
    r63 = int(mpmath.nint(mpmath.mpf(2) ** 63 * 4 / mpmath.pi))
    kh, kl = split(2 * mpmath.pi / mpmath.mpf(2) ** 64)
    out = [
        "// Generated by gen_trig_table.py -- do not edit.",
        f"// {{sin hi, sin lo, cos hi, cos lo}} of 2 pi k / {M}, k = 0..{M - 1}.",
        f"#define SOAX_TRIG_TABLE_SIZE {M}",
        f"#define SOAX_FOUR_OVER_PI_2P63 0x{r63:016X}ull  // round(2^63 * 4/pi)",
        f"#define SOAX_TWO_PI_2M64_HI {hexf(kh)}  // 2 pi / 2^64 = hi + lo",
        f"#define SOAX_TWO_PI_2M64_LO {hexf(kl)}",
        "#define SOAX_TRIG_TABLE_ENTRIES \\",
    ] + [ln + " \\" for ln in lines[:-1]] + [lines[-1].rstrip(",")]
    with open(os.path.join(HERE, "trig_table.inc"), "w") as fh:
        fh.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()

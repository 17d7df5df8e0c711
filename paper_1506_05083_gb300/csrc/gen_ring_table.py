"""Writes ring_table_q62.inc: (cos, sin)(2 pi i / 1024), i = 0 .. 1023, as
signed 64-bit fixed-point numbers with 62 fractional bits, each the value
rounded to nearest from 200-bit arithmetic (mpmath): the initializer of the
device table that trig.cuh's fixed-point sin/cos reads. The library build
only includes the generated file.

Run: python paper_1506_05083_gb300/csrc/gen_ring_table.py
"""
import os

import mpmath as mp

N = 1024


def main():
    mp.mp.prec = 200
    # the initializer of a [1024][2] array of long long: the including file
    # declares the array (with the memory space it wants) around it
    lines = ["// Generated by gen_ring_table.py: (cos, sin)(2 pi i / 1024) x 2^62, rounded to",
             "// nearest; the initializer of a long long [1024][2]. Do not edit."]
    for i in range(N):
        a = 2 * mp.pi * i / N
        c = int(mp.nint(mp.cos(a) * mp.mpf(2) ** 62))
        s = int(mp.nint(mp.sin(a) * mp.mpf(2) ** 62))
        lines.append(f"    {{{c}ll, {s}ll}},")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ring_table_q62.inc")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

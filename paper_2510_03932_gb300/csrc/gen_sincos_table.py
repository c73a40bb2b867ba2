"""Write sincos_table_data.h: {sin(i pi/512), cos(i pi/512)} for i = 0..255, each the double
nearest the exact value (mpmath at 60 significant digits, then one rounding to double), the table
of the kernels' table-driven sine and cosine (sincos_table.cuh).

Usage: python gen_sincos_table.py  (needs mpmath; its output is committed)."""
import os

import mpmath

STEPS = 512  # table spacing pi/STEPS; the quadrant [0, pi/2) holds STEPS/2 entries


def rows():
    mpmath.mp.dps = 60
    out = []
    for i in range(STEPS // 2):
        a = mpmath.mpf(i) * mpmath.pi / STEPS
        out.append((float(mpmath.sin(a)), float(mpmath.cos(a))))  # mpf -> float rounds to nearest
    return out


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "sincos_table_data.h"), "w") as fh:
        fh.write("// Generated by gen_sincos_table.py: {sin(i pi/%d), cos(i pi/%d)} for i = 0..%d, each the\n"
                 "// double nearest the exact value.\n" % (STEPS, STEPS, STEPS // 2 - 1))
        fh.write("static __device__ const double2 kSinCosTable[%d] = {\n" % (STEPS // 2))
        for i, (s, c) in enumerate(rows()):
            fh.write("    {%s, %s},  // %d\n" % (s.hex(), c.hex(), i))
        fh.write("};\n")


if __name__ == "__main__":
    main()

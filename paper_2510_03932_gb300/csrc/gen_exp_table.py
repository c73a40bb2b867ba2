"""Write exp_table_data.h: 2^(j/32) for j = 0..31, each the double nearest the exact value
(mpmath at 60 significant digits, then one rounding to double), the table of the kernels'
table-driven exponential (exp_table.cuh).

Usage: python gen_exp_table.py  (needs mpmath; its output is committed)."""
import os

import mpmath

STEPS = 32  # table spacing ln 2 / STEPS


def rows():
    mpmath.mp.dps = 60
    return [float(mpmath.power(2, mpmath.mpf(j) / STEPS)) for j in range(STEPS)]  # rounds to nearest


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "exp_table_data.h"), "w") as fh:
        fh.write("// Generated by gen_exp_table.py: 2^(j/%d) for j = 0..%d, each the double nearest the exact\n"
                 "// value.\n" % (STEPS, STEPS - 1))
        fh.write("static __device__ const double kExp2Table[%d] = {\n" % STEPS)
        for j, v in enumerate(rows()):
            fh.write("    %s,  // %d\n" % (v.hex(), j))
        fh.write("};\n")


if __name__ == "__main__":
    main()

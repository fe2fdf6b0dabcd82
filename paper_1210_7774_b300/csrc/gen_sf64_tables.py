"""Write sf64_tables.h: the fixed-point constants of sf64.cuh, computed with
mpmath at 80 significant digits and rounded to nearest.

    python paper_1210_7774_b300/csrc/gen_sf64_tables.py

Tables:
  VBE_EXP2_TAB[j]  = 2^(j/64),          j = 0..63,   unsigned, scale 2^-63
  VBE_LOG_INV[i]   = 128 / (96 + i),    i = 0..96,   unsigned, scale 2^-63
  VBE_LOG_TAB[i]   = log((96 + i)/128), i = 0..96,   signed,   scale 2^-64
  VBE_LN2_HI/LO    = ln 2 as a 128-bit fraction (hi, lo words), scale 2^-128
  VBE_LN2_64TH_HI/LO = ln(2)/64 at scale 2^-112 (a 106-bit integer in two words)
"""
import os

import mpmath

mpmath.mp.dps = 80
HERE = os.path.dirname(os.path.abspath(__file__))


def rnd(x):
    return int(mpmath.nint(x))


def main():
    lines = ["// Generated by gen_sf64_tables.py (mpmath, 80 digits); do not edit.",
             "#ifndef VBE_SF64_TABLES_H", "#define VBE_SF64_TABLES_H", ""]
    exp2 = [rnd(mpmath.power(2, mpmath.mpf(j) / 64) * 2**63) for j in range(64)]
    assert all(2**63 <= v < 2**64 for v in exp2)
    inv = [rnd(mpmath.mpf(128) / (96 + i) * 2**63) for i in range(97)]
    assert all(0 < v < 2**64 for v in inv)
    logt = [rnd(mpmath.log(mpmath.mpf(96 + i) / 128) * 2**64) for i in range(97)]
    assert all(-(2**63) <= v < 2**63 for v in logt)
    ln2 = rnd(mpmath.log(2) * 2**128)
    ln2_64 = rnd(mpmath.log(2) / 64 * 2**112)

    def arr(name, typ, vals, fmt):
        out = [f"__device__ const {typ} {name}[{len(vals)}] = {{"]
        for k in range(0, len(vals), 3):
            out.append("  " + ", ".join(fmt(v) for v in vals[k:k + 3]) + ",")
        out.append("};")
        return out

    lines += arr("VBE_EXP2_TAB", "unsigned long long", exp2, lambda v: f"0x{v:016x}ull")
    lines += arr("VBE_LOG_INV", "unsigned long long", inv, lambda v: f"0x{v:016x}ull")
    lines += arr("VBE_LOG_TAB", "long long", logt,
                 lambda v: f"(long long)0x{v & (2**64 - 1):016x}ull")
    lines += [f"#define VBE_LN2_HI 0x{ln2 >> 64:016x}ull", f"#define VBE_LN2_LO 0x{ln2 & (2**64 - 1):016x}ull",
              f"#define VBE_LN2_64TH_HI 0x{ln2_64 >> 64:016x}ull",
              f"#define VBE_LN2_64TH_LO 0x{ln2_64 & (2**64 - 1):016x}ull", "", "#endif", ""]
    with open(os.path.join(HERE, "sf64_tables.h"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()

"""Writes dft_consts.cuh: cos(2 pi k / R) and sin(2 pi k / R), k < R, for the
small odd radices of the mixed-radix FFT (fft_mr.cuh), as FP32 literals of the
values computed in double precision, the angle 2 pi k / R being reduced to the
first octant in integers before sin and cos are taken."""
import math
import os

RADICES = (3, 5, 7, 9, 11, 13)


def sincos2pi(k, r):
    """sin and cos of 2 pi k / r with the argument reduced to [0, pi/4]."""
    k %= r
    # angle = pi * (2k) / r; work with numerator n over denominator d = r, angle = pi n / d
    n, d = 2 * k, r
    s_sign = c_sign = 1.0
    if n > d:                       # sin(2 pi - a) = -sin a
        n, s_sign = 2 * d - n, -1.0
    if 2 * n > d:                   # cos(pi - a) = -cos a
        n, c_sign = d - n, -1.0
    if 4 * n <= d:
        a = math.pi * n / d
        s, c = math.sin(a), math.cos(a)
    else:
        b = math.pi * (d - 2 * n) / (2 * d)
        s, c = math.cos(b), math.sin(b)
    return s_sign * s, c_sign * c


def main():
    out = ["// Generated by gen_dft_consts.py: cos and sin of 2 pi k / R, k < R, for the",
           "// odd radices of the mixed-radix FFT (fft_mr.cuh).",
           "#pragma once", "", "namespace s2g {", "", "template <int R> struct DftConst;"]
    for r in RADICES:
        cs, sn = [], []
        for k in range(r):
            s, c = sincos2pi(k, r)
            cs.append("%.9ef" % c)
            sn.append("%.9ef" % s)
        out.append("template <> struct DftConst<%d> {" % r)
        out.append("    __host__ __device__ static constexpr float c(int k)")
        out.append("    {")
        out.append("        constexpr float v[%d] = {%s};" % (r, ", ".join(cs)))
        out.append("        return v[k];")
        out.append("    }")
        out.append("    __host__ __device__ static constexpr float s(int k)")
        out.append("    {")
        out.append("        constexpr float v[%d] = {%s};" % (r, ", ".join(sn)))
        out.append("        return v[k];")
        out.append("    }")
        out.append("};")
    out += ["", "}  // namespace s2g", ""]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dft_consts.cuh")
    open(path, "w").write("\n".join(out))


if __name__ == "__main__":
    main()

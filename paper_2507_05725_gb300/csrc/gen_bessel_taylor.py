"""Generate bessel_taylor.h: piecewise Taylor expansions of J0(z) and of the regular part
Yhat0(z) = Y0(z) - (2/pi)(ln(z/2) + gamma) J0(z) on 0 <= z <= 20.

Both functions are entire (their power series converge for every z), so about each centre
c_k = 0.25 + 0.5 k (k = 0..39) the expansion in d = z - c_k, |d| <= 1/4, converges fast: the k-th
Taylor coefficient of J0 or Yhat0 is bounded by a small multiple of 1/k!, so 13 terms reach 1e-17.
Coefficients are computed with mpmath at 50 digits and rounded to the nearest double.

Usage: python gen_bessel_taylor.py > bessel_taylor.cuh   (needs mpmath; the output is committed)
"""
import mpmath as mp

mp.mp.dps = 50
NINT, WIDTH, DEG = 40, mp.mpf("0.5"), 12


def yhat0(z):
    return mp.bessely(0, z) - (2 / mp.pi) * (mp.log(z / 2) + mp.euler) * mp.besselj(0, z)


def yhat0_series(z):
    # (2/pi) sum_{k>=1} (-1)^{k+1} H_k (z^2/4)^k / (k!)^2, valid for all z (used near z = 0)
    x = z * z / 4
    s, term, H, k = mp.mpf(0), mp.mpf(1), mp.mpf(0), 0
    while True:
        k += 1
        term *= -x / (k * k)
        H += mp.mpf(1) / k
        s -= H * term
        if abs(term) * H < mp.mpf(10) ** (-45) and k > 5:
            break
    return 2 / mp.pi * s


def main():
    rows_j, rows_y = [], []
    for k in range(NINT):
        c = mp.mpf("0.25") + WIDTH * k
        cj = mp.taylor(lambda z: mp.besselj(0, z), c, DEG)
        cy = mp.taylor(yhat0_series, c, DEG)
        rows_j.append([float(v) for v in cj])
        rows_y.append([float(v) for v in cy])
    out = ["// Generated by gen_bessel_taylor.py (mpmath, 50 digits): Taylor coefficients of J0 and Yhat0 about",
           "// c_k = 0.25 + 0.5 k; device constants, included by one translation unit.",
           f"// kTaylorJ0[k][n] = J0^(n)(c_k)/n!, kTaylorYh[k][n] = Yhat0^(n)(c_k)/n!, k < {NINT}, n <= {DEG}.",
           "#pragma once", f"constexpr int kTaylorIntervals = {NINT};", f"constexpr int kTaylorDegree = {DEG};"]
    for name, rows in (("kTaylorJ0", rows_j), ("kTaylorYh", rows_y)):
        out.append(f"__device__ const double {name}[{NINT}][{DEG + 1}] = {{")
        for r in rows:
            out.append("  {" + ", ".join(repr(v) for v in r) + "},")
        out.append("};")
    print("\n".join(out))


if __name__ == "__main__":
    main()

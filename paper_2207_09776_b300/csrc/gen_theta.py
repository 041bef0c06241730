"""Generate theta_tables.h: truncated-Taylor admissible norms theta_m.

The exponential action exp(A) b is evaluated as (T_m(A/s))^s b, T_m the
degree-m Taylor polynomial.  Following the backward-error analysis of
Al-Mohy & Higham ("Computing the action of the matrix exponential, with an
application to exponential integrators", SIAM J. Sci. Comput. 33, 2011),
T_m(X) = exp(X + E) with E = h_{m+1}(X), where
    h_{m+1}(x) = log(e^{-x} T_m(x)) = sum_{k >= m+1} c_k x^k,
and ||E|| / ||X|| <= h~_{m+1}(||X||) / ||X|| with h~ the series of |c_k|.
theta_m is the largest theta with h~_{m+1}(theta) / theta <= tol.

The coefficients are built here from first principles: e^{-x} T_m(x) =
1 + sum_{k > m} g_k x^k with g_k = (-1)^{k-m} C(k-1, m) / k! (alternating
partial binomial sums), and log(1 + G) through the recurrence
k l_k = k f_k - sum_{j=1}^{k-1} j l_j f_{k-j} for l = log f.
Run: python gen_theta.py > theta_tables.h   (needs mpmath).
"""
import mpmath as mp

mp.mp.dps = 80
NTERMS = 420


def log_series_coeffs(m):
    f = [mp.mpf(0)] * (NTERMS + 1)
    f[0] = mp.mpf(1)
    for k in range(m + 1, NTERMS + 1):
        f[k] = (-1) ** (k - m) * mp.binomial(k - 1, m) / mp.factorial(k)
    lg = [mp.mpf(0)] * (NTERMS + 1)
    for k in range(1, NTERMS + 1):
        acc = k * f[k]
        for j in range(1, k):
            if lg[j] != 0 and f[k - j] != 0:
                acc -= j * lg[j] * f[k - j]
        lg[k] = acc / k
    return lg


def theta(m, tol):
    c = log_series_coeffs(m)
    absc = [abs(x) for x in c]

    def ratio(t):
        return mp.fsum(absc[k] * t ** (k - 1) for k in range(m + 1, NTERMS + 1))

    lo, hi = mp.mpf(0), mp.mpf(1)
    while ratio(hi) <= tol:
        hi *= 2
    for _ in range(200):
        mid = (lo + hi) / 2
        if ratio(mid) <= tol:
            lo = mid
        else:
            hi = mid
    # the tail beyond NTERMS must be negligible at theta
    tail = absc[NTERMS] * lo ** (NTERMS - 1)
    assert tail < tol * mp.mpf(10) ** -6, (m, tail)
    return lo


# Tolerances: the double path uses its unit roundoff 2^-53; the float path uses
# 2^-20 (~1e-6), far below its required accuracy (1e-4 relative against the
# double-precision solution) -- the float unit roundoff 2^-24 would only buy
# accuracy that the float arithmetic of the terms cannot deliver, at ~25 % more
# stencil applications.
TOL64_EXP, TOL32_EXP = 53, 20


def main():
    mmax64, mmax32 = 120, 120
    t64 = [theta(m, mp.mpf(2) ** -TOL64_EXP) for m in range(1, mmax64 + 1)]
    t32 = [theta(m, mp.mpf(2) ** -TOL32_EXP) for m in range(1, mmax32 + 1)]
    print(f"/* Generated by gen_theta.py: theta_m for tolerances 2^-{TOL64_EXP} (double) and "
          f"2^-{TOL32_EXP} (float). */")
    print("#pragma once")
    print(f"#define MSK_THETA_MMAX_F64 {mmax64}")
    print(f"#define MSK_THETA_MMAX_F32 {mmax32}")
    print("static const double msk_theta_f64[MSK_THETA_MMAX_F64] = {")
    print(",\n".join("  " + mp.nstr(t, 17, min_fixed=-100, max_fixed=100) for t in t64))
    print("};")
    print("static const double msk_theta_f32[MSK_THETA_MMAX_F32] = {")
    print(",\n".join("  " + mp.nstr(t, 17, min_fixed=-100, max_fixed=100) for t in t32))
    print("};")


if __name__ == "__main__":
    main()

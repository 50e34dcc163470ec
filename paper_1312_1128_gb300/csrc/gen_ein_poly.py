"""Coefficients of the polynomial for Ein(u) = int_0^u (1 - e^-t)/t dt on
[0, 4.5] used by the potential walk (potential.cuh, ein_cheb_coef): Ein(u) =
u p(u - 9/4), p of degree 9 interpolating Ein(u)/u at the 10 Chebyshev nodes
of [0, 4.5], from 40-digit quadrature of the definition (mpmath); the
monomial coefficients of p in t = u - 9/4 are solved in 40 digits and printed
as C++ literals.  Run: python gen_ein_poly.py > coefficients (pasted into
potential.cuh)."""
import mpmath

U, DEG = mpmath.mpf("4.5"), 9


def ein(u):
    return mpmath.quad(lambda t: (1 - mpmath.exp(-t)) / t, [0, u])


def coefficients():
    mpmath.mp.dps = 40
    h = U / 2
    nodes = [mpmath.cos(mpmath.pi * (k + mpmath.mpf(1) / 2) / (DEG + 1)) for k in range(DEG + 1)]
    ts = [h * z for z in nodes]
    fs = [ein(t + h) / (t + h) for t in ts]
    A = mpmath.matrix([[t ** k for k in range(DEG + 1)] for t in ts])
    return [c for c in mpmath.lu_solve(A, mpmath.matrix(fs))]


if __name__ == "__main__":
    for k, c in enumerate(coefficients()):
        print(f"        case {k}: return {mpmath.nstr(c, 20, min_fixed=-1, max_fixed=-1)};")

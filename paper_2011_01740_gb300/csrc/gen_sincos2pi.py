"""Coefficients of sincos2pi_poly (rhs.cuh): weighted minimax polynomials, by
the Remez exchange algorithm in 60-digit arithmetic (mpmath), for

  sin(2 pi r) = r P(u),      P of degree 6 in u = r^2, relative error,
  cos(2 pi r) = 1 + u Q(u),  Q of degree 6, absolute error,

on |r| <= 1/8 (u in [0, 1/64]).  Prints the coefficients, highest degree
first, as C hex literals, and the error bounds after rounding them to double.
Run: python gen_sincos2pi.py
"""
import mpmath as mp

mp.mp.dps = 60
TWO_PI = 2 * mp.pi
U_MAX = mp.mpf(1) / 64


def _sin_ratio(u):
    return mp.sin(TWO_PI * mp.sqrt(u)) / mp.sqrt(u) if u > 0 else TWO_PI


def _cos_ratio(u):
    return (mp.cos(TWO_PI * mp.sqrt(u)) - 1) / u if u > 0 else -TWO_PI ** 2 / 2


def remez(f, w, a, b, m, iters=40, grid=4000):
    """Degree-m polynomial minimising max |w(u) (P(u) - f(u))| on [a, b]."""
    n = m + 2
    xs = [(a + b) / 2 - (b - a) / 2 * mp.cos(mp.pi * k / (n - 1)) for k in range(n)]
    c, level = None, None
    for _ in range(iters):
        A = mp.matrix(n, n)
        rhs = mp.matrix(n, 1)
        for i, x in enumerate(xs):
            for j in range(m + 1):
                A[i, j] = x ** j
            A[i, m + 1] = (-1) ** i / w(x)
            rhs[i] = f(x)
        sol = mp.lu_solve(A, rhs)
        c = [sol[j] for j in range(m + 1)]
        level = abs(sol[m + 1])
        pts = [a + (b - a) * k / grid for k in range(grid + 1)]
        err = [w(x) * (mp.polyval(c[::-1], x) - f(x)) for x in pts]
        ext = [0] + [k for k in range(1, grid) if (err[k] - err[k - 1]) * (err[k + 1] - err[k]) <= 0] + [grid]
        alt = []
        for k in ext:
            if alt and mp.sign(alt[-1][1]) == mp.sign(err[k]):
                if abs(err[k]) > abs(alt[-1][1]):
                    alt[-1] = (pts[k], err[k])
            else:
                alt.append((pts[k], err[k]))
        while len(alt) > n:
            alt.pop(0 if abs(alt[0][1]) < abs(alt[-1][1]) else -1)
        if len(alt) < n:
            break
        xs = [x for x, _ in alt]
        if abs(max(abs(e) for _, e in alt) - level) < level * mp.mpf("1e-6"):
            break
    return c


def main():
    a, b = mp.mpf(0), U_MAX
    check = [b * k / 4000 for k in range(4001)]
    p = remez(_sin_ratio, lambda u: 1 / _sin_ratio(u), a, b, 6)
    pd = [mp.mpf(float(x)) for x in p]
    e_sin = max(abs((mp.polyval(pd[::-1], u) - _sin_ratio(u)) / _sin_ratio(u)) for u in check)
    q = remez(_cos_ratio, lambda u: u if u > 0 else mp.mpf("1e-30"), a, b, 6)
    qd = [mp.mpf(float(x)) for x in q]
    e_cos = max(abs(u * (mp.polyval(qd[::-1], u) - _cos_ratio(u))) for u in check)
    print("P (sin), highest degree first:", ", ".join(float(x).hex() for x in reversed(p)))
    print("Q (cos), highest degree first:", ", ".join(float(x).hex() for x in reversed(q)))
    print(f"relative error of r P(r^2): {mp.nstr(e_sin, 3)}; absolute error of 1 + r^2 Q(r^2): {mp.nstr(e_cos, 3)}")


if __name__ == "__main__":
    main()

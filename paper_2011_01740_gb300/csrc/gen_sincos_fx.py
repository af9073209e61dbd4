"""Coefficients of sincos2pi_fx (sincos_fx.cuh): the Taylor series of sine
and cosine of pi w / 2 for |w| <= 1/2 (a reduced argument of at most 1/8
turn), in 64-bit fixed point (value x 2^64, rounded to nearest), for

  sin(pi w / 2) = 2 w S(w^2),      S(v) = sum_k (-1)^k S_k v^k,  k = 0..9,
  cos(pi w / 2) = 1 - 2 w^2 Q(w^2), Q(v) = sum_k (-1)^k Q_k v^k,  k = 0..8,

  S_k = (pi/2)^(2k+1) / (2k+1)! / 2,   Q_k = (pi/2)^(2k+2) / (2k+2)! / 2.

The first omitted terms are below 1.2e-22 (sine) and 3.3e-21 (cosine) at
|w| = 1/2.  Every S_k and Q_k lies in (0, 1), and each Horner partial sum
stays positive (the ratio of consecutive coefficients is at most 0.21 and
v <= 1/4), so the evaluation runs on unsigned 64-bit integers.
Prints the coefficients as C literals and the truncation bounds.
Run: python gen_sincos_fx.py
"""
import mpmath as mp

mp.mp.dps = 80
H = mp.pi / 2


def fixed(x):
    v = int(mp.nint(x * mp.mpf(2) ** 64))
    assert 0 < v < 2 ** 64
    return v


def coefficients():
    S = [H ** (2 * k + 1) / mp.factorial(2 * k + 1) / 2 for k in range(10)]
    Q = [H ** (2 * k + 2) / mp.factorial(2 * k + 2) / 2 for k in range(9)]
    return [fixed(s) for s in S], [fixed(q) for q in Q]


def main():
    S, Q = coefficients()
    print("// S_0 .. S_9")
    for k, v in enumerate(S):
        print(f"    0x{v:016x}ull,  // S_{k}")
    print("// Q_0 .. Q_8")
    for k, v in enumerate(Q):
        print(f"    0x{v:016x}ull,  // Q_{k}")
    w = mp.mpf(1) / 2
    print("sine truncation bound  ", mp.nstr((H * w) ** 21 / mp.factorial(21), 3))
    print("cosine truncation bound", mp.nstr((H * w) ** 20 / mp.factorial(20), 3))


if __name__ == "__main__":
    main()

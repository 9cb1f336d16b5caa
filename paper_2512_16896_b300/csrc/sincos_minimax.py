"""Coefficients of the sine and cosine polynomials in common.cuh (sincos_cw).

Remez exchange on |r| <= pi/4 (the range left by the Cody-Waite reduction):
  sin r = r + r^3 (s1 + s2 r^2 + s3 r^4), minimising the relative error of sin;
  cos r = 1 + r^2 (c1 + c2 r^2 + c3 r^4 + c4 r^6), minimising the absolute error.
Prints the coefficients (17 significant digits; the header stores them as
FP32 literals) and the equioscillation error of each fit. Run with
`python sincos_minimax.py` (needs mpmath, ~30 s).
"""
import mpmath as mp

mp.mp.dps = 40
R = mp.pi / 4
GRID = [R * mp.mpf(i) / 4000 for i in range(1, 4001)]


def remez(f, w, basis, iters=30):
    """Coefficients c minimising max |w(x) (f(x) - sum_k c_k basis_k(x))| on (0, R]."""
    m = len(basis)
    xs = [R * (1 - mp.cos(mp.pi * (i + 0.5) / (m + 1))) / 2 for i in range(m + 1)]
    c, worst = None, None
    for _ in range(iters):
        A = mp.matrix(m + 1, m + 1)
        b = mp.matrix(m + 1, 1)
        for i, x in enumerate(xs):
            for k in range(m):
                A[i, k] = basis[k](x) * w(x)
            A[i, m] = (-1) ** i
            b[i] = f(x) * w(x)
        sol = mp.lu_solve(A, b)
        c = [sol[k] for k in range(m)]
        err = [w(x) * (f(x) - sum(c[k] * basis[k](x) for k in range(m))) for x in GRID]
        worst = max(abs(e) for e in err)
        peaks = [i for i in range(len(GRID))
                 if (i == 0 or abs(err[i]) >= abs(err[i - 1])) and (i + 1 == len(GRID) or abs(err[i]) >= abs(err[i + 1]))]
        alt = []
        for i in peaks:  # alternating signs, the larger of equal-sign neighbours
            if alt and mp.sign(err[i]) == mp.sign(err[alt[-1]]):
                if abs(err[i]) > abs(err[alt[-1]]):
                    alt[-1] = i
            else:
                alt.append(i)
        while len(alt) > m + 1:
            alt.pop(0 if abs(err[alt[0]]) < abs(err[alt[-1]]) else -1)
        if len(alt) < m + 1:
            break
        xs = [GRID[i] for i in alt]
    return c, worst


def main():
    s, es = remez(lambda x: (mp.sin(x) - x) / x ** 3, lambda x: x ** 3 / mp.sin(x),
                  [lambda x: 1, lambda x: x ** 2, lambda x: x ** 4])
    c, ec = remez(lambda x: (mp.cos(x) - 1) / x ** 2, lambda x: x ** 2,
                  [lambda x: 1, lambda x: x ** 2, lambda x: x ** 4, lambda x: x ** 6])
    for name, v in zip(("kS1", "kS2", "kS3"), s):
        print(f"{name} = {mp.nstr(v, 17)}")
    for name, v in zip(("kC1", "kC2", "kC3", "kC4"), c):
        print(f"{name} = {mp.nstr(v, 17)}")
    print(f"sin: max relative error {mp.nstr(es, 3)}; cos: max absolute error {mp.nstr(ec, 3)}")


if __name__ == "__main__":
    main()

"""Pure-Python integer references used to pin the oracle.

These are independent of ``oracle/``: affine textbook formulas over Python
integers (instead of the oracle's Jacobian formulas in Montgomery form), the
O(N^2) DFT (instead of the radix-2 NTT), Lagrange interpolation evaluated at a
point, and SplitMix64 written from its published definition (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).
"""
from __future__ import annotations

P = 21888242871839275222246405745257275088696311157297823662689037894645226208583
R = 21888242871839275222246405745257275088548364400416034343698204186575808495617
MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


# ---------------- SplitMix64 ----------------
class SplitMix64:
    def __init__(self, seed: int, purpose: int = 0):
        self.s = (seed ^ ((purpose * GOLDEN) & MASK64)) & MASK64

    def next(self) -> int:
        self.s = (self.s + GOLDEN) & MASK64
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def fr(self) -> int:
        while True:
            w = [self.next() for _ in range(4)]
            w[3] &= (1 << 62) - 1
            v = w[0] | (w[1] << 64) | (w[2] << 128) | (w[3] << 192)
            if v < R:
                return v


# ---------------- Fp2 = Fp[u]/(u^2+1) ----------------
def f2_add(a, b):
    return ((a[0] + b[0]) % P, (a[1] + b[1]) % P)


def f2_sub(a, b):
    return ((a[0] - b[0]) % P, (a[1] - b[1]) % P)


def f2_mul(a, b):
    return ((a[0] * b[0] - a[1] * b[1]) % P, (a[0] * b[1] + a[1] * b[0]) % P)


def f2_inv(a):
    n = pow(a[0] * a[0] + a[1] * a[1], P - 2, P)
    return (a[0] * n % P, (-a[1]) * n % P)


def f2_scalar(a, k):
    return (a[0] * k % P, a[1] * k % P)


# ---------------- affine curve arithmetic ----------------
B1 = 3
B2 = f2_mul((3, 0), f2_inv((9, 1)))


def g1_on_curve(pt):
    if pt is None:
        return True
    x, y = pt
    return (y * y - x * x * x - B1) % P == 0


def g1_add(p1, p2):
    if p1 is None:
        return p2
    if p2 is None:
        return p1
    x1, y1 = p1
    x2, y2 = p2
    if x1 == x2:
        if (y1 + y2) % P == 0:
            return None
        lam = 3 * x1 * x1 * pow(2 * y1, P - 2, P) % P
    else:
        lam = (y2 - y1) * pow(x2 - x1, P - 2, P) % P
    x3 = (lam * lam - x1 - x2) % P
    return (x3, (lam * (x1 - x3) - y1) % P)


def g1_mul(pt, k):
    acc = None
    add = pt
    while k:
        if k & 1:
            acc = g1_add(acc, add)
        add = g1_add(add, add)
        k >>= 1
    return acc


def g2_on_curve(pt):
    if pt is None:
        return True
    x, y = pt
    lhs = f2_mul(y, y)
    rhs = f2_add(f2_mul(f2_mul(x, x), x), B2)
    return lhs == rhs


def g2_add(p1, p2):
    if p1 is None:
        return p2
    if p2 is None:
        return p1
    x1, y1 = p1
    x2, y2 = p2
    if x1 == x2:
        if f2_add(y1, y2) == (0, 0):
            return None
        lam = f2_mul(f2_scalar(f2_mul(x1, x1), 3), f2_inv(f2_scalar(y1, 2)))
    else:
        lam = f2_mul(f2_sub(y2, y1), f2_inv(f2_sub(x2, x1)))
    x3 = f2_sub(f2_sub(f2_mul(lam, lam), x1), x2)
    y3 = f2_sub(f2_mul(lam, f2_sub(x1, x3)), y1)
    return (x3, y3)


def g2_mul(pt, k):
    acc = None
    add = pt
    while k:
        if k & 1:
            acc = g2_add(acc, add)
        add = g2_add(add, add)
        k >>= 1
    return acc


G1 = (1, 2)
G2 = ((10857046999023057135944570762232829481370756359578518086990519993285655852781,
       11559732032986387107991004021392285783925812861821192530917403151452391805634),
      (8495653923123431417604973247489272438418190587263600148770280649306958101930,
       4082367875863433681332203403145435568316851327593401208105741076214120093531))


# ---------------- transforms ----------------
def dft(values, omega):
    """O(N^2) evaluation: out_i = sum_j v_j omega^{ij}."""
    n = len(values)
    return [sum(v * pow(omega, i * j, R) for j, v in enumerate(values)) % R for i in range(n)]


def lagrange_eval(evals, rho, omega):
    """Value at rho of the polynomial of degree < N taking evals[i] at omega^i,
    with L_i(rho) = (rho^N - 1) omega^i / (N (rho - omega^i))."""
    n = len(evals)
    zr = (pow(rho, n, R) - 1) % R
    ninv = pow(n, R - 2, R)
    acc = 0
    wi = 1
    for v in evals:
        li = zr * wi % R * ninv % R * pow((rho - wi) % R, R - 2, R) % R
        acc = (acc + v * li) % R
        wi = wi * omega % R
    return acc


def poly_eval(coeffs, x):
    acc = 0
    for c in reversed(coeffs):
        acc = (acc * x + c) % R
    return acc


def ints_from_bytes(b: bytes, width: int = 32):
    return [int.from_bytes(b[i:i + width], "little") for i in range(0, len(b), width)]


def ints_to_bytes(vals, width: int = 32) -> bytes:
    return b"".join(int(v).to_bytes(width, "little") for v in vals)

"""Oracle quadrature and Hermite tables, in high-precision decimal arithmetic.

TEST INFRASTRUCTURE ONLY. This module belongs to the FP64 oracle: only tests,
the smoke check and the CPU-baseline leg of the benchmark may import it. The
product never does.

Everything here is derived from the paper's definitions, in Python's `decimal`
module at a working precision far above double, and rounded to float at the end:

* half-range Gauss-Hermite rule (Sec. III, the half-range quadrature equation):
  weight w(z) = exp(-z^2/2)/sqrt(2 pi) on [0, inf); nodes are the roots of the
  half-range Hermite polynomial of order Q; exact for monomials z^s, s < 2Q.
  Built from the closed-form moments of w by the Chebyshev algorithm (moments ->
  three-term recurrence), roots by Newton's method on the recurrence, weights as
  Christoffel numbers 1 / sum_l h_l(z_i)^2.
* full-range Gauss-Hermite rule (Sec. III, Eq. boltzk): weight
  exp(-y^2/2)/sqrt(2 pi) on the real line, roots of He_Q (read: the
  probabilists' Hermite polynomial, since the weight has exp(-y^2/2)).
* orthonormal half-range polynomials h_l and their monomial coefficients
  h_{l,s}, and the table Phi_{s,i} = sum_{l=s}^{N} h_{l,s} h_l(z_i) of Eq. gx
  (as a double-double pair, since Eq. gx cancels heavily at large N).
"""
from __future__ import annotations

from decimal import Decimal, localcontext

import numpy as np


def _prec_for(Q: int) -> int:
    # The Chebyshev algorithm loses roughly one digit per degree on this weight;
    # keep a wide margin so the doubles at the end are correctly rounded.
    return 80 + 5 * Q


def _pi(prec: int) -> Decimal:
    """pi by Machin's formula pi = 16 atan(1/5) - 4 atan(1/239), in decimal."""
    with localcontext() as ctx:
        ctx.prec = prec + 10

        def atan_inv(x: int) -> Decimal:
            x = Decimal(x)
            x2 = x * x
            term = 1 / x
            total = term
            k = 1
            eps = Decimal(10) ** (-(prec + 8))
            while True:
                term = term / x2
                t = term / (2 * k + 1)
                if t < eps:
                    break
                total += -t if k % 2 else t
                k += 1
            return total

        return +(16 * atan_inv(5) - 4 * atan_inv(239))


def half_range_moments(K: int, prec: int) -> list[Decimal]:
    """mu_k = int_0^inf z^k exp(-z^2/2)/sqrt(2 pi) dz, k = 0..K-1.

    Even k = 2m: half of the full-line Gaussian moment (2m-1)!!.
    Odd k = 2m+1: substitute t = z^2/2 -> 2^m m! / sqrt(2 pi).
    """
    with localcontext() as ctx:
        ctx.prec = prec
        inv_s2pi = 1 / (2 * _pi(prec)).sqrt()
        mu = []
        for k in range(K):
            if k % 2 == 0:
                m = k // 2
                dfact = 1
                for j in range(1, 2 * m, 2):
                    dfact *= j
                mu.append(Decimal(dfact) / 2)
            else:
                m = (k - 1) // 2
                f = 1
                for j in range(1, m + 1):
                    f *= j
                mu.append(Decimal(2 ** m * f) * inv_s2pi)
        return mu


def full_range_moments(K: int, prec: int) -> list[Decimal]:
    """mu_k = int_R y^k exp(-y^2/2)/sqrt(2 pi) dy: (k-1)!! for even k, 0 for odd."""
    with localcontext() as ctx:
        ctx.prec = prec
        mu = []
        for k in range(K):
            if k % 2:
                mu.append(Decimal(0))
            else:
                d = 1
                for j in range(1, k, 2):
                    d *= j
                mu.append(Decimal(d))
        return mu


def chebyshev_recurrence(mu: list[Decimal], n: int, prec: int):
    """Monic recurrence pi_{k+1} = (z - alpha_k) pi_k - beta_k pi_{k-1}, k < n.

    Chebyshev's algorithm on ordinary moments mu_0..mu_{2n-1}; beta_0 = mu_0.
    """
    assert len(mu) >= 2 * n
    with localcontext() as ctx:
        ctx.prec = prec
        alpha = [Decimal(0)] * n
        beta = [Decimal(0)] * n
        sig_prev = [Decimal(0)] * (2 * n)          # sigma_{k-2, l}
        sig = [mu[l] for l in range(2 * n)]         # sigma_{k-1, l}, k = 1
        alpha[0] = mu[1] / mu[0]
        beta[0] = mu[0]
        for k in range(1, n):
            sig_new = [Decimal(0)] * (2 * n)
            for l in range(k, 2 * n - k):
                sig_new[l] = sig[l + 1] - alpha[k - 1] * sig[l] - beta[k - 1] * sig_prev[l]
            alpha[k] = sig_new[k + 1] / sig_new[k] - sig[k] / sig[k - 1]
            beta[k] = sig_new[k] / sig[k - 1]
            sig_prev, sig = sig, sig_new
        return alpha, beta


def _orthonormal_values(alpha, beta, z: Decimal, L: int) -> list[Decimal]:
    """h_0(z)..h_L(z) for the orthonormal family of the recurrence."""
    h = [1 / beta[0].sqrt()]
    if L >= 1:
        h.append((z - alpha[0]) * h[0] / beta[1].sqrt())
    for k in range(1, L):
        h.append(((z - alpha[k]) * h[k] - beta[k].sqrt() * h[k - 1]) / beta[k + 1].sqrt())
    return h


def _orthonormal_coeffs(alpha, beta, L: int) -> list[list[Decimal]]:
    """Monomial coefficients c[l][s] of h_l(z) = sum_s c[l][s] z^s, l <= L."""
    c = [[Decimal(0)] * (L + 1) for _ in range(L + 1)]
    c[0][0] = 1 / beta[0].sqrt()
    if L >= 1:
        sb = beta[1].sqrt()
        c[1][1] = c[0][0] / sb
        c[1][0] = -alpha[0] * c[0][0] / sb
    for k in range(1, L):
        sb = beta[k + 1].sqrt()
        sbk = beta[k].sqrt()
        for s in range(k + 2):
            v = Decimal(0)
            if s >= 1:
                v += c[k][s - 1]
            v -= alpha[k] * c[k][s]
            v -= sbk * c[k - 1][s]
            c[k + 1][s] = v / sb
    return c


def _monic_and_derivative(alpha, beta, z: Decimal, n: int):
    p_prev, p = Decimal(0), Decimal(1)
    d_prev, d = Decimal(0), Decimal(0)
    for k in range(n):
        p_next = (z - alpha[k]) * p - beta[k] * p_prev
        d_next = p + (z - alpha[k]) * d - beta[k] * d_prev
        p_prev, p = p, p_next
        d_prev, d = d, d_next
    return p, d


def gauss_rule(alpha, beta, n: int, prec: int):
    """Nodes (ascending) and weights of the n-point Gauss rule of the recurrence.

    Start values from the symmetric tridiagonal Jacobi matrix in double
    precision, then Newton iterations on pi_n in decimal; weights are the
    Christoffel numbers 1 / sum_{l<n} h_l(z_i)^2.
    """
    a = np.array([float(x) for x in alpha[:n]])
    b = np.array([float(x) for x in beta[1:n]])
    Jm = np.diag(a) + np.diag(np.sqrt(b), 1) + np.diag(np.sqrt(b), -1)
    start = np.sort(np.linalg.eigvalsh(Jm))
    nodes, weights = [], []
    with localcontext() as ctx:
        ctx.prec = prec
        tol = Decimal(10) ** (-(prec - 10))
        for z0 in start:
            z = Decimal(repr(float(z0)))
            for _ in range(200):
                p, d = _monic_and_derivative(alpha, beta, z, n)
                dz = p / d
                z -= dz
                if abs(dz) <= tol * (1 + abs(z)):
                    break
            h = _orthonormal_values(alpha, beta, z, n - 1)
            nodes.append(z)
            weights.append(1 / sum(x * x for x in h))
    return nodes, weights


class HalfRangeRule:
    """Half-range Gauss-Hermite rule of order Q and its orthonormal polynomials.

    Attributes (decimal lists unless noted): z (Q nodes, ascending), w (weights,
    sum 1/2), alpha, beta (recurrence to index Q), coeff[l][s] = h_{l,s} for
    l <= Q.
    """

    def __init__(self, Q: int):
        self.Q = Q
        self.prec = _prec_for(Q)
        mu = half_range_moments(2 * Q + 2, self.prec)
        self.alpha, self.beta = chebyshev_recurrence(mu, Q + 1, self.prec)
        self.z, self.w = gauss_rule(self.alpha, self.beta, Q, self.prec)
        with localcontext() as ctx:
            ctx.prec = self.prec
            self.coeff = _orthonormal_coeffs(self.alpha, self.beta, Q)

    def values(self, z: Decimal, L: int) -> list[Decimal]:
        with localcontext() as ctx:
            ctx.prec = self.prec
            return _orthonormal_values(self.alpha, self.beta, z, L)

    def phi_table(self, N: int):
        """Phi[s][i] = sum_{l=s}^{N} h_{l,s} h_l(z_i) (Eq. gx) as a double-double
        pair (hi, lo) of float64 arrays: hi + lo carries ~32 digits."""
        hi = np.zeros((N + 1, self.Q))
        lo = np.zeros((N + 1, self.Q))
        with localcontext() as ctx:
            ctx.prec = self.prec
            for i, zi in enumerate(self.z):
                h = _orthonormal_values(self.alpha, self.beta, zi, N)
                for s in range(N + 1):
                    v = sum(self.coeff[l][s] * h[l] for l in range(s, N + 1))
                    hi[s, i] = float(v)
                    lo[s, i] = float(v - Decimal(hi[s, i]))
        return hi, lo


class FullRangeRule:
    """Full-range Gauss-Hermite rule of order Q (weight exp(-y^2/2)/sqrt(2 pi))."""

    def __init__(self, Q: int):
        self.Q = Q
        self.prec = _prec_for(Q)
        mu = full_range_moments(2 * Q + 2, self.prec)
        self.alpha, self.beta = chebyshev_recurrence(mu, Q + 1, self.prec)
        self.y, self.w = gauss_rule(self.alpha, self.beta, Q, self.prec)

    def he_table(self, N: int):
        """He[l][j] = He_l(y_j), probabilists' Hermite (He_{l+1} = y He_l - l He_{l-1}),
        as a double-double pair (hi, lo) of float64 arrays."""
        hi = np.zeros((N + 1, self.Q))
        lo = np.zeros((N + 1, self.Q))
        with localcontext() as ctx:
            ctx.prec = self.prec
            for j, yj in enumerate(self.y):
                hm, h = Decimal(0), Decimal(1)
                hi[0, j] = 1.0
                for l in range(N):
                    hm, h = h, yj * h - l * hm
                    hi[l + 1, j] = float(h)
                    lo[l + 1, j] = float(h - Decimal(hi[l + 1, j]))
        return hi, lo


def paper_half_range_weight(rule: HalfRangeRule) -> list[float]:
    """Half-range weights from the closed formula printed in Sec. III:

        w_i = z_i a_{Q-1}^2 / ( h_{Q-1}(z_i)^2 [ z_i + h_Q(0)^2 / sqrt(2 pi) ] ),

    with a_l = h_{l+1,l+1} / h_{l,l} (ratio of leading coefficients), orthonormal
    h_l, p0 = 1. Used only as an independent cross-check of the Christoffel
    weights.
    """
    Q = rule.Q
    with localcontext() as ctx:
        ctx.prec = rule.prec
        a = rule.coeff[Q][Q] / rule.coeff[Q - 1][Q - 1]
        hQ0 = rule.values(Decimal(0), Q)[Q]
        s2pi = (2 * _pi(rule.prec)).sqrt()
        out = []
        for zi in rule.z:
            hq1 = rule.values(zi, Q - 1)[Q - 1]
            out.append(float(zi * a * a / (hq1 * hq1 * (zi + hQ0 * hQ0 / s2pi))))
        return out


def paper_full_range_weight(rule: FullRangeRule) -> list[float]:
    """Full-range weights from Sec. III: w_j = Q! / He_{Q+1}(y_j)^2."""
    Q = rule.Q
    with localcontext() as ctx:
        ctx.prec = rule.prec
        fact = 1
        for k in range(2, Q + 1):
            fact *= k
        out = []
        for yj in rule.y:
            hm, h = Decimal(0), Decimal(1)
            for l in range(Q + 1):
                hm, h = h, yj * h - l * hm
            out.append(float(Decimal(fact) / (h * h)))
        return out


_cache: dict = {}


def tables(Qx: int, Qy: int, Nx_exp: int, Ny_exp: int) -> dict:
    """All float64 tables the oracle stepper needs, cached per orders."""
    key = (Qx, Qy, Nx_exp, Ny_exp)
    if key in _cache:
        return _cache[key]
    hr = HalfRangeRule(Qx)
    fr = FullRangeRule(Qy)
    phi_hi, phi_lo = hr.phi_table(Nx_exp)
    he_hi, he_lo = fr.he_table(Ny_exp)
    out = dict(
        zx=np.array([float(v) for v in hr.z]),
        wx=np.array([float(v) for v in hr.w]),
        yy=np.array([float(v) for v in fr.y]),
        wy=np.array([float(v) for v in fr.w]),
        Phi=phi_hi, Phi_lo=phi_lo,
        He=he_hi, He_lo=he_lo,
    )
    _cache[key] = out
    return out

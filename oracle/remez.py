"""1-BURA of t^(1-alpha) on [0,1] by the modified Remez algorithm (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

What is computed
----------------
For 0 < alpha < 1 and k >= 1 the best uniform rational approximation
r = P_k/Q_k in R(k,k) of t^(1-alpha) on [0,1] (Definition 2.1 "def-BURA",
Sec. 2.1, with beta = 1, m = k), its error E_alpha(k,k;1), its 2k+2 extreme
points, and the partial-fraction coefficients of t^{-1} r(t) (eq. (simplified),
Sec. 2.2):

    t^{-1} r(t) = sum_{j=0}^k c_j / (t - d_j),   d_0 = 0 > d_1 > ... > d_k.

How (the modified Remez method of Sec. 3.2, Algorithm 1)
---------------------------------------------------------
The best approximation is characterised by equioscillation: f - r takes the
values -E, +E, -E, ... with |E| maximal on 2k+2 ordered points of [0,1].  The
oracle alternates two sub-problems until the extrema of |f - r| are level:
* Representation: Chebyshev polynomials in s = 2t - 1 (eq. (eq1bua)),
  r(s) = sum pbar_j T_j(s) / (1 + sum_{j>=1} qbar_j T_j(s)).
* Fit on fixed points: the equations f(s_i) - r(s_i) = (-1)^i E (i = 1..l,
  l = 2k+2) are nonlinear only through E multiplying the denominator.  Freezing
  that E makes them a linear system in (pbar, qbar, new E); the level is the fixed
  point of this map, reached with Aitken-Steffensen extrapolation over three
  successive values (the acceleration Sec. 3.2 recommends), with a secant
  iteration as fallback.
* Exchange of points: between consecutive zeros of f - r each new point is the
  maximiser of |f - r|; then the global maximiser of |f - r| on [0,1] replaces
  the neighbour of the same error sign, so that the signs keep alternating.
* Stop when max_i |f - r|(t_i) - min_i |f - r|(t_i) < delta.
* Output: E = |E_n| and the points; poles are the roots of Q mapped back with
  t = (1+s)/2, and c_0 = P(0)/Q(0), c_j = P(d_j) / (d_j Q'(d_j)) (eq. (simplified);
  c_0 = E by eq. (c0,beta), Sec. 4.1).

Readings where the paper leaves a choice
----------------------------------------
* Arithmetic: mpmath with max(60, 40 + 4 |log10 eta_2|) decimal digits.  Table
  (tabLastS) shows that quad precision stops converging at k = 7..11; the extreme
  points cluster at 0 (eta_2 ~ 1e-25 for alpha = 0.9, k = 9) and the fit's matrix
  loses about 4 digits per decade of eta_2, so far more digits are used.
* Initialisation (the paper uses uniformly sampled points and a least-squares
  r_0, without detail): continuation.  At alpha = 1/2 the k = 1 problem starts
  from the points {0, 0.01, 0.3, 1} and the points for k+1 are those for k with
  two points added below eta_2 by geometric extrapolation of the three smallest
  nonzero points.  Any other alpha starts from the converged points of the same k
  at alpha -/+ 0.05 (towards 1/2).  r_0 is the exact fit on these points; it must
  alternate with E > 0 there, as the method's initialisation requires, otherwise
  the run stops with an error.
* Stopping: delta = 1e-13 E; a run that does not reach it within N = 80
  iterations raises (the extreme points are located to about 1e-15 in log t, so
  the spread floors near 1e-14 E).
* Search for zeros and maxima: the paper refines on shrinking local meshes; here
  zeros are bracketed by bisection in log t and maxima found by golden-section
  search in log t after a coarse scan.  The end points t = 0 and t = 1 are extreme
  points of the BURA error (Lemma BURA_caracter, item 3) and are never displaced by
  the insertion of the global maximiser.
* Sign convention: i = 1 is s = -1 (t = 0), so f(0) - r(0) = -E and r(0) = +E,
  matching Lemma 2.2 ("BURA_caracter") item 3 and eq. (c0,beta).
* Normalisation of the monomial form: q_k = 1, as in Tables ta:coeff1-3.
"""
from __future__ import annotations

import functools

import mpmath as mp

__all__ = ["bura", "remez_bura", "partial_fractions", "BuraResult"]


def _cheb(s, n):
    """T_0(s) .. T_n(s) by the three-term recurrence of eq. (eq1bua)."""
    T = [mp.mpf(1), s]
    for _ in range(2, n + 1):
        T.append(2 * s * T[-1] - T[-2])
    return T[: n + 1]


class _Problem:
    def __init__(self, alpha, k):
        self.g = 1 - mp.mpf(alpha)  # exponent beta - alpha with beta = 1
        self.k = k

    def f(self, t):
        return mp.mpf(0) if t <= 0 else t ** self.g

    def r(self, pbar, qbar, t):
        T = _cheb(2 * t - 1, self.k)
        return mp.fsum(a * b for a, b in zip(pbar, T)) / mp.fsum(a * b for a, b in zip(qbar, T))

    def e(self, pbar, qbar, t):
        """f - r at t (the error whose extrema are equalised)."""
        return self.f(t) - self.r(pbar, qbar, t)


def _fit_frozen_level(P, pts, E_prev):
    """The fit on fixed points with the level multiplying the denominator frozen at E_prev: a
    linear system in (pbar, qbar_1..k, E)."""
    k = P.k
    l = 2 * k + 2
    M = mp.matrix(l, l)
    rhs = mp.matrix(l, 1)
    for i in range(l):
        sgn = -1 if i % 2 == 0 else 1  # (-1)^i with the paper's i = 1..l
        T = _cheb(2 * pts[i] - 1, k)
        fi = P.f(pts[i])
        for j in range(k + 1):
            M[i, j] = T[j]
        for j in range(1, k + 1):
            M[i, k + j] = -(fi - sgn * E_prev) * T[j]
        M[i, l - 1] = sgn
        rhs[i] = fi
    x = mp.lu_solve(M, rhs)
    pbar = [x[j] for j in range(k + 1)]
    qbar = [mp.mpf(1)] + [x[k + j] for j in range(1, k + 1)]
    return pbar, qbar, x[l - 1]


def _fit(P, pts, E0, V=60):
    """The equioscillating fit on fixed points: the fixed point E = phi(E), phi(E) being the level
    the frozen-level linear system returns.  Aitken-Steffensen over three successive values; when
    that does not settle the residual g(E) = phi(E) - E within V steps, a secant iteration on g
    takes over."""
    E = E0
    eps = mp.mpf(10) ** (-(mp.mp.dps - 20))

    def phi(x):
        return _fit_frozen_level(P, pts, x)[2]

    for _ in range(V):
        E1 = phi(E)
        E2 = phi(E1)
        den = E2 - 2 * E1 + E
        En = E2 if den == 0 else E - (E1 - E) ** 2 / den
        done = abs(En - E) <= eps * abs(En)
        E = En
        if done:
            break
    g = phi(E) - E
    if abs(g) > eps * max(abs(E), mp.mpf(10) ** -30):
        a, ga = E, g
        b = E * (1 + mp.mpf(10) ** -6) if E != 0 else mp.mpf(10) ** -8
        gb = phi(b) - b
        for _ in range(4 * V):
            if gb == ga:
                break
            c = b - gb * (b - a) / (gb - ga)
            a, ga = b, gb
            b = c
            gb = phi(b) - b
            if abs(gb) <= eps * abs(b):
                break
        E = b
    return _fit_frozen_level(P, pts, E)


def _zero_between(P, pbar, qbar, a, b):
    """A zero of f - r in (a, b) where the error changes sign (bisection in log t)."""
    ea = P.e(pbar, qbar, a)
    tiny = mp.mpf(10) ** (-(mp.mp.dps - 5))
    for _ in range(500):
        if a > 0:
            m = mp.sqrt(a * b)
        else:
            m = b / 1000 if b > tiny else b / 2
        em = P.e(pbar, qbar, m)
        if (em > 0) == (ea > 0):
            a, ea = m, em
        else:
            b = m
        if a > 0 and b / a - 1 < mp.mpf(10) ** -20:
            break
    return (a + b) / 2


def _golden_max(P, pbar, qbar, a, b):
    la, lb = mp.log(a), mp.log(b)
    gr = (mp.sqrt(5) - 1) / 2
    x1, x2 = lb - gr * (lb - la), la + gr * (lb - la)
    f1 = abs(P.e(pbar, qbar, mp.exp(x1)))
    f2 = abs(P.e(pbar, qbar, mp.exp(x2)))
    while lb - la > mp.mpf(10) ** -15:
        if f1 > f2:
            lb, x2, f2 = x2, x1, f1
            x1 = lb - gr * (lb - la)
            f1 = abs(P.e(pbar, qbar, mp.exp(x1)))
        else:
            la, x1, f1 = x1, x2, f2
            x2 = la + gr * (lb - la)
            f2 = abs(P.e(pbar, qbar, mp.exp(x2)))
    return mp.exp((la + lb) / 2)


def _argmax_between(P, pbar, qbar, a, b, nscan=12):
    """argmax of |f - r| on [a, b], an interval between consecutive zeros (a may be 0, b may be 1).

    t = 0 and t = 1 are extreme points of the BURA error (Lemma BURA_caracter, item 3), so on the
    first and the last interval the point is the end point itself: a scan would otherwise pick a
    neighbour whose |f - r| equals the end value up to rounding (t = 1e-58, or 1 - 4e-16)."""
    if a == 0:
        return mp.mpf(0)
    if b == 1:
        return mp.mpf(1)
    lo = a
    cands = [lo * (b / lo) ** (mp.mpf(i) / nscan) for i in range(nscan)] + [b]
    vals = [abs(P.e(pbar, qbar, t)) for t in cands]
    i = max(range(len(cands)), key=vals.__getitem__)
    t = cands[i]
    left = cands[i - 1] if i > 0 else a
    right = cands[i + 1] if i + 1 < len(cands) else b
    return _golden_max(P, pbar, qbar, max(left, lo), min(right, b))


def _global_argmax(P, pbar, qbar, pts, nscan=400):
    """Global maximiser of |f - r| on [0,1] (scan + refine)."""
    lo_exp = mp.mp.dps - 15
    grid = sorted(set([mp.mpf(0), mp.mpf(1)] + list(pts)
                      + [mp.mpf(10) ** (-lo_exp + lo_exp * mp.mpf(i) / nscan) for i in range(nscan)]
                      + [mp.mpf(i) / 64 for i in range(1, 64)]))
    vals = [abs(P.e(pbar, qbar, t)) for t in grid]
    i = max(range(len(grid)), key=vals.__getitem__)
    t = grid[i]
    if t in pts or t == 0 or t == 1:
        return t
    # a maximiser that does not beat the current points beyond rounding is "already in the set"
    if vals[i] <= max(abs(P.e(pbar, qbar, s)) for s in pts) * (1 + mp.mpf(10) ** (-(mp.mp.dps // 2))):
        return pts[0]
    return _golden_max(P, pbar, qbar, grid[i - 1], grid[i + 1])


def remez_bura(alpha, k, pts0, dps=60, N=80, delta_rel=mp.mpf(10) ** -13):
    """The modified Remez method (Sec. 3.2) for beta = 1, m = k, from the initial points ``pts0`` (in t).

    Returns (pbar, qbar, E, pts): Chebyshev coefficients of P and Q in s = 2t-1
    (qbar_0 = 1), the signed level E (> 0 at convergence) and the 2k+2 points in t.
    """
    with mp.workdps(dps):
        P = _Problem(alpha, k)
        l = 2 * k + 2
        pts = [mp.mpf(t) for t in pts0]
        if len(pts) != l:
            raise ValueError("need 2k+2 initial points")
        # r_0: the fit on the initial points; it must alternate there with E > 0.
        pbar, qbar, E = _fit(P, pts, mp.mpf(0))
        if not E > 0:
            raise RuntimeError("inadmissible initial points for alpha=%s k=%d" % (alpha, k))
        converged = False
        for _n in range(1, N + 1):
            # zeros of the error between neighbouring points, then the maximiser between zeros
            zeros = [_zero_between(P, pbar, qbar, pts[i], pts[i + 1]) for i in range(l - 1)]
            bnd = [mp.mpf(0)] + zeros + [mp.mpf(1)]
            new = [_argmax_between(P, pbar, qbar, bnd[i], bnd[i + 1]) for i in range(l)]
            # the global maximiser replaces the neighbour of the same sign (signs keep alternating)
            ts = _global_argmax(P, pbar, qbar, new)
            # t = 0 and t = 1 are extreme points of the BURA error (Lemma BURA_caracter, item 3):
            # they stay in the set, so a maximiser that would displace them is not inserted
            if ts not in new and new[1] < ts < new[-2]:
                j = max(i for i in range(l) if new[i] < ts) if ts > new[0] else 0
                if j + 1 < l and mp.sign(P.e(pbar, qbar, ts)) != mp.sign(P.e(pbar, qbar, new[j])):
                    new[j + 1] = ts
                else:
                    new[j] = ts
            eta = [abs(P.e(pbar, qbar, t)) for t in new]
            pts = new
            # level extrema: done
            if max(eta) - min(eta) < delta_rel * abs(E):
                converged = True
                break
            # refit on the exchanged points
            pbar, qbar, E = _fit(P, pts, E)
            if not E > 0:
                raise RuntimeError("Remez lost the alternation for alpha=%s k=%d" % (alpha, k))
        if not converged:
            raise RuntimeError("Remez did not converge for alpha=%s k=%d" % (alpha, k))
        return pbar, qbar, E, pts


def _cheb_to_monomial(cb):
    """Coefficients (ascending powers of t) of sum_j cb_j T_j(2t-1)."""
    n = len(cb) - 1
    Tm = [[mp.mpf(1)], [mp.mpf(-1), mp.mpf(2)]]
    for j in range(2, n + 1):
        a, b = Tm[-1], Tm[-2]
        nxt = [mp.mpf(0)] * (j + 1)
        for i, v in enumerate(a):  # 2(2t-1) * T_{j-1}
            nxt[i] -= 2 * v
            nxt[i + 1] += 4 * v
        for i, v in enumerate(b):
            nxt[i] -= v
        Tm.append(nxt)
    out = [mp.mpf(0)] * (n + 1)
    for j, c in enumerate(cb):
        for i, v in enumerate(Tm[j]):
            out[i] += c * v
    return out


def _polyval(c, t):
    return mp.fsum(ci * t ** i for i, ci in enumerate(c))


def partial_fractions(pbar, qbar):
    """Monomial p, q (q_k = 1), poles d_0 = 0 > d_1 > ... > d_k, zeros zeta and c_j.

    eq. (simplified): t^{-1} P(t)/Q(t) = sum_j c_j / (t - d_j) with d_0 = 0;
    c_0 = P(0)/Q(0) and c_j = P(d_j) / (d_j Q'(d_j)) for the simple poles d_j.
    """
    p = _cheb_to_monomial(pbar)
    q = _cheb_to_monomial(qbar)
    lead = q[-1]
    p = [v / lead for v in p]
    q = [v / lead for v in q]
    k = len(q) - 1
    extra = mp.mp.dps
    poles = mp.polyroots(list(reversed(q)), maxsteps=400, extraprec=4 * extra)
    zeros = mp.polyroots(list(reversed(p)), maxsteps=400, extraprec=4 * extra)
    poles = sorted((mp.re(z) for z in poles), reverse=True)
    zeros = sorted((mp.re(z) for z in zeros), reverse=True)
    dq = [i * q[i] for i in range(1, k + 1)]
    c = [_polyval(p, 0) / _polyval(q, 0)]
    for d in poles:
        c.append(_polyval(p, d) / (d * _polyval(dq, d)))
    return p, q, [mp.mpf(0)] + poles, c, zeros


class BuraResult:
    """alpha, k, E, eta (extreme points), p, q (monomial, q_k = 1), d, c, zeta."""

    def __init__(self, alpha, k, E, eta, p, q, d, c, zeta, pbar, qbar):
        self.alpha, self.k, self.E, self.eta = alpha, k, E, eta
        self.p, self.q, self.d, self.c, self.zeta = p, q, d, c, zeta
        self.pbar, self.qbar = pbar, qbar

    def r(self, t):
        """r(t) = P(t)/Q(t) (multi-precision)."""
        t = mp.mpf(t)
        return _polyval(self.p, t) / _polyval(self.q, t)

    def floats(self):
        return {"alpha": float(self.alpha), "k": self.k, "E": float(self.E),
                "c": [float(v) for v in self.c], "d": [float(v) for v in self.d]}


def _extend_points(pts):
    """Continuation k -> k+1: two extra points below eta_2 (geometric extrapolation)."""
    r1 = pts[2] / pts[1]
    r2 = pts[3] / pts[2]
    n1 = pts[1] / (r1 * r1 / r2)
    n0 = n1 / (r1 ** 3 / r2 ** 2)
    return [mp.mpf(0), n0, n1] + list(pts[1:])


@functools.lru_cache(maxsize=None)
def bura(alpha, k, dps=60):
    """1-BURA data for (alpha, k), by continuation (see the module notes)."""
    alpha = round(float(alpha), 6)
    if not (0 < alpha < 1) or k < 1:
        raise ValueError("need 0 < alpha < 1 and k >= 1")
    with mp.workdps(dps):
        if alpha == 0.5:
            if k == 1:
                pts = [mp.mpf(0), mp.mpf("0.01"), mp.mpf("0.3"), mp.mpf(1)]
            else:
                pts = _extend_points(bura(0.5, k - 1, dps).eta)
        else:
            nxt = 0.5 if abs(alpha - 0.5) <= 0.05 + 1e-12 else round(alpha - (0.05 if alpha > 0.5 else -0.05), 6)
            pbar, qbar, E, pts = _continue_alpha(alpha, k, nxt, list(bura(nxt, k, dps).eta), dps)
            work = _work_dps(pts, dps)
        if alpha == 0.5:
            # k-continuation: a run that does not converge at the estimated precision is retried with
            # 40 and then 80 more digits (Table tabLastS: convergence fails for lack of digits)
            work = _work_dps(pts, dps)
            for attempt in range(3):
                try:
                    with mp.workdps(work):
                        pbar, qbar, E, pts1 = remez_bura(alpha, k, pts, dps=work)
                    pts = pts1
                    break
                except RuntimeError:
                    if attempt == 2:
                        raise
                    work += 40
        # r(0) = E holds exactly for the BURA (t = 0 is an extreme point, where the error is -r(0)); the
        # fit on the points meets it only to its working precision divided by |Q(s = -1)|, which can be as
        # small as 1e-89 of Q's coefficients.  When the computed r(0) misses E by more than 1e-25
        # relative, Algorithm 1 is rerun from the converged points with 40 more digits.
        for _ in range(4):
            with mp.workdps(work):
                if abs(_r_at_zero(pbar, qbar) - E) <= mp.mpf(10) ** -25 * abs(E):
                    break
            work += 40
            with mp.workdps(work):
                pbar, qbar, E, pts = remez_bura(alpha, k, pts, dps=work)
        with mp.workdps(work):
            p, q, d, c, zeta = partial_fractions(pbar, qbar)
            return BuraResult(alpha, k, abs(E), pts, p, q, d, c, zeta, pbar, qbar)


def _r_at_zero(pbar, qbar):
    """r(0) = P(s = -1) / Q(s = -1) from the Chebyshev coefficients (T_i(-1) = (-1)^i)."""
    num = mp.fsum(v if i % 2 == 0 else -v for i, v in enumerate(pbar))
    den = mp.fsum(v if i % 2 == 0 else -v for i, v in enumerate(qbar))
    return num / den


def _work_dps(pts, dps):
    """The fit's matrix loses about 4 digits per decade that eta_2 sits below 1 (its rows at the
    clustered points near s = -1 become nearly equal), so the working precision grows with
    -log10(eta_2) of the starting points."""
    return max(dps, int(mp.ceil(40 + 4 * (-mp.log10(pts[1])))))


def _continue_alpha(alpha, k, alpha0, pts0, dps, depth=0):
    """Algorithm 1 at alpha from the extreme points pts0 of the BURA at alpha0.  When the iteration
    from there does not converge (it can slide onto the degree-(k-1) best approximation, whose error
    cannot equioscillate on 2k+2 points), the step alpha0 -> alpha is halved, up to four times."""
    with mp.workdps(_work_dps(pts0, dps)):
        try:
            return remez_bura(alpha, k, pts0, dps=mp.mp.dps)
        except RuntimeError:
            if depth >= 4:
                raise
    mid = round((alpha + alpha0) / 2, 8)
    _, _, _, pmid = _continue_alpha(mid, k, alpha0, pts0, dps, depth + 1)
    return _continue_alpha(alpha, k, mid, list(pmid), dps, depth + 1)


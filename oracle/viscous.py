"""Viscous-correction oracle (test infrastructure): Thwaites's laminar
boundary-layer method on the inviscid surface speed of Section 2, giving the
momentum thickness, skin friction, laminar separation and the drag that the
paper's viscosity correction adds to the panel method (Section 2 names
Thwaites's method for the drag and validates it on a circular cylinder against
the method's analytic solution; the fitness of Section 3's optimisation is the
lift-to-drag ratio).  Plain numpy, one airfoil at a time; only tests/ use it
and it shares no code with the CUDA library.

The paper gives no formulas; the textbook method is restated here, and every
choice it leaves open is a reading of this library:
  * surface speed U_j = |gamma_j| / v_inf at the control points (constant-strength
    panels, the speed of Section 2's sheet);
  * stagnation point: the first j (node order) with gamma_j > 0 >= gamma_{j+1},
    placed by linear interpolation of gamma along the surface between the two
    control points (distance d_j = (L_j + L_{j+1}) / 2); the upper surface runs
    from it through control points j, j-1, .., 0 to the trailing-edge node, the
    lower through j+1, .., n-1 (j+1 left out when gamma_{j+1} = 0) to the
    trailing edge, the last half panel at the last control point's speed;
  * Thwaites's integral  theta^2 U^6 = (0.45 / Re) int_0^s U^5 ds  (lengths in
    chords, speeds in v_inf, Re = v_inf c / nu), with U linear between
    consecutive points so that each piece integrates exactly; at the
    stagnation point the limit theta^2 = 0.075 / (Re U'(0));
  * lambda = Re theta^2 dU/ds with the derivative of the quadratic through
    each point and its two neighbours (one-sided at the stagnation point and
    at the last control point), the trailing edge taking the last control
    point's lambda;
  * the Cebeci-Bradshaw fits of Thwaites's shear and shape functions l(lambda),
    H(lambda), with lambda clamped to [-0.09, 0.1];
  * laminar separation at the first control point with lambda < -0.09 (or
    U = 0); from there to the trailing edge the wall shear is zero and the
    shape factor keeps its separation value H(-0.09), while theta follows the
    same integral (an early separation, with the speed falling behind it,
    raises theta at the trailing edge);
  * skin friction cf = 2 l U / (Re theta) (per 1/2 rho v_inf^2), friction drag
    Cd_f = sum over both surfaces of the integral of cf along the freestream
    direction (trapezoid between consecutive points);
  * profile drag by Squire and Young at the trailing edge, Cd = sum over both
    surfaces of 2 theta_TE U_TE^((H_TE + 5) / 2).  It falls with the inviscid
    trailing-edge speed, which tends to zero at a blunt trailing edge: shapes
    are meant to keep a small trailing-edge angle.
"""
from __future__ import annotations

import math

import numpy as np

LAMBDA_SEP = -0.09
LAMBDA_MAX = 0.1


def shear_shape(lam):
    """Thwaites's l(lambda) and H(lambda) (Cebeci-Bradshaw fits), lambda
    clamped to [-0.09, 0.1]."""
    lam = min(max(float(lam), LAMBDA_SEP), LAMBDA_MAX)
    if lam >= 0.0:
        l = 0.22 + 1.57 * lam - 1.8 * lam * lam
        H = 2.61 - 3.75 * lam + 5.24 * lam * lam
    else:
        l = 0.22 + 1.402 * lam + 0.018 * lam / (lam + 0.107)
        H = 2.088 + 0.0731 / (lam + 0.14)
    return l, H


def squire_young(theta, U, H):
    """Momentum thickness far downstream (one surface's share of Cd / 2), the
    closed form of Squire and Young: theta U^((H + 5) / 2) at the trailing edge."""
    return theta * U ** ((H + 5.0) / 2.0)


def march(h, U, Re):
    """Thwaites's method along one surface.

    h[k] (k = 1..K+1) is the distance from point k-1 to point k (h[0] unused),
    U[k] the speed at point k with U[0] = 0 (the stagnation point) and the last
    point K+1 the trailing edge.  Returns theta, lam (per point) and e, the
    end point (the first k >= 1 with lambda < -0.09 or U = 0, else K+1)."""
    h = np.asarray(h, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    npt = len(U)
    K = npt - 2
    I = np.zeros(npt)
    for k in range(1, npt):
        a, b = U[k - 1], U[k]
        I[k] = I[k - 1] + h[k] * (a**5 + a**4 * b + a**3 * b**2 + a**2 * b**3 + a * b**4 + b**5) / 6.0
    dU = np.zeros(npt)
    dU[0] = U[1] / h[1]
    for k in range(1, K + 1):
        if k < K:
            hm, hp = h[k], h[k + 1]
            dU[k] = (hm * hm * (U[k + 1] - U[k]) + hp * hp * (U[k] - U[k - 1])) / (hm * hp * (hm + hp))
        elif K >= 2:
            a, b = h[k - 1], h[k]
            dU[k] = (U[k - 2] * b / (a * (a + b)) - U[k - 1] * (a + b) / (a * b)
                     + U[k] * (a + 2.0 * b) / (b * (a + b)))
        else:
            dU[k] = (U[k] - U[k - 1]) / h[k]
    dU[K + 1] = dU[K]
    theta2 = np.empty(npt)
    theta2[0] = 0.075 / (Re * dU[0])
    lam = np.empty(npt)
    lam[0] = 0.075
    e = K + 1
    for k in range(1, npt):
        if U[k] == 0.0:
            theta2[k] = math.inf
            lam[k] = -math.inf
        else:
            theta2[k] = 0.45 * I[k] / (Re * U[k] ** 6)
            lam[k] = Re * theta2[k] * dU[k]
    lam[K + 1] = lam[K]
    for k in range(1, K + 1):
        if not (lam[k] >= LAMBDA_SEP):
            e = k
            break
    return np.sqrt(theta2), lam, e


def _surfaces(n, xy, q):
    """Stagnation index j and fraction f, and per surface the control-point
    indices in marching order."""
    j = -1
    for i in range(n - 1):
        if q[i] > 0.0 and q[i + 1] <= 0.0:
            j = i
            break
    if j < 0:
        return None
    f = q[j] / (q[j] - q[j + 1])
    upper = list(range(j, -1, -1))
    lower = list(range(j + 1, n)) if q[j + 1] != 0.0 else list(range(j + 2, n))
    return j, f, upper, lower


def viscous_airfoil(xy, gamma, alpha, Re, vinf=1.0, chord=1.0):
    """One airfoil: xy [n][2] nodes (counter-clockwise, x_0 at the trailing
    edge), gamma [n] panel strengths.  Returns dict(cd, cd_f, theta [n],
    cf [n], sep (upper, lower): the separating control point, -1 if attached,
    stagnation: the stagnation point's coordinates)."""
    xy = np.asarray(xy, dtype=np.float64)
    n = len(xy)
    out = dict(cd=math.nan, cd_f=math.nan, theta=np.full(n, math.nan), cf=np.full(n, math.nan),
               sep=(-2, -2), stagnation=None)
    if not (Re > 0.0 and math.isfinite(Re)):
        return out
    q = np.asarray(gamma, dtype=np.float64) / vinf
    xs = xy / chord
    nxt = np.roll(xs, -1, axis=0)
    L = np.hypot(nxt[:, 0] - xs[:, 0], nxt[:, 1] - xs[:, 1])
    mid = 0.5 * (xs + nxt)
    srf = _surfaces(n, xs, q)
    if srf is None:
        return out
    j, f, upper, lower = srf
    if not lower:
        return out
    dj = 0.5 * (L[j] + L[j + 1])
    # stagnation point on the polyline m_j -> x_{j+1} -> m_{j+1}
    t = f * dj
    if t <= 0.5 * L[j]:
        p0 = mid[j] + (t / (0.5 * L[j])) * (nxt[j] - mid[j])
    else:
        p0 = nxt[j] + ((t - 0.5 * L[j]) / (0.5 * L[j + 1])) * (mid[j + 1] - nxt[j])
    ehat = np.array([math.cos(alpha), math.sin(alpha)])
    te = xs[0]
    cd = 0.0
    cd_f = 0.0
    sep = []
    for side, cps in (("upper", upper), ("lower", lower)):
        K = len(cps)
        h = np.zeros(K + 2)
        U = np.zeros(K + 2)
        P = np.zeros((K + 2, 2))
        P[0] = p0
        for k, c in enumerate(cps, start=1):
            U[k] = abs(q[c])
            P[k] = mid[c]
            if k == 1:
                h[k] = f * dj if side == "upper" else (1.0 - f) * dj
                if side == "lower" and q[j + 1] == 0.0:
                    h[k] = 0.5 * (L[j + 1] + L[j + 2])
            else:
                prev = cps[k - 2]
                h[k] = 0.5 * (L[prev] + L[c])
        last = cps[-1]
        h[K + 1] = 0.5 * L[last]
        U[K + 1] = U[K]
        P[K + 1] = te
        theta, lam, e = march(h, U, Re)
        separated = e <= K
        cf = np.zeros(K + 2)
        for k in range(1, K + 2):
            if not (separated and k >= e):
                l, _ = shear_shape(lam[k])
                cf[k] = 2.0 * l * U[k] / (Re * theta[k])
        for k in range(1, K + 2):
            cd_f += 0.5 * (cf[k - 1] + cf[k]) * float(np.dot(P[k] - P[k - 1], ehat))
        _, He = shear_shape(LAMBDA_SEP if separated else lam[K + 1])
        cd += 2.0 * squire_young(theta[K + 1], U[K + 1], He)
        for k, c in enumerate(cps, start=1):
            out["theta"][c] = theta[k]
            out["cf"][c] = cf[k]
        if side == "lower" and q[j + 1] == 0.0:
            out["theta"][j + 1] = theta[0]
            out["cf"][j + 1] = 0.0
        sep.append(cps[e - 1] if e <= K else -1)
    out["cd"] = cd
    out["cd_f"] = cd_f
    out["sep"] = tuple(sep)
    out["stagnation"] = p0 * chord
    return out


def viscous_batch(nodes, offsets, u, alpha, Re, vinf=None, chord=None, info=None):
    """Batch layout of the library: nodes [sum n][2], offsets [B+1], u packed
    per airfoil at offsets[b] + b (gamma_0..gamma_{n-1}, C)."""
    B = len(offsets) - 1
    N = int(offsets[-1])
    res = dict(cd=np.full(B, math.nan), cd_f=np.full(B, math.nan), theta=np.full(N, math.nan),
               cf=np.full(N, math.nan), sep=np.full((B, 2), -2, dtype=np.int32))
    for b in range(B):
        o0, o1 = int(offsets[b]), int(offsets[b + 1])
        if info is not None and info[b] != 0:
            continue
        n = o1 - o0
        r = viscous_airfoil(nodes[o0:o1], u[o0 + b:o0 + b + n], float(alpha[b]),
                            float(np.broadcast_to(Re, (B,))[b]),
                            1.0 if vinf is None else float(vinf[b]),
                            1.0 if chord is None else float(chord[b]))
        res["cd"][b] = r["cd"]
        res["cd_f"][b] = r["cd_f"]
        res["theta"][o0:o1] = r["theta"]
        res["cf"][o0:o1] = r["cf"]
        res["sep"][b] = r["sep"]
    return res

"""Pins of the viscous-correction oracle (oracle/viscous.py, Thwaites's method
on the panel solution) against what does not depend on it: closed forms of
Thwaites's integral for power-law speeds, exact Falkner-Skan similarity
solutions computed here by shooting, the method's analytic solution on a
circular cylinder (the validation case of Section 2), the Blasius flat-plate
drag as the thin-airfoil limit, and Reynolds-number scaling."""
import math

import numpy as np
import pytest

import oracle
from oracle import viscous as ov
from paper_1511_02166_gb300 import inputs

scipy_integrate = pytest.importorskip("scipy.integrate")
scipy_optimize = pytest.importorskip("scipy.optimize")


def test_linear_speed_is_exact():
    # U = a s (plane stagnation flow): Thwaites gives theta^2 = 0.075 / (a Re) and
    # lambda = 0.075 everywhere; U is piecewise linear, so the discrete march is exact.
    rng = np.random.default_rng(3)
    h = np.concatenate([[0.0], 0.01 + 0.05 * rng.random(40)])
    s = np.cumsum(h)
    a, Re = 2.7, 3.0e5
    theta, lam, e = ov.march(h, a * s, Re)
    assert e == len(s) - 1
    assert np.max(np.abs(theta**2 * a * Re / 0.075 - 1.0)) < 1e-12
    assert np.max(np.abs(lam - 0.075)) < 1e-13


@pytest.mark.parametrize("m", [0.5, 2.0])
def test_power_law_speed_converges_at_second_order(m):
    # U = s^m: theta^2 = 0.45 s^(1-m) / ((5m + 1) Re), lambda = 0.45 m / (5m + 1).
    Re = 1.0e6
    errs = []
    for K in (100, 200, 400):
        t = np.linspace(0.0, 1.0, K + 2)
        s = (t ** 1.5)  # graded towards the stagnation point
        h = np.concatenate([[0.0], np.diff(s)])
        theta, lam, _ = ov.march(h, s ** m, Re)
        sel = s >= 0.2
        th_ex = np.sqrt(0.45 * s[sel] ** (1 - m) / ((5 * m + 1) * Re))
        errs.append(max(np.max(np.abs(theta[sel] / th_ex - 1)),
                        np.max(np.abs(lam[sel] - 0.45 * m / (5 * m + 1)))))
    assert errs[-1] < 2e-4
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def _falkner_skan(m, etamax=10.0):
    """Exact wedge-flow boundary layer f''' + f f'' + beta (1 - f'^2) = 0,
    beta = 2m / (m + 1), by shooting on f''(0); returns f''(0) and the
    momentum and displacement integrals in the similarity variable."""
    beta = 2 * m / (m + 1)

    def rhs(t, y):
        return [y[1], y[2], -y[0] * y[2] - beta * (1 - y[1] ** 2)]

    def over(t, y):
        return y[1] - 2.0
    over.terminal = True

    def under(t, y):
        return y[1] + 0.5
    under.terminal = True

    def shoot(s):
        sol = scipy_integrate.solve_ivp(rhs, [0, etamax], [0, 0, s], rtol=1e-11, atol=1e-12,
                                        events=[over, under])
        if sol.t_events[0].size:
            return 1.0
        if sol.t_events[1].size:
            return -1.0
        return sol.y[1, -1] - 1.0

    s = scipy_optimize.brentq(shoot, 0.0 if m >= 0 else 1e-4, 2.0, xtol=1e-13)
    sol = scipy_integrate.solve_ivp(rhs, [0, etamax], [0, 0, s], rtol=1e-11, atol=1e-12,
                                    dense_output=True)
    eta = np.linspace(0, etamax, 20001)
    fp = sol.sol(eta)[1]
    return s, np.trapezoid(fp * (1 - fp), eta), np.trapezoid(1 - fp, eta)


@pytest.mark.parametrize("m,tol", [(0.0, 0.01), (0.1, 0.04), (0.3, 0.05), (1.0, 0.06),
                                   (-0.03, 0.04)])
def test_shear_and_shape_functions_against_similarity_solutions(m, tol):
    # Thwaites's l and H are fits to exact solutions; the Cebeci-Bradshaw forms
    # stay within a few per cent of Falkner-Skan flows (lambda = 2m/(m+1) Theta^2,
    # l = f''(0) Theta, H = Delta / Theta).
    fpp, Th, De = _falkner_skan(m)
    lam = 2 * m / (m + 1) * Th ** 2
    l, H = ov.shear_shape(lam)
    assert abs(l / (fpp * Th) - 1) < tol
    assert abs(H / (De / Th) - 1) < tol


def test_separation_value_of_the_shear_function():
    # Laminar separation (zero wall shear) is where l vanishes: lambda = -0.09.
    l, H = ov.shear_shape(-0.09)
    assert abs(l) < 0.005 and 3.4 < H < 3.7
    assert ov.shear_shape(-0.2) == ov.shear_shape(-0.09)
    assert ov.shear_shape(0.3) == ov.shear_shape(0.1)


R_CYL = 0.5


def _i5(phi):
    return scipy_integrate.quad(lambda t: math.sin(t) ** 5, 0, phi, epsabs=0, epsrel=1e-13)[0]


def _cyl_lambda(phi):
    # U = 2 sin(phi), s = R phi:  lambda = 0.45 cos(phi) int_0^phi sin^5 / sin^6(phi)
    return 0.45 * _i5(phi) * math.cos(phi) / math.sin(phi) ** 6


def _cyl_theta(phi, Re):
    return math.sqrt(0.45 * R_CYL * _i5(phi) / (2 * Re * math.sin(phi) ** 6))


def test_cylinder_against_the_analytic_solution():
    # Section 2 validates the viscous correction on a circular cylinder against
    # Thwaites's analytic solution; here the whole oracle path (panel solve,
    # stagnation point, march, separation, friction integral) is compared with it.
    Re = 1.0e5
    phi_sep = scipy_optimize.brentq(lambda p: _cyl_lambda(p) + 0.09, 1.6, 2.5)
    cf = lambda p: 2 * ov.shear_shape(_cyl_lambda(p))[0] * 2 * math.sin(p) / (Re * _cyl_theta(p, Re))
    cdf_exact = 2 * scipy_integrate.quad(lambda p: cf(p) * math.sin(p) * R_CYL, 1e-9, phi_sep,
                                         limit=200)[0]
    errs = []
    for n in (200, 400, 800):
        xy = inputs.cylinder(n)
        u = oracle.evaluate(xy, 0.0)["u"]
        v = ov.viscous_airfoil(xy, u[:n], 0.0, Re)
        mid = 0.5 * (xy + np.roll(xy, -1, axis=0))
        phi = np.abs(np.arctan2(mid[:, 1], 0.5 - mid[:, 0]))  # angle from the front stagnation point
        dphi = 2 * math.pi / n
        for s in v["sep"]:
            assert phi_sep < phi[s] <= phi_sep + dphi + 1e-12
        j = int(np.argmin(np.abs(phi[: n // 2] - math.radians(60))))
        errs.append(abs(v["theta"][j] / _cyl_theta(phi[j], Re) - 1))
        # zero wall shear past separation, as the analytic integral ending there
        up, lo = v["sep"]
        assert np.all(v["cf"][:up + 1] == 0.0) and np.all(v["cf"][lo:] == 0.0)
        assert np.all(v["cf"][up + 1:lo] > 0.0)
        if n == 800:
            assert abs(v["cd_f"] / cdf_exact - 1) < 2e-4
    assert errs[-1] < 5e-5 and errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_reynolds_scaling():
    # theta ~ Re^-1/2 at fixed speeds, lambda independent of Re.
    xy = inputs.naca4(0.02, 0.4, 0.12, 160)
    u = oracle.evaluate(xy, math.radians(3.0))["u"]
    a = ov.viscous_airfoil(xy, u[:160], math.radians(3.0), 1e5)
    b = ov.viscous_airfoil(xy, u[:160], math.radians(3.0), 1e7)
    assert a["sep"] == b["sep"]
    assert abs(a["cd"] / b["cd"] - 10.0) < 1e-11
    assert abs(a["cd_f"] / b["cd_f"] - 10.0) < 1e-11
    ok = np.isfinite(a["theta"])
    assert np.max(np.abs(a["theta"][ok] / b["theta"][ok] - 10.0)) < 1e-11


def test_thin_symmetric_airfoil_flat_plate_limit():
    # A 2 % thick symmetric section at zero incidence: both surfaces see nearly
    # the freestream, so the Squire-Young drag approaches Blasius's flat plate,
    # 2 x 1.328 / sqrt(Re) (both sides; the closed trailing edge, where the
    # inviscid speed falls, keeps it a few per cent off), friction and profile
    # drag nearly agree, and the two surfaces mirror each other.
    n, Re = 400, 1.0e6
    xy = inputs.naca4(0.0, 0.4, 0.02, n)
    u = oracle.evaluate(xy, 0.0)["u"]
    v = ov.viscous_airfoil(xy, u[:n], 0.0, Re)
    assert abs(v["cd"] * math.sqrt(Re) / 2.656 - 1) < 0.05
    assert 0.95 < v["cd_f"] / v["cd"] < 1.05
    up, lo = v["sep"]
    assert up + lo == n - 1
    ok = np.isfinite(v["theta"])
    assert np.array_equal(ok, ok[::-1])
    assert np.max(np.abs(v["theta"][ok] - v["theta"][::-1][ok])) < 1e-9 * np.max(v["theta"][ok])


def test_degenerate_inputs_give_nan():
    xy = inputs.naca4(0.02, 0.4, 0.12, 60)
    u = oracle.evaluate(xy, 0.0)["u"]
    v = ov.viscous_airfoil(xy, np.abs(u[:60]) + 1.0, 0.0, 1e6)  # no stagnation point
    assert math.isnan(v["cd"]) and v["sep"] == (-2, -2)
    v = ov.viscous_airfoil(xy, u[:60], 0.0, 0.0)
    assert math.isnan(v["cd"]) and np.all(np.isnan(v["theta"]))


@pytest.mark.parametrize("U_te,H_te", [(0.9, 2.6), (0.75, 3.55), (1.1, 2.3)])
def test_squire_young_from_the_wake_momentum_equation(U_te, H_te):
    # Squire and Young's closed form is the wake momentum integral without wall
    # shear, d ln(theta) / d ln(U) = -(H + 2), with H - 1 falling linearly in
    # ln U from H_te - 1 at the trailing edge to 0 far downstream (U = 1);
    # integrated here numerically, independently of the closed form
    s0 = math.log(U_te)

    def rhs(s, y):
        H = 1.0 + (H_te - 1.0) * s / s0
        return [-(H + 2.0)]

    sol = scipy_integrate.solve_ivp(rhs, [s0, 0.0], [math.log(0.01)], rtol=1e-12, atol=1e-14)
    theta_inf = math.exp(sol.y[0, -1])
    assert abs(ov.squire_young(0.01, U_te, H_te) / theta_inf - 1) < 1e-9


@pytest.mark.parametrize("alpha_deg", [0.0, 3.0, 8.0])
def test_cylinder_stagnation_point_under_incidence(alpha_deg):
    # With the Kutta condition at its rear point a cylinder carries the
    # circulation that keeps the rear stagnation point there; the front one then
    # sits at the polar angle pi + 2 alpha (potential flow); the linear zero of
    # gamma between two control points must find it well inside one panel
    # (spacing 2 pi / n: 0.031 rad at n = 200)
    a = math.radians(alpha_deg)
    for n in (200, 400, 800):
        xy = inputs.cylinder(n)
        u = oracle.evaluate(xy, a)["u"]
        p0 = ov.viscous_airfoil(xy, u[:n], a, 1e6)["stagnation"]
        ang = math.atan2(p0[1], p0[0] - 0.5) % (2 * math.pi)
        assert abs(ang - (math.pi + 2 * a)) < 1e-4, n

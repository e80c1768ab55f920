"""Closed forms the paper (and elementary kinematics) fix, used to pin the
oracle.  Written independently of the oracle's code.

* beam survival through a piecewise-constant column: exp(-sigma * column),
  the unscattered fraction of Eq. density_injected;
* at most one / two excitations of a beam: the n_s and n_s,2 expressions of
  Sec. 4 (Excitation) integrated over a segment;
* truncated-Lorentzian CDF of the ionization secondary energy;
* relativistic speed and simulated time (Eq. simulated_time).
"""
import math

import numpy as np

C_LIGHT = 299792458.0


def speed(e_ev, m_ev):
    """beta = sqrt(1 - 1/gamma^2) with gamma = 1 + x, x = E/mc^2, written as
    sqrt(x (2 + x)) / (1 + x) so thermal ions (x ~ 1e-11) keep full precision."""
    x = e_ev / m_ev
    return C_LIGHT * math.sqrt(x * (2.0 + x)) / (1.0 + x)


def column_to_faces(n_seg, dz):
    return np.concatenate([[0.0], np.cumsum(n_seg) * dz])


def survival_at_faces(n_seg, dz, sigma):
    """P(no collision before face k) for a +z beam born at z = 0."""
    return np.exp(-sigma * column_to_faces(n_seg, dz))


def survival_segment_integrals(n_seg, dz, sigma):
    """int over segment j of P(no collision before z) dz."""
    c = column_to_faces(n_seg, dz)
    out = np.empty(len(n_seg))
    for j, n in enumerate(n_seg):
        a = sigma * n
        out[j] = math.exp(-sigma * c[j]) * (dz if a == 0 else -math.expm1(-a * dz) / a)
    return out


def excitation_probabilities(x, lam1, lam2):
    """Probability of zero, exactly one and exactly two scatterings after a
    distance x in gas (two excitations at most): S, P1, P2 (Sec. 4, Excitation)."""
    s = math.exp(-x / lam1)
    if abs(lam2 - lam1) < 1e-15 * lam1:
        p1 = x / lam1 * s
    else:
        p1 = lam2 / (lam2 - lam1) * (math.exp(-x / lam2) - math.exp(-x / lam1))
    return s, p1, 1.0 - s - p1


def segment_average(fn, lo, hi, n=400):
    """Gauss-Legendre integral of fn over [lo, hi]."""
    xs, ws = np.polynomial.legendre.leggauss(n)
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    return half * sum(w * fn(mid + half * x) for x, w in zip(xs, ws))


def lorentz_cdf(w, eps, wmax):
    """CDF of W with pdf ~ 1/(1+(W/eps)^2) on [0, wmax]."""
    w = np.clip(w, 0.0, wmax)
    return np.arctan(w / eps) / math.atan(wmax / eps)


def bound_sigma(mean, xmax, n):
    """Standard deviation bound of a sum of n i.i.d. variables in [0, xmax]
    with the given total mean: Var(X) <= E[X](xmax - E[X])."""
    m = mean / n
    return math.sqrt(max(n * m * (xmax - m), 0.0))


# ---------------------------------------------------------------------------
# charge exchange on a Maxwellian gas (Sec. 3.3 Charge exchange): the ion
# takes the velocity w of a target met at a rate proportional to the relative
# speed, i.e. w ~ |u - w| f(w), f the Maxwellian with per-component variance
# a^2.  Written in units of a; both forms reduce the angular integral to
# closed form.

def _shell_relative_speed(x, x0):
    """Mean of |u - w| over directions of w, |u| = x0, |w| = x (units of a):
    ((x0 + x)^3 - |x0 - x|^3) / (6 x0 x)."""
    if x <= 0.0:
        return x0
    return ((x0 + x) ** 3 - abs(x0 - x) ** 3) / (6.0 * x0 * x)


def maxwell_mean_relative_speed(x):
    """g(x) = E|u - w| over w ~ f for |u| = x (units of a):
    sqrt(2/pi) exp(-x^2/2) + (x + 1/x) erf(x / sqrt 2)."""
    if x < 1e-8:
        return 2.0 * math.sqrt(2.0 / math.pi)
    return (math.sqrt(2.0 / math.pi) * math.exp(-0.5 * x * x)
            + (x + 1.0 / x) * math.erf(x / math.sqrt(2.0)))


def cx_one_collision_speed_moments(x0):
    """E[|w|^2] and E[|w|^4] (units of a) after one charge exchange of an ion
    of speed x0."""
    from scipy import integrate
    w = lambda x, p: x ** p * math.exp(-0.5 * x * x) * _shell_relative_speed(x, x0)
    hi = 12.0
    z = integrate.quad(lambda x: w(x, 2), 0, hi, limit=200)[0]
    m2 = integrate.quad(lambda x: w(x, 4), 0, hi, limit=200)[0] / z
    m4 = integrate.quad(lambda x: w(x, 6), 0, hi, limit=200)[0] / z
    return m2, m4


def cx_stationary_speed_moments():
    """E[|u|^2] and E[|u|^4] (units of a) of the ion velocity after a collision
    once repeated charge exchange has forgotten the start: the chain
    u' ~ |u - w| f(w) has the stationary density f(u) g(u)."""
    from scipy import integrate
    w = lambda x, p: x ** p * math.exp(-0.5 * x * x) * maxwell_mean_relative_speed(x)
    hi = 12.0
    z = integrate.quad(lambda x: w(x, 2), 0, hi, limit=200)[0]
    m2 = integrate.quad(lambda x: w(x, 4), 0, hi, limit=200)[0] / z
    m4 = integrate.quad(lambda x: w(x, 6), 0, hi, limit=200)[0] / z
    return m2, m4


def cx_one_collision_mean_wz(x0):
    """E[w_z] (units of a) after one charge exchange of an ion moving along +z
    with speed x0: targets moving against the ion are met more often."""
    from scipy import integrate
    g = lambda c, x: x * x * math.exp(-0.5 * x * x) * math.sqrt(
        max(x0 * x0 + x * x - 2.0 * x0 * x * c, 0.0))
    num = integrate.dblquad(lambda c, x: x * c * g(c, x), 0, 12.0, -1.0, 1.0)[0]
    den = integrate.dblquad(g, 0, 12.0, -1.0, 1.0)[0]
    return num / den

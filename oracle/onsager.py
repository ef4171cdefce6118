"""Exact results of the 2D square-lattice Ising model (test infrastructure only).

Used to pin the CTM oracle through a PEPS whose norm network is the classical
Ising partition function.  Nothing in the product path imports this module.

* Onsager (1944): free energy per site, written two independent ways (double
  integral over the Brillouin zone and the single elliptic-type integral).
* Nearest-neighbour correlation <s s'> from the complete elliptic integral K.
* Yang (1952): spontaneous magnetisation (1 - sinh(2 beta)^-4)^(1/8) above beta_c.
"""
import numpy as np
from scipy import integrate, special

BETA_C = 0.5 * np.log(1.0 + np.sqrt(2.0))


def lnz_double_integral(beta):
    """ln Z / N = ln 2 + (1/8 pi^2) iint ln[cosh^2 2b - sinh 2b (cos t1 + cos t2)] dt1 dt2.

    The inner angle is integrated in closed form with
    int_0^{2 pi} ln(a - s cos t) dt = 2 pi ln[(a + sqrt(a^2 - s^2)) / 2].
    """
    c2, s2 = np.cosh(2 * beta) ** 2, np.sinh(2 * beta)

    def inner(t1):
        a = c2 - s2 * np.cos(t1)
        return np.log(0.5 * (a + np.sqrt(a * a - s2 * s2)))

    val, _ = integrate.quad(inner, 0.0, np.pi, epsabs=1e-14, epsrel=1e-13, limit=400)
    # inner() is even in t1: the [0, 2 pi] integral is twice this one
    return np.log(2.0) + 2.0 * np.pi * 2.0 * val / (8.0 * np.pi ** 2)


def lnz_single_integral(beta):
    """ln Z / N = ln(2 cosh 2b) + (1/pi) int_0^{pi/2} ln[(1 + sqrt(1 - k^2 sin^2 t)) / 2] dt."""
    k = 2.0 * np.sinh(2 * beta) / np.cosh(2 * beta) ** 2
    f = lambda t: np.log(0.5 * (1.0 + np.sqrt(1.0 - (k * np.sin(t)) ** 2)))
    val, _ = integrate.quad(f, 0.0, 0.5 * np.pi, epsabs=1e-14, epsrel=1e-13, limit=400)
    return np.log(2.0 * np.cosh(2 * beta)) + val / np.pi


def nn_correlation(beta):
    """<s_i s_j> on a nearest-neighbour bond:
    (1/2) coth(2b) [1 + (2/pi)(2 tanh^2 2b - 1) K(k)], k = 2 sinh 2b / cosh^2 2b."""
    k = 2.0 * np.sinh(2 * beta) / np.cosh(2 * beta) ** 2
    K = special.ellipk(k * k)  # scipy takes the parameter m = k^2
    t2 = np.tanh(2 * beta) ** 2
    return 0.5 / np.tanh(2 * beta) * (1.0 + 2.0 / np.pi * (2.0 * t2 - 1.0) * K)


def magnetization(beta):
    """Spontaneous magnetisation (Yang): (1 - sinh(2 beta)^-4)^(1/8) for beta > beta_c."""
    if beta <= BETA_C:
        return 0.0
    return (1.0 - np.sinh(2 * beta) ** -4) ** 0.125

"""Reference solution of the layered two-phase Poiseuille flow (Sec. 4.4).

The steady x-invariant momentum balance with the diffuse viscosity profile,
d/dy (zeta(y) du/dy) + F_x = 0 with u(0) = u(H) = 0 (Eq. NSE_for_layered_poiseuille)
and zeta(y) of Eq. viscosity_prof, integrates once to zeta u' = -F_x (y - y*), so

    u(y) = F_x * integral_0^y (y* - s) / zeta(s) ds,
    y*   = integral_0^H s / zeta ds  /  integral_0^H 1 / zeta ds,

evaluated here by the trapezoidal rule on a fine grid (the paper solves the same
equation with second-order finite differences at dy = 4e-8 m).  Test
infrastructure: independent of the oracle and of the CUDA path."""
import numpy as np


def zeta_profile(s, H, W, zeta_l, zeta_g):
    """Eq. viscosity_prof: liquid (zeta_l) below y = H/2, gas above."""
    return 0.5 * (zeta_l + zeta_g) - 0.5 * (zeta_l - zeta_g) * np.tanh((2.0 * s - H) / W)


def layered_reference(y, H, W, Fx, zeta_l, zeta_g, n=400001):
    s = np.linspace(0.0, H, n)
    inv = 1.0 / zeta_profile(s, H, W, zeta_l, zeta_g)
    ds = np.diff(s)

    def cumtrap(f):
        return np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * ds)])

    i0, i1 = cumtrap(inv), cumtrap(s * inv)
    ystar = i1[-1] / i0[-1]
    return np.interp(y, s, Fx * (ystar * i0 - i1))


def reference_for(w):
    return layered_reference(w["y"], w["H"], w["W"], w["Fx"], w["zeta_l"], w["zeta_g"])


def e2(u, ref):
    """Global relative error of Sec. 4 (Eq. error_norm_2), as a fraction."""
    return float(np.sqrt(np.sum((np.asarray(u) - ref) ** 2) / np.sum(ref ** 2)))

"""Closed-form solutions used as pins (no method arithmetic of the BEM).

Sound-soft sphere in a plane wave (the classical Mie series): the incident
field e^{i k d.x} = sum_l (2l + 1) i^l j_l(k r) P_l(cos g) has the scattered
field outside the sphere of radius a
    u_s(x) = - sum_l (2l + 1) i^l (j_l(k a) / h_l(k a)) h_l(k r) P_l(cos g),
with h_l = j_l + i y_l the outgoing spherical Hankel function and g the angle
between x and d, so that u_i + u_s = 0 on |x| = a.
"""
import numpy as np
from scipy import special


def mie_sound_soft(k, d, X, radius=1.0, lmax=None):
    """Scattered field at points X (P, 3), |X| >= radius, for unit direction d."""
    X = np.asarray(X, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    if lmax is None:
        lmax = int(np.ceil(k * radius)) + 30
    r = np.linalg.norm(X, axis=1)
    ct = np.clip(X @ d / r, -1.0, 1.0)
    u = np.zeros(len(X), dtype=np.complex128)
    for l in range(lmax + 1):
        ja = special.spherical_jn(l, k * radius)
        ha = ja + 1j * special.spherical_yn(l, k * radius)
        hr = special.spherical_jn(l, k * r) + 1j * special.spherical_yn(l, k * r)
        u -= (2 * l + 1) * (1j ** l) * (ja / ha) * hr * special.eval_legendre(l, ct)
    return u

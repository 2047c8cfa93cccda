"""Diagnostics of computed fields (oracle; test infrastructure only).

Sec. "Verification tests" plots a spherically averaged I-front position without
defining it; the reading used here is the radius of the sphere whose volume
equals the ionised volume, r_I = (3 V_ion / (4 pi))^{1/3} with
V_ion = sum_cells x_HII dV (times 8 for an octant set-up with the source in the
corner cell and zero-flux walls).
"""
import math

import numpy as np


def ifront_radius(nHI, nH, dx, octant):
    """Comoving equivalent-volume radius of the ionised region [cm]."""
    xHII = 1.0 - np.asarray(nHI) / np.asarray(nH)
    V = float(np.sum(xHII)) * dx**3 * (8.0 if octant else 1.0)
    return (3.0 * V / (4.0 * math.pi)) ** (1.0 / 3.0)

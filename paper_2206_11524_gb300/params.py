"""Host-side parameter conversions of the paper (no lattice arithmetic).

Huang et al.'s correlation between the adhesion parameter and the contact
angle (Eq. 15, Table 1): G_ads,2 = -G_ads,1 = G_inter,12 (rho_1 - rho_dis,2)
cos(theta) / 4.  The viscosity of the lattice BGK model (Appendix A):
nu = c_s^2 (tau - 1/2), c_s^2 = 1/3.  The gray-scale permeability of a
uniform bounce-back fraction (Eq. 2): k = nu (1 - n_s) / (2 n_s).
"""
from __future__ import annotations

import math


def gads_from_contact_angle(theta_deg: float, G: float = 1.75,
                            rho_1: float = 0.99, rho_dis_2: float = 0.01) -> float:
    """G_ads,2 for a contact angle theta (degrees), Table 1 / Eq. 15."""
    return 0.25 * G * (rho_1 - rho_dis_2) * math.cos(math.radians(theta_deg))


def contact_angle_from_gads(gads2: float, G: float = 1.75, rho_1: float = 0.99,
                            rho_dis_2: float = 0.01) -> float:
    """theta_H in degrees for G_ads,2 (Eq. 15)."""
    return math.degrees(math.acos(4.0 * gads2 / (G * (rho_1 - rho_dis_2))))


def viscosity(tau: float) -> float:
    """Kinematic viscosity nu = c_s^2 (tau - 1/2) in lattice units."""
    return (tau - 0.5) / 3.0


def permeability(ns: float, tau: float = 1.0) -> float:
    """Eq. 2: permeability of a uniform gray medium, lattice units."""
    return viscosity(tau) * (1.0 - ns) / (2.0 * ns)

"""Closed-form LO gg -> Q Qbar matrix element -- TEST INFRASTRUCTURE ONLY.

Ellis, Stirling, Webber, "QCD and collider physics" (heavy-quark production at lowest order;
Combridge 1979): averaged over initial spins and colours and summed over final ones,

    sum|M|^2 / g^4 = (1/(6 tau1 tau2) - 3/8) (tau1^2 + tau2^2 + rho - rho^2/(4 tau1 tau2)),
    tau1 = 2 p1.p3 / s,  tau2 = 2 p1.p4 / s,  rho = 4 m^2 / s,  g^2 = 4 pi alpha_s.

For m -> 0 it reduces to the textbook gg -> q qbar result (t^2+u^2)/(6tu) - 3(t^2+u^2)/(8 s^2).
"""
import math

import numpy as np


def mdot(a, b):
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def ggtt_me(mom, mt, alphas):
    """mom[..., 4, 4] in particle order g1 g2 t tbar."""
    mom = np.asarray(mom, dtype=np.float64)
    p1, p2, p3, p4 = mom[..., 0, :], mom[..., 1, :], mom[..., 2, :], mom[..., 3, :]
    s = mdot(p1 + p2, p1 + p2)
    t1 = 2.0 * mdot(p1, p3) / s
    t2 = 2.0 * mdot(p1, p4) / s
    rho = 4.0 * mt * mt / s
    g2 = 4.0 * math.pi * alphas
    return g2 * g2 * (1.0 / (6.0 * t1 * t2) - 3.0 / 8.0) * (t1 * t1 + t2 * t2 + rho - rho * rho / (4.0 * t1 * t2))

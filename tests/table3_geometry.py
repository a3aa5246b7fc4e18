"""Equilibrium shape of the quaternary compound drop of Sec. 4.3 (the
analytical reference of Table 3, App. D), in a construction of our own.

Three drops (phases 1, 2, 3, side by side on a flat wall y = 0, each of the
area of a semicircle of radius 1) sit in the ambient phase 4; all surface
tensions are equal and theta_14 = theta_24 = 90 deg, so theta_12 = 90 deg
by Eq. 2.9, and theta_23 = 180 deg - theta_34.  As App. D does, the 1|2
interface is the straight segment BF normal to the wall (B at the origin);
every other interface is a circular arc:
  * phase 1: the arc AF is centred on the wall (it meets the wall at
    theta_14 = 90 deg) and meets BF at F under 120 deg (equal tensions), so
    its centre is at (-a, 0), its radius r = 2a and F = (0, sqrt(3) a); its
    area pi r^2 / 3 + sqrt(3) r^2 / 8 fixes r, and L1 = AB = a + r;
  * phase 2: the arc FG leaves F at 30 deg above the wall (the third
    direction of the 120-deg junction at F); at the triple junction G the
    arcs GF, GC (2|3) and GE (3|4) leave 120 deg apart; GC meets the wall
    at C under theta_23 (measured in phase 2), GE meets it at E under
    theta_34 (measured in phase 3);
  * the curvature and length of FG are the two unknowns, solved by
    Newton's method (scipy's hybrid solver) from the areas of phases 2 and
    3; the curvatures of GC and GE follow from their wall angles.
L2 = BC and L3 = CE.  At theta_34 = 90 deg the shape is symmetric, and then
L3 = L1 and L2 solves w h + (pi/6 - sqrt(3)/4) w^2 = pi/2 in closed form.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq, fsolve

DEG = math.pi / 180.0


def phase1(area=math.pi / 2):
    r = math.sqrt(area / (math.pi / 3.0 + math.sqrt(3.0) / 8.0))
    a = r / 2.0
    return r, a, math.sqrt(3.0) * a


def arc(P0, phi0, k, s, n=2000):
    """Points of the arc from P0 with initial tangent angle phi0, signed
    curvature k (positive: turning counter-clockwise), length s."""
    t = np.linspace(0.0, s, n)
    if abs(k) < 1e-12:
        return np.c_[P0[0] + t * math.cos(phi0), P0[1] + t * math.sin(phi0)]
    return np.c_[P0[0] + (np.sin(phi0 + k * t) - math.sin(phi0)) / k,
                 P0[1] + (math.cos(phi0) - np.cos(phi0 + k * t)) / k]


def to_wall(P0, phi0, k):
    """Arc length from P0 (above the wall) to the first crossing of y = 0,
    or None."""
    if abs(k) < 1e-12:
        sn = math.sin(phi0)
        return -P0[1] / sn if sn < 0 else None
    c = math.cos(phi0) + k * P0[1]
    if abs(c) > 1.0:
        return None
    best = None
    for base in (math.acos(c), -math.acos(c)):
        for n in range(-3, 4):
            s = (base + 2.0 * math.pi * n - phi0) / k
            if s > 1e-12 and (best is None or s < best):
                best = s
    return best


def wall_angle(P0, phi0, k):
    """Angle between the wall ray towards -x and the interface at its
    wall end (measured in the phase to the left of the end point)."""
    s = to_wall(P0, phi0, k)
    if s is None:
        return None
    phi = phi0 + k * s
    up = math.atan2(-math.sin(phi), -math.cos(phi))
    return 180.0 - up / DEG


def _curvature_for(P0, phi0, target):
    ks = np.linspace(-2.0, 2.0, 401)
    vals = [wall_angle(P0, phi0, k) for k in ks]
    for i in range(len(ks) - 1):
        if vals[i] is None or vals[i + 1] is None:
            continue
        if (vals[i] - target) * (vals[i + 1] - target) <= 0.0:
            return brentq(lambda k: wall_angle(P0, phi0, k) - target, ks[i], ks[i + 1], xtol=1e-15)
    raise RuntimeError("no arc meets the wall under %.3f deg" % target)


def _shoelace(P):
    x, y = P[:, 0], P[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def spreading_lengths(theta34_deg, area=math.pi / 2):
    """(L1, L2, L3) in units of the initial radius."""
    r, a, h = phase1(area)
    F = (0.0, h)
    th23 = 180.0 - theta34_deg

    def shape(k1, s1):
        fg = arc(F, 30.0 * DEG, k1, s1)
        G = tuple(fg[-1])
        back = 30.0 * DEG + k1 * s1 + math.pi                  # at G, towards F
        tgc, tge = back + 2.0 * math.pi / 3.0, back - 2.0 * math.pi / 3.0
        k2 = _curvature_for(G, tgc, th23)
        k3 = _curvature_for(G, tge, theta34_deg)
        gc = arc(G, tgc, k2, to_wall(G, tgc, k2))
        ge = arc(G, tge, k3, to_wall(G, tge, k3))
        p2 = np.vstack([[[0.0, 0.0]], fg, gc[1:]])
        p3 = np.vstack([gc[::-1], ge[1:]])
        return _shoelace(p2), _shoelace(p3), gc[-1, 0], ge[-1, 0]

    def resid(v):
        A2, A3, _, _ = shape(*v)
        return [A2 - area, A3 - area]

    w = symmetric_L2(area)
    k1, s1 = fsolve(resid, [-1.0 / w, w * math.pi / 3.0], xtol=1e-12)
    _, _, xc, xe = shape(k1, s1)
    return a + r, xc, xe - xc


def symmetric_L2(area=math.pi / 2):
    """theta_34 = 90 deg: phase 2 is the rectangle under BF and its mirror
    plus the circular segment of the arc FG (radius w, half-angle 30 deg)."""
    _, _, h = phase1(area)
    q = math.pi / 6.0 - math.sqrt(3.0) / 4.0
    return (-h + math.sqrt(h * h + 4.0 * q * area)) / (2.0 * q)

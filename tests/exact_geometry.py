"""Independent reference geometry used to pin the oracle.

Nothing here shares code with the oracle: these are closed forms and brute
force constructions of the SES (§1) for special cases.

* single atom: the SES is the van der Waals sphere;
* two atoms: the molecule is a solid of revolution; distances are computed in
  the meridian half-plane by dense sampling of the free boundary, and area and
  volume by Pappus' theorems on the exact profile (spherical zones + the probe
  arc, cut at the axis in the spindle case);
* a few atoms: dense Fibonacci sampling of the expanded spheres gives free
  probe centres; the distance to the nearest free sample bounds
  dist(x, Omega_free) from above, within the sample spacing.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate
from scipy.spatial import cKDTree


def fibonacci_sphere(n: int) -> np.ndarray:
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    rr = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([rr * np.cos(phi), rr * np.sin(phi), z], axis=1)


def sphere_first_root(s: np.ndarray, axis: int, h: float, c: np.ndarray, r: float):
    """Smallest tau in [0,1] with |s + tau h e_axis - c| = r (or None)."""
    d = s - c
    # |d + t e|^2 = r^2 with t = tau*h: t^2 + 2 d_a t + |d|^2 - r^2 = 0
    b = d[axis]
    cc = float(d @ d) - r * r
    disc = b * b - cc
    if disc < 0:
        return None
    sq = math.sqrt(disc)
    roots = sorted([(-b - sq) / h, (-b + sq) / h])
    for t in roots:
        if -1e-12 <= t <= 1 + 1e-12:
            return min(max(t, 0.0), 1.0)
    return None


class TwoAtoms:
    """Two atoms on the z' axis of a local frame: c1 = 0, c2 = D e."""

    def __init__(self, c1, c2, r1, r2, rp, n_samples=200000):
        self.c1 = np.asarray(c1, float)
        self.c2 = np.asarray(c2, float)
        self.r1, self.r2, self.rp = float(r1), float(r2), float(rp)
        self.R1, self.R2 = r1 + rp, r2 + rp
        d = self.c2 - self.c1
        self.D = float(np.linalg.norm(d))
        self.e = d / self.D
        D, R1, R2 = self.D, self.R1, self.R2
        assert abs(R1 - R2) < D < R1 + R2, "expanded spheres must meet in a circle"
        self.a = (D * D + R1 * R1 - R2 * R2) / (2 * D)
        self.rho = math.sqrt(R1 * R1 - self.a * self.a)
        # free boundary in the meridian half-plane (z, w >= 0): upper arcs of
        # both expanded circles that lie outside the other disk
        th = np.linspace(0.0, math.pi, n_samples)
        arc1 = np.stack([R1 * np.cos(th), R1 * np.sin(th)], 1)
        arc2 = np.stack([D + R2 * np.cos(th), R2 * np.sin(th)], 1)
        free1 = arc1[(arc1[:, 0] - D) ** 2 + arc1[:, 1] ** 2 >= R2 * R2]
        free2 = arc2[arc2[:, 0] ** 2 + arc2[:, 1] ** 2 >= R1 * R1]
        pts = np.concatenate([free1, free2, [[self.a, self.rho]]], 0)
        self.tree = cKDTree(pts)
        self.spacing = math.pi * max(R1, R2) / n_samples

    def meridian(self, x):
        x = np.atleast_2d(np.asarray(x, float)) - self.c1
        z = x @ self.e
        w = np.linalg.norm(x - z[:, None] * self.e[None, :], axis=1)
        return z, w

    def distance(self, x):
        """dist(x, Omega_free) from the sampled meridian free boundary (0 if x is free)."""
        z, w = self.meridian(x)
        free = (z * z + w * w >= self.R1 ** 2) & ((z - self.D) ** 2 + w * w >= self.R2 ** 2)
        d, _ = self.tree.query(np.stack([z, w], 1))
        return np.where(free, 0.0, d)

    def area_volume(self):
        """SES area and enclosed volume by Pappus on the exact profile."""
        r1, r2, rp, D, a, rho = self.r1, self.r2, self.rp, self.D, self.a, self.rho
        R1, R2 = self.R1, self.R2
        cos1 = a / R1              # angle of P seen from c1 (from +z)
        cos2 = (D - a) / R2        # angle of P seen from c2 (from -z)
        A = 2 * math.pi * r1 * r1 * (1 + cos1) + 2 * math.pi * r2 * r2 * (1 + cos2)
        t1z = a * r1 / R1
        t2z = D + (r2 / R2) * (a - D)
        psi1 = math.atan2(-rho, -a)
        psi2 = math.atan2(-rho, D - a)

        def torus_area(pa, pb):
            return 2 * math.pi * rp * (rho * (pb - pa) - rp * (math.cos(pb) - math.cos(pa)))

        if rho >= rp:
            A += torus_area(psi1, psi2)
        else:
            cut = math.asin(rho / rp)
            A += torus_area(psi1, -math.pi + cut) + torus_area(-cut, psi2)
        V1 = math.pi * ((r1 * r1 * t1z - t1z ** 3 / 3) - (-(r1 ** 3) + r1 ** 3 / 3))
        u0, u1 = t2z - D, r2
        V2 = math.pi * ((r2 * r2 * u1 - u1 ** 3 / 3) - (r2 * r2 * u0 - u0 ** 3 / 3))

        def w2(z):
            s = rp * rp - (z - a) ** 2
            w = rho - math.sqrt(max(s, 0.0))
            return max(w, 0.0) ** 2

        brk = []
        if rho < rp:
            h0 = math.sqrt(rp * rp - rho * rho)
            brk = [a - h0, a + h0]
        Vm, _ = integrate.quad(w2, t1z, t2z, points=brk or None, epsabs=1e-13, epsrel=1e-12, limit=400)
        return A, V1 + V2 + math.pi * Vm


class SampledFree:
    """Dense free probe centres on the expanded spheres of a few atoms."""

    def __init__(self, xyz, radii, rp, n_per_sphere=200000):
        xyz = np.asarray(xyz, float)
        R = np.asarray(radii, float) + rp
        u = fibonacci_sphere(n_per_sphere)
        pts = []
        for i in range(len(R)):
            p = xyz[i] + R[i] * u
            d2 = ((p[:, None, :] - xyz[None, :, :]) ** 2).sum(-1)
            ok = np.ones(len(p), bool)
            for k in range(len(R)):
                if k != i:
                    ok &= d2[:, k] >= R[k] * R[k]
            pts.append(p[ok])
        self.pts = np.concatenate(pts, 0)
        self.tree = cKDTree(self.pts)
        self.xyz, self.R = xyz, R
        self.spacing = max(math.sqrt(4 * math.pi / n_per_sphere) * float(R.max()), 1e-9)

    def distance(self, x):
        x = np.atleast_2d(np.asarray(x, float))
        d2 = ((x[:, None, :] - self.xyz[None, :, :]) ** 2).sum(-1)
        free = np.all(d2 >= self.R[None, :] ** 2, axis=1)
        d, _ = self.tree.query(x)
        return np.where(free, 0.0, d)


def circle_of_spheres(ci, Ri, cj, Rj):
    """Intersection circle of two spheres: centre, unit axis, radius (closed form)."""
    d = cj - ci
    D = np.linalg.norm(d)
    u = d / D
    a = (D * D + Ri * Ri - Rj * Rj) / (2.0 * D)
    return ci + a * u, u, math.sqrt(max(Ri * Ri - a * a, 0.0))


def trilaterate(c, R):
    """The two points at distance R[k] from c[k], k = 0..2 (closed form)."""
    ex = (c[1] - c[0]) / np.linalg.norm(c[1] - c[0])
    i = ex @ (c[2] - c[0])
    ey = c[2] - c[0] - i * ex
    ey /= np.linalg.norm(ey)
    ez = np.cross(ex, ey)
    d = np.linalg.norm(c[1] - c[0])
    j = ey @ (c[2] - c[0])
    x = (R[0] ** 2 - R[1] ** 2 + d * d) / (2 * d)
    y = (R[0] ** 2 - R[2] ** 2 + i * i + j * j) / (2 * j) - i * x / j
    z = math.sqrt(max(R[0] ** 2 - x * x - y * y, 0.0))
    base = c[0] + x * ex + y * ey
    return base + z * ez, base - z * ez


def patch_offset(xyz, rad, rp, p, kind, ids):
    """|distance from p to the patch (kind, ids) - its radius|, by closed forms:
    0 the van der Waals sphere of ids[0], 1 the torus of radius r_p around the
    intersection circle of the pair's expanded spheres, 2 the probe sphere at
    the nearer-fitting of the triple's two meeting points (inf for a bad kind)."""
    R = np.asarray(rad) + rp
    if kind == 0:
        return abs(np.linalg.norm(p - xyz[ids[0]]) - rad[ids[0]])
    if kind == 1:
        o, u, rho = circle_of_spheres(xyz[ids[0]], R[ids[0]], xyz[ids[1]], R[ids[1]])
        w = p - o
        z = w @ u
        return abs(math.hypot(math.sqrt(max(w @ w - z * z, 0.0)) - rho, z) - rp)
    if kind == 2:
        q1, q2 = trilaterate(xyz[list(ids[:3])], R[list(ids[:3])])
        return min(abs(np.linalg.norm(p - q1) - rp), abs(np.linalg.norm(p - q2) - rp))
    return math.inf

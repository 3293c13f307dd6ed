"""End-to-end pins of the oracle discretisation (Sections 3.1-3.4, 4) against
closed-form solutions: the Mie series for a sound-soft sphere and an exterior
field manufactured by an interior point source."""
import numpy as np
import pytest

import workloads as wl
from oracle import exact
from oracle import nystrom as ny


def _solve(surface, Np, Mt, k, op, g, ggq):
    N = 16 * Np * Mt
    A = ny.operator_rows(surface, Np, Mt, k, ggq[0], ggq[1], np.arange(N), op=op)
    return np.linalg.solve(A, g)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("Np,Mt,op,tol", [(2, 16, "S", 1e-8), (3, 16, "CFIE", 1e-7)])
def test_sphere_plane_wave_matches_mie(ggq, Np, Mt, op, tol):
    k, d = 1.0, [0.0, 0.0, 1.0]
    surf = wl.sphere()
    phi = _solve(surf, Np, Mt, k, op, ny.plane_wave_rhs(surf, Np, Mt, k, d), ggq)
    pts = wl.exterior_points(10, 3.0)
    assert _rel(ny.field(surf, Np, Mt, k, phi, pts, rep=op), exact.mie_sound_soft(k, pts, d)) <= tol
    dirs = wl.Stream(0, 9).directions(8)
    assert _rel(ny.far_field(surf, Np, Mt, k, phi, dirs, rep=op), exact.mie_far_field(k, dirs, d)) <= tol


def test_ellipsoid_point_source_manufactured(ggq):
    surf, Np, Mt, k, src = wl.ellipsoid(1.0, 0.8, 0.6), 3, 24, 2.0, [0.1, 0.1, -0.05]
    phi = _solve(surf, Np, Mt, k, "CFIE", ny.point_source_rhs(surf, Np, Mt, k, src), ggq)
    pts = wl.exterior_points(10, 3.0)
    assert _rel(ny.field(surf, Np, Mt, k, phi, pts, rep="CFIE"), exact.point_source(k, pts, src)) <= 1e-7


def test_mie_series_is_the_exterior_solution():
    # the closed form itself: u^s = -u^i on the unit sphere
    k, d = 3.0, np.array([0.3, -0.2, 0.9]) / np.linalg.norm([0.3, -0.2, 0.9])
    pts = wl.exterior_points(20, 1.0)
    assert np.max(np.abs(exact.mie_sound_soft(k, pts, d) + np.exp(1j * k * pts @ d))) <= 1e-12

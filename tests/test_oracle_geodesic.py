"""Pins for the oracle's geodesic ray launching (Sec. II-A.1, Fig. 1).

Each check comes from geometry, not from the oracle's own formula: the
count of a class-I subdivision, icosahedral symmetry, the convex hull of the
directions (Qhull) for the sub-triangle edges that define alpha.
"""
import numpy as np
import pytest
from scipy.spatial import ConvexHull

import oracle

PHI = (1 + 5 ** 0.5) / 2


@pytest.mark.parametrize("N", [1, 2, 3, 7, 20])
def test_count_and_unit_norm(N):
    d = oracle.geodesic_dirs(N)
    assert d.shape == (10 * N * N + 2, 3)
    assert np.abs(np.linalg.norm(d, axis=1) - 1).max() < 1e-15
    # icosahedral symmetry: the directions sum to zero
    assert np.abs(d.sum(axis=0)).max() < 1e-11


@pytest.mark.parametrize("N", [3, 9])
def test_no_duplicates(N):
    d = oracle.geodesic_dirs(N)
    g = d @ d.T
    np.fill_diagonal(g, -2)
    assert g.max() < 1 - 1e-6


def _rot(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


@pytest.mark.parametrize("N", [1, 4, 6])
def test_icosahedral_rotation_invariance(N):
    d = oracle.geodesic_dirs(N)
    rots = [
        _rot([0, 1, PHI], 2 * np.pi / 5),                    # through a vertex
        _rot(np.array([0, 1, PHI]) + [0, -1, PHI] + [PHI, 0, 1], 2 * np.pi / 3),  # face centre
        _rot([0, 0, 1], np.pi),                              # through an edge midpoint
    ]
    for R in rots:
        e = d @ R.T
        # every rotated direction coincides with one of the originals
        best = (e @ d.T).max(axis=1)
        assert best.min() > 1 - 1e-12


@pytest.mark.parametrize("N", [2, 3, 5, 8, 13])
def test_alpha_equals_max_convex_hull_edge_angle(N):
    d = oracle.geodesic_dirs(N)
    h = ConvexHull(d)
    assert len(h.simplices) == 20 * N * N
    e = set()
    for s in h.simplices:
        for a, b in ((s[0], s[1]), (s[1], s[2]), (s[0], s[2])):
            e.add((min(a, b), max(a, b)))
    e = np.array(sorted(e))
    a, b = d[e[:, 0]], d[e[:, 1]]
    ang = np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.einsum("ij,ij->i", a, b))
    assert abs(ang.max() - oracle.alpha(N)) < 1e-14


def test_alpha_n1_is_icosahedron_edge_angle():
    # the angle subtended by an icosahedron edge: arctan(2) = 63.43 degrees
    assert abs(oracle.alpha(1) - np.arctan(2.0)) < 1e-15


@pytest.mark.parametrize("N", [50, 100])
def test_alpha_matches_literature_scale(N):
    # about 69 degrees / N for geodesic launching grids; within 20%
    a = np.degrees(oracle.alpha(N)) * N
    assert abs(a / 69.0 - 1) < 0.2

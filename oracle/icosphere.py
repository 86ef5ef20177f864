"""Far-field direction grid: a level-L subdivided icosahedron on the unit
sphere (10 * 4^L + 2 vertices; 2562 at L = 4).  Each triangle is split into
four by its edge midpoints, which are pushed out to the sphere.  A vertex's
weight is one third of the summed spherical areas of the triangles touching
it, so the weights add to 4 pi.  The paper does not fix a far-field
quadrature (the CL far field is integrated over the full solid angle,
Eq. 42); this grid is the reading adopted by both implementations.
"""
from __future__ import annotations

import numpy as np


def _base():
    t = (1.0 + np.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1)[:, None]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    return [tuple(x) for x in v], f


def icosphere(level: int = 4):
    verts, faces = _base()
    for _ in range(level):
        cache = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                a = np.array(verts[i])
                b = np.array(verts[j])
                m = a + b
                verts.append(tuple(m / np.linalg.norm(m)))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    F = np.array(faces)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    # spherical triangle area (solid angle), Van Oosterom & Strackee (1983)
    num = np.abs(np.einsum("ij,ij->i", a, np.cross(b, c)))
    den = 1.0 + np.einsum("ij,ij->i", a, b) + np.einsum("ij,ij->i", b, c) + np.einsum("ij,ij->i", c, a)
    omega = 2.0 * np.arctan2(num, den)
    w = np.zeros(len(V))
    for col in range(3):
        np.add.at(w, F[:, col], omega / 3.0)
    return V, w

"""Triangle mesh of the SES from the grid labels and the edge intersections
(cube by cube, in the manner of marching cubes).  TEST INFRASTRUCTURE ONLY:
called by the tests; the GPU library never uses it and shares no code with it.

The paper defines the surface through the labels and the edge intersections
(Eq. 2-4); a mesh of it is the next item of the build (reading M1, below).
Plain numpy and Python loops, written for checking by eye.

Reading M1 (the cube rule).  Corner i of a grid cube sits at offset
((i >> 2) & 1, (i >> 1) & 1, i & 1) from its lower corner (axis 0 first, the
grid's C order).  Cube edge 4 a + j runs along axis a from the j-th corner (in
increasing corner number) whose axis-a offset is 0.  An edge is cut when its
two corner labels differ; its surface point is the edge intersection.  On each
cube face the cut edges pair up into segments: two cut edges make one segment;
four (inside corners on a diagonal) make two, each joining the two edges at
one inside corner (the inside corners are kept apart).  The rule depends only
on the face's four labels, so two cubes sharing a face make the same
segments and the mesh is closed.  Every cut edge lies on two faces, so the
segments form loops; each loop, started at its smallest edge number, is
oriented so that its Newell normal (from the edge midpoints) points from the
inside corner to the outside corner of its edges on the whole, and is cut
into a fan of triangles (v0, v_i, v_i+1).  Loops are taken in the order of
their smallest edge number.
"""
from __future__ import annotations

import numpy as np


def _corner(i):
    return ((i >> 2) & 1, (i >> 1) & 1, i & 1)


def _edges():
    """Cube edges: list of (axis, lower corner, upper corner)."""
    out = []
    for a in range(3):
        lows = [i for i in range(8) if _corner(i)[a] == 0]
        for c in lows:
            out.append((a, c, c | (1 << (2 - a))))
    return out


EDGES = _edges()


def _faces():
    """Cube faces: list of the four edge numbers lying in each face."""
    out = []
    for a in range(3):
        for side in (0, 1):
            out.append([e for e, (b, lo, hi) in enumerate(EDGES)
                        if b != a and _corner(lo)[a] == side and _corner(hi)[a] == side])
    return out


FACES = _faces()


def case_triangles(case: int):
    """Triangles (three cube-edge numbers each) of the cube whose corner i is
    inside iff bit i of `case` is set."""
    inside = [(case >> i) & 1 for i in range(8)]
    cut = [inside[lo] != inside[hi] for (_, lo, hi) in EDGES]
    # segments on the faces
    segs = []
    for fe in FACES:
        ce = [e for e in fe if cut[e]]
        if len(ce) == 2:
            segs.append((ce[0], ce[1]))
        elif len(ce) == 4:
            corners = sorted({c for e in fe for c in EDGES[e][1:]})
            for c in corners:
                if inside[c]:
                    at = [e for e in fe if c in EDGES[e][1:]]
                    segs.append((at[0], at[1]))
    nbr = {e: [] for e in range(12) if cut[e]}
    for s0, s1 in segs:
        nbr[s0].append(s1)
        nbr[s1].append(s0)
    for e, v in nbr.items():
        assert len(v) == 2, (case, e, v)
    # loops, from the smallest unvisited edge
    seen = set()
    tris = []
    for start in sorted(nbr):
        if start in seen:
            continue
        loop = [start]
        seen.add(start)
        prev, cur = None, start
        nxt = min(nbr[start])
        while nxt != start:
            loop.append(nxt)
            seen.add(nxt)
            a, b = nbr[nxt]
            prev, cur, nxt = cur, nxt, (b if a == cur else a)
        # orientation: Newell normal of the midpoints against inside -> outside
        mid = [0.5 * (np.array(_corner(EDGES[e][1]), float) + np.array(_corner(EDGES[e][2]), float)) for e in loop]
        nrm = np.zeros(3)
        for k in range(len(loop)):
            p, q = mid[k], mid[(k + 1) % len(loop)]
            nrm += np.array([(p[1] - q[1]) * (p[2] + q[2]), (p[2] - q[2]) * (p[0] + q[0]),
                             (p[0] - q[0]) * (p[1] + q[1])])
        score = 0.0
        for e in loop:
            _, lo, hi = EDGES[e]
            ci, co = (lo, hi) if inside[lo] else (hi, lo)
            score += float(np.dot(np.array(_corner(co), float) - np.array(_corner(ci), float), nrm))
        assert score != 0.0, (case, loop)
        if score < 0.0:
            loop = [loop[0]] + loop[1:][::-1]
        for k in range(1, len(loop) - 1):
            tris.append((loop[0], loop[k], loop[k + 1]))
    return tris


TABLE = [case_triangles(c) for c in range(256)]


def mesh(labels: np.ndarray, lo, h: float, idx, tau):
    """Mesh of a whole-grid result: (keys int64 (n, 3), xyz float64 (n, 3, 3)).
    A vertex's key is 3 * (lower point of its edge) + axis; triangles come
    cube by cube in C order of the lower corner, then in table order."""
    dims = labels.shape
    where = {}
    for a in range(3):
        for i, t in zip(np.asarray(idx[a]).tolist(), np.asarray(tau[a]).tolist()):
            where[3 * i + a] = t
    keys, xyz = [], []
    lo = np.asarray(lo, float)
    for i in range(dims[0] - 1):
        for j in range(dims[1] - 1):
            for k in range(dims[2] - 1):
                case = 0
                for c in range(8):
                    o = _corner(c)
                    if labels[i + o[0], j + o[1], k + o[2]]:
                        case |= 1 << c
                for tri in TABLE[case]:
                    kt, pt = [], []
                    for e in tri:
                        a, c, _ = EDGES[e]
                        o = _corner(c)
                        g = (i + o[0], j + o[1], k + o[2])
                        p = (g[0] * dims[1] + g[1]) * dims[2] + g[2]
                        key = 3 * p + a
                        pos = lo + h * np.array(g, float)
                        pos[a] += where[key] * h
                        kt.append(key)
                        pt.append(pos)
                    keys.append(kt)
                    xyz.append(pt)
    return np.array(keys, np.int64).reshape(-1, 3), np.array(xyz, np.float64).reshape(-1, 3, 3)

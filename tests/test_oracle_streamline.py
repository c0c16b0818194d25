"""Pins of the oracle's PL streamline trace (Sec. 3.2: the loop is traced back from the first point
reached, against the gradient of the arrival time), no GPU.

  * On a plane, a field that is linear in position is linear on every face whatever the
    triangulation, so its steepest-descent path is a straight line along -grad: every point of the
    trace away from the clamped sources lies on that line (to rounding), on a jittered
    triangulation whose faces the line crosses at arbitrary points.
  * A valley field |x| + y with the valley on a mesh line: the trace runs diagonally into the valley
    and then along the valley's edges, every later point on the valley's line.
  * A cut edge is never crossed; a start with no descent fails; a start on a source ends at once.
  * In the tunnel and refinement passes: the streamline closes, every segment but the closure lies
    in one face whose edges are not cut, its points lie on the surface's edges, and on the torus the
    tunnel streamline winds once around the major circle while the refined streamline winds once
    around the minor circle.
  * The fractional arrival time lies in (T - 1, T] for the integer arrival step T.
"""
import numpy as np
import pytest

import meshgen
import oracle

OK = 0


def box(n: int, jitter: float = 0.0, seed: int = 0, keep_col=None):
    """Closed surface of the cube [0, n]^3 with an n x n grid per side, two triangles per cell.
    Interior vertices of the top side (z = n) are moved within that plane by up to jitter cells;
    vertices on column keep_col of the top side keep their x."""
    key, X = {}, []

    def vid(p):
        if p not in key:
            key[p] = len(X)
            X.append(p)
        return key[p]

    F = []
    for axis in range(3):
        for side in (0, n):
            for i in range(n):
                for j in range(n):
                    def pt(a, b):
                        q = [0, 0, 0]
                        q[axis] = side
                        q[(axis + 1) % 3] = a
                        q[(axis + 2) % 3] = b
                        return vid(tuple(q))
                    a, b, c, d = pt(i, j), pt(i + 1, j), pt(i + 1, j + 1), pt(i, j + 1)
                    tris = [(a, b, c), (a, c, d)] if (i + j) % 2 == 0 else [(a, b, d), (b, c, d)]
                    for t in tris:
                        # orient outward: normal . axis direction has the sign of the side
                        P = np.array([X[t[0]], X[t[1]], X[t[2]]], float)
                        nrm = np.cross(P[1] - P[0], P[2] - P[0])
                        out = 1.0 if side == n else -1.0
                        F.append(t if nrm[axis] * out > 0 else (t[0], t[2], t[1]))
    X = np.array(X, float)
    top = X[:, 2] == n
    if jitter > 0:
        rng = np.random.default_rng(seed)
        inner = top & (X[:, 0] > 0) & (X[:, 0] < n) & (X[:, 1] > 0) & (X[:, 1] < n)
        dx = rng.uniform(-jitter, jitter, (len(X), 2))
        if keep_col is not None:
            dx[X[:, 0] == keep_col, 0] = 0.0
        X[inner, :2] += dx[inner]
    return meshgen.Mesh(X, np.array(F, np.int32), f"box{n}"), top


def on_line(P, p0, d):
    d = d / np.linalg.norm(d)
    r = P - p0
    return np.linalg.norm(r - np.outer(r @ d, d), axis=1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_linear_field_gives_a_straight_line(seed):
    n = 24
    m, top = box(n, jitter=0.3, seed=seed)
    g = np.array([0.37, 1.0, 0.0])
    lin = (m.X - np.array([0.0, 3.0, n])) @ g
    tf = np.where(top, np.maximum(lin, 0.0), -1.0)
    start = int(np.argmin(np.where(top, np.abs(m.X[:, 0] - 6.0) + np.abs(m.X[:, 1] - 20.0), 1e9)))
    st, P, end = oracle.trace_streamline(m, tf, start)
    assert st == OK and tf[end] == 0.0
    assert np.array_equal(P[0], m.X[start])
    far = (P - [0.0, 3.0, n]) @ g > 2.5  # away from the faces that touch a clamped vertex
    assert far.sum() >= 10
    d = on_line(P[far], m.X[start], -g)
    assert d.max() < 1e-11, d.max()
    # the line is crossed face by face: interior points on edges, tf decreasing
    tl = (P - [0.0, 3.0, n]) @ g
    assert (np.diff(tl[far]) < 0).all()


def test_valley_runs_along_its_edges():
    n = 24
    m, top = box(n, jitter=0.25, seed=5, keep_col=12)
    x, y = m.X[:, 0] - 12.0, m.X[:, 1] - 2.0
    tf = np.where(top, np.maximum(np.abs(x) + y, 0.0), -1.0)
    start = int(np.argmin(np.where(top, np.abs(m.X[:, 0] - 5.0) + np.abs(m.X[:, 1] - 20.0), 1e9)))
    st, P, end = oracle.trace_streamline(m, tf, start)
    assert st == OK and tf[end] == 0.0
    hit = np.flatnonzero(np.abs(P[:, 0] - 12.0) < 1e-12)
    assert len(hit) > 5
    k = hit[0]
    away = P[:, 1] - 2.0 > 2.0  # away from the faces that touch a clamped vertex
    assert (np.abs(P[k:, 0] - 12.0)[away[k:]] < 1e-12).all()
    # before the valley: the straight line of the left half's field, direction (1, -1)
    d = on_line(P[:k], m.X[start], np.array([1.0, -1.0, 0.0]))
    assert d.max() < 1e-11
    assert np.all(np.diff(P[k:, 1]) <= 0)


def test_cut_edges_are_not_crossed_and_failures():
    n = 16
    m, top = box(n)
    lin = m.X[:, 1] - 2.0 + 0.3 * m.X[:, 0]
    tf = np.where(top, np.maximum(lin, 0.0), -1.0)
    start = int(np.flatnonzero(top & (m.X[:, 0] == 8) & (m.X[:, 1] == 12))[0])
    # a wall of cut edges across the top between y = 6 and y = 7, spanning every column
    cut = []
    for f in m.F:
        for k in range(3):
            a, b = int(f[k]), int(f[(k + 1) % 3])
            if top[a] and top[b] and {m.X[a, 1], m.X[b, 1]} == {6.0, 7.0}:
                cut.append((a, b))
    st, P, end = oracle.trace_streamline(m, tf, start, cut_edges=np.array(cut))
    assert st != OK  # the wall closes every way down
    assert (P[:, 1] >= 7.0 - 1e-12).all()
    st, P, end = oracle.trace_streamline(m, tf, start)
    assert st == OK and P[-1, 1] <= 2.0 + 1e-12
    src = int(np.flatnonzero(top & (tf == 0.0))[0])
    st, P, end = oracle.trace_streamline(m, tf, src)
    assert st == OK and end == src and len(P) == 1
    # a local minimum that is no source: no descent left
    bowl = np.where(top, 1.0 + np.hypot(m.X[:, 0] - 8, m.X[:, 1] - 8), -1.0)
    st, _, _ = oracle.trace_streamline(m, bowl, start)
    assert st != OK


def _face_of_segment(m, cut_slots, p, q):
    """The faces with both points on their boundary; True if one of them has no cut edge."""
    X = m.X
    found = False
    for f, (a, b, c) in enumerate(m.F):
        tri = X[[a, b, c]]
        ok = True
        for r in (p, q):
            on = False
            for (u, w) in ((0, 1), (1, 2), (2, 0)):
                e = tri[w] - tri[u]
                t = np.clip((r - tri[u]) @ e / (e @ e), 0, 1)
                if np.linalg.norm(tri[u] + t * e - r) < 1e-9:
                    on = True
                    break
            ok &= on
        if ok:
            found = True
            if not any((min(x, y), max(x, y)) in cut_slots for x, y in ((a, b), (b, c), (c, a))):
                return True
    return False if found else None


def _winding(P, fn):
    a = fn(P)
    d = np.diff(np.concatenate([a, a[:1]]))
    d = (d + np.pi) % (2 * np.pi) - np.pi
    return int(np.rint(d.sum() / (2 * np.pi)))


def test_torus_streamlines_wind_and_stay_in_uncut_faces():
    R0, r0 = 2.0, 0.7
    m = meshgen.torus(24, 12, R0, r0)
    res = oracle.detect(m, meshgen.seed_vertex(0, m.nv), record_steps=1)
    assert res.status == OK and len(res.handles) == 1
    h, t, rf = res.handles[0], res.tunnels[0], res.refined[0]
    assert t.stream_status == OK and rf.stream_status == OK
    major = lambda P: np.arctan2(P[:, 1], P[:, 0])
    minor = lambda P: np.arctan2(P[:, 2], np.hypot(P[:, 0], P[:, 1]) - R0)
    assert abs(_winding(t.stream, major)) == 1
    assert abs(_winding(rf.stream, minor)) == 1 and _winding(rf.stream, major) == 0
    cut = {(min(a, b), max(a, b)) for a, b in h.edges}
    P = t.stream
    # the trace part: from b* until the first source vertex (a loop-side vertex) is reached
    src = {int(a) for a, _ in h.edges}
    first_src = next(i for i, p in enumerate(P) if any(np.array_equal(p, m.X[s]) for s in src))
    for i in range(first_src):
        assert _face_of_segment(m, cut, P[i], P[i + 1]), i
    L = np.linalg.norm(P - np.roll(P, -1, 0), axis=1).sum()
    assert abs(L - t.stream_length) < 1e-9
    assert np.array_equal(P[0], m.X[t.bstar])


def test_fractional_arrival_brackets_the_step():
    m = meshgen.torus(24, 12)
    res = oracle.detect(m, meshgen.seed_vertex(3, m.nv), record_steps=1)
    for t in res.tunnels:
        T, tf = t.arrival, t.arrival_time
        reached = T > 0
        assert reached.sum() > 10
        assert (tf[T == 0] == 0.0).all() and (tf[T < 0] == -1.0).all()
        assert (tf[reached] > T[reached] - 1).all() and (tf[reached] <= T[reached]).all()
        assert not np.array_equal(tf[reached], T[reached].astype(float))

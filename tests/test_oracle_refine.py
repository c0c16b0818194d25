"""Pins of the oracle's handle-refinement pass (Sec. 3.3) and loop classification (Sec. 3.5), no GPU.

Refinement: the refined handle is a vertex cycle that
  * is a closed primal cycle, not null-homologous, whose cut leaves the surface connected;
  * crosses its tunnel loop an odd number of times -- counted against a push-off of the tunnel
    loop to its LEFT side (the pass starts on the tunnel loop and spreads to the left; its border is
    on the right, so the left push-off is a different edge set from the pass's border);
  * on the grid torus, winds once around the minor circle and not around the major one (the
    meridian class of the handle loop it refines);
  * together with the other refined handles has the GF(2) rank of the handle loops (g where that is
    full), and with the tunnels twice that.
Classification: each loop's offset length change against numpy (unit vertex normals from the
summed face normals, mean edge length over the unique edges), and the sign rule on the handle loops.
"""
import numpy as np
import pytest

import meshgen
import oracle
from topology import Topo, gf2_rank

OK = 0


def left_pushoff(m, cyc):
    """Edges from each vertex of the simple cycle (closed sub-loops erased) to its neighbours met
    clockwise from c_{i+1} to c_{i-1}, i.e. on its left (faces are counter-clockwise)."""
    st, pos = [], {}
    for v in cyc:
        v = int(v)
        if v in pos and pos[v] < len(st) and st[pos[v]] == v:
            del st[pos[v] + 1:]
        else:
            pos[v] = len(st)
            st.append(v)
    on = set(st)
    # the face left of half-edge a->b, as its third vertex
    third = {}
    for f in m.F:
        for k in range(3):
            third[(int(f[k]), int(f[(k + 1) % 3]))] = int(f[(k + 2) % 3])
    out = []
    n = len(st)
    for i, c in enumerate(st):
        prv, nxt = st[i - 1], st[(i + 1) % n]
        u = nxt
        for _ in range(64):
            u = third[(c, u)]  # counter-clockwise from c_{i+1} towards c_{i-1}: the left side
            if u == prv:
                break
            if u not in on:
                out.append((c, u))
    return np.array(out, dtype=np.int64)


def _grid_winding(verts, nu, nv):
    I, J = np.asarray(verts) // nv, np.asarray(verts) % nv
    di = np.diff(np.concatenate([I, I[:1]]))
    dj = np.diff(np.concatenate([J, J[:1]]))
    di = (di + nu // 2) % nu - nu // 2
    dj = (dj + nv // 2) % nv - nv // 2
    return int(di.sum()), int(dj.sum())


def test_torus_refined_handle_is_a_meridian():
    nu, nv = 64, 32
    m = meshgen.torus(nu, nv, 2.0, 0.7)
    r = oracle.detect(m, meshgen.seed_vertex(0, m.nv))
    assert r.status == OK and len(r.refined) == 1 and r.refined[0].status == OK
    wi, wj = _grid_winding(r.refined[0].verts, nu, nv)
    assert wi == 0 and abs(wj) == nv
    # the refined loop is shorter than the tunnel loop it was built from
    L = lambda v: np.linalg.norm(np.roll(m.X[v], -1, axis=0) - m.X[v], axis=1).sum()
    assert L(r.refined[0].verts) < L(r.tunnels[0].verts)


@pytest.mark.parametrize("which,seeds", [("chain2", (0, 1)), ("chain3", (0,)), ("batch44", (2,))])
def test_refined_handles_homology(which, seeds):
    if which == "batch44":
        m, ss = meshgen.batch_problem(44)
        seeds = [ss[k] for k in seeds]
    else:
        m = meshgen.tube_chain(2, 64) if which == "chain2" else meshgen.tube_chain(3, 80)
        seeds = [meshgen.seed_vertex(k, m.nv) for k in seeds]
    topo = Topo(m.F, m.nv)
    for s in seeds:
        r = oracle.detect(m, s)
        g = m.genus()
        assert r.status == OK and len(r.refined) == g
        cr, ct, ch = [], [], []
        for h, t, f in zip(r.handles, r.tunnels, r.refined):
            ch.append(topo.class_dual(topo.crossing_edges(h.edges)))
            assert t.status == OK and f.status == OK
            z = topo.vertex_cycle_edges(f.verts)
            assert topo.is_primal_cycle(z) and not topo.primal_is_null(z) and topo.cut_connected_primal(z)
            zt = topo.vertex_cycle_edges(t.verts)
            x = topo.crossing_edges(left_pushoff(m, t.verts))
            assert topo.is_dual_cycle(x)
            # the left push-off is homologous to the tunnel loop: pairs oddly with the tunnel's handle
            assert int((z & x).sum()) % 2 == 1, "refined handle must cross its tunnel loop an odd number of times"
            assert int((z & x).sum()) % 2 == int(topo.class_primal(z) @ topo.class_dual(x)) % 2
            cr.append(topo.class_primal(z))
            ct.append(topo.class_primal(zt))
        # refinement keeps the rank of the handle loops it starts from: g where theirs is full (a loop
        # kept at a merge can be homologous to a combination of earlier handles: batch mesh 44, seed 2)
        rh = gf2_rank(np.array(ch))
        assert gf2_rank(np.array(cr)) == rh and gf2_rank(np.array(cr + ct)) == 2 * rh
        assert rh == g or (which, s) == ("batch44", 4518)


def _numpy_offset_change(m, pts, nrm, frac, mean_edge):
    d = frac * mean_edge
    q = pts + d * nrm
    L = lambda P: np.linalg.norm(np.roll(P, -1, axis=0) - P, axis=1).sum()
    return L(q) - L(pts)


@pytest.mark.parametrize("which", ["torus", "chain2"])
def test_offset_change_against_numpy(which):
    m = meshgen.torus(64, 32, 2.0, 0.7) if which == "torus" else meshgen.tube_chain(2, 64)
    r = oracle.detect(m, meshgen.seed_vertex(1, m.nv))
    X, F = m.X, m.F.astype(np.int64)
    fn = np.cross(X[F[:, 1]] - X[F[:, 0]], X[F[:, 2]] - X[F[:, 0]])
    vn = np.zeros_like(X)
    for k in range(3):
        np.add.at(vn, F[:, k], fn)
    vn /= np.linalg.norm(vn, axis=1, keepdims=True)
    E = np.unique(np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1), axis=0)
    mean_edge = np.linalg.norm(X[E[:, 0]] - X[E[:, 1]], axis=1).mean()
    assert r.mean_edge == pytest.approx(mean_edge, rel=1e-12)
    for i, (h, t, f) in enumerate(zip(r.handles, r.tunnels, r.refined)):
        s = vn[h.edges[:, 0]] + vn[h.edges[:, 1]]
        s /= np.linalg.norm(s, axis=1, keepdims=True)
        ref = [_numpy_offset_change(m, h.points, s, 0.5, mean_edge),
               _numpy_offset_change(m, X[t.verts], vn[t.verts], 0.5, mean_edge),
               _numpy_offset_change(m, X[f.verts], vn[f.verts], 0.5, mean_edge)]
        assert np.allclose(r.offset_change[i], ref, rtol=1e-10, atol=1e-12), (r.offset_change[i], ref)
        # handle loops around a tube grow when pushed outwards (Sec. 3.5)
        assert r.offset_change[i, 0] > 0 and r.offset_change[i, 2] > 0

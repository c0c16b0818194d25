"""Z2-homology tools for pinning loops on closed oriented triangle meshes (test helper).

Two independent methods:

* tree-cotree generators (Eppstein 2003, cited by the paper in Sec. 1): a primal
  spanning tree T, a dual spanning tree C on the faces avoiding T, and the 2g leftover
  edges X.  Each leftover edge e gives a primal generator cycle gamma_e and a dual
  generator cycle delta_e with gamma_e . delta_f = [e == f].  A primal cycle z has class
  c_e = |z & delta_e| mod 2; a dual cycle (set of crossed edges) has class
  c_e = |cut & gamma_e| mod 2.
* cut 2-colouring: a set of crossed edges is a coboundary (null-homologous) iff the
  components of the graph without those edges can be 2-coloured so that every crossed
  edge joins different colours; dually for a primal cycle on the face graph.
"""
from __future__ import annotations

from collections import deque

import numpy as np


class Topo:
    def __init__(self, F: np.ndarray, nv: int):
        F = np.asarray(F, dtype=np.int64)
        self.F = F
        self.nv = nv
        nf = len(F)
        self.nf = nf
        a = np.concatenate([F[:, 0], F[:, 1], F[:, 2]])
        b = np.concatenate([F[:, 1], F[:, 2], F[:, 0]])
        fid = np.concatenate([np.arange(nf)] * 3)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        key = lo * nv + hi
        uniq, inv = np.unique(key, return_inverse=True)
        self.edges = np.stack([uniq // nv, uniq % nv], axis=1)
        self.ne = len(uniq)
        self.edge_index = {int(k): i for i, k in enumerate(uniq)}
        # faces of each edge
        ef = -np.ones((self.ne, 2), np.int64)
        cnt = np.zeros(self.ne, np.int64)
        for h in range(len(inv)):
            e = inv[h]
            ef[e, cnt[e]] = fid[h]
            cnt[e] += 1
        assert (cnt == 2).all(), "mesh is not closed / edge-manifold"
        self.edge_faces = ef
        self.adj = [[] for _ in range(nv)]
        for i, (u, v) in enumerate(self.edges):
            self.adj[u].append((int(v), i))
            self.adj[v].append((int(u), i))
        self.fadj = [[] for _ in range(nf)]
        for i in range(self.ne):
            f, g = ef[i]
            self.fadj[f].append((int(g), i))
            self.fadj[g].append((int(f), i))
        self._build_generators()

    def eid(self, u: int, v: int) -> int:
        a, b = (u, v) if u < v else (v, u)
        return self.edge_index[a * self.nv + b]

    # ------------------------------------------------------------ tree-cotree
    def _build_generators(self):
        nv, nf, ne = self.nv, self.nf, self.ne
        parent = -np.ones(nv, np.int64)
        pedge = -np.ones(nv, np.int64)
        depth = np.zeros(nv, np.int64)
        in_tree = np.zeros(ne, bool)
        seen = np.zeros(nv, bool)
        seen[0] = True
        q = deque([0])
        while q:
            u = q.popleft()
            for v, e in self.adj[u]:
                if not seen[v]:
                    seen[v] = True
                    parent[v], pedge[v], depth[v] = u, e, depth[u] + 1
                    in_tree[e] = True
                    q.append(v)
        assert seen.all(), "mesh is disconnected"
        fpar = -np.ones(nf, np.int64)
        fpedge = -np.ones(nf, np.int64)
        fdepth = np.zeros(nf, np.int64)
        in_cotree = np.zeros(ne, bool)
        fseen = np.zeros(nf, bool)
        fseen[0] = True
        q = deque([0])
        while q:
            f = q.popleft()
            for g, e in self.fadj[f]:
                if not in_tree[e] and not fseen[g]:
                    fseen[g] = True
                    fpar[g], fpedge[g], fdepth[g] = f, e, fdepth[f] + 1
                    in_cotree[e] = True
                    q.append(g)
        leftover = np.nonzero(~in_tree & ~in_cotree)[0]
        self.leftover = leftover
        self.g2 = len(leftover)

        def tree_path(u, v, par, pe, dep):
            out = []
            while u != v:
                if dep[u] >= dep[v]:
                    out.append(pe[u]); u = par[u]
                else:
                    out.append(pe[v]); v = par[v]
            return out

        self.gamma = np.zeros((self.g2, ne), np.uint8)  # primal generator cycles (edge sets)
        self.delta = np.zeros((self.g2, ne), np.uint8)  # dual generator cycles (crossed edges)
        for k, e in enumerate(leftover):
            u, v = self.edges[e]
            for x in tree_path(int(u), int(v), parent, pedge, depth):
                self.gamma[k, x] ^= 1
            self.gamma[k, e] ^= 1
            f, g = self.edge_faces[e]
            for x in tree_path(int(f), int(g), fpar, fpedge, fdepth):
                self.delta[k, x] ^= 1
            self.delta[k, e] ^= 1

    # ------------------------------------------------------------ loops -> sets
    def vertex_cycle_edges(self, verts) -> np.ndarray:
        z = np.zeros(self.ne, np.uint8)
        n = len(verts)
        for i in range(n):
            u, v = int(verts[i]), int(verts[(i + 1) % n])
            if u != v:
                z[self.eid(u, v)] ^= 1
        return z

    def crossing_edges(self, pairs) -> np.ndarray:
        x = np.zeros(self.ne, np.uint8)
        for a, b in pairs:
            x[self.eid(int(a), int(b))] = 1
        return x

    def class_primal(self, z: np.ndarray) -> np.ndarray:
        return (self.delta.astype(np.int64) @ z.astype(np.int64)) % 2

    def class_dual(self, x: np.ndarray) -> np.ndarray:
        return (self.gamma.astype(np.int64) @ x.astype(np.int64)) % 2

    def is_primal_cycle(self, z: np.ndarray) -> bool:
        deg = np.zeros(self.nv, np.int64)
        for e in np.nonzero(z)[0]:
            deg[self.edges[e, 0]] += 1
            deg[self.edges[e, 1]] += 1
        return bool((deg % 2 == 0).all())

    def is_dual_cycle(self, x: np.ndarray) -> bool:
        deg = np.zeros(self.nf, np.int64)
        for e in np.nonzero(x)[0]:
            deg[self.edge_faces[e, 0]] += 1
            deg[self.edge_faces[e, 1]] += 1
        return bool((deg % 2 == 0).all())

    # ------------------------------------------------------------ 2-colouring
    @staticmethod
    def _two_colour(n, adj, cut) -> bool:
        col = -np.ones(n, np.int64)
        for s in range(n):
            if col[s] >= 0:
                continue
            col[s] = 0
            q = deque([s])
            while q:
                u = q.popleft()
                for v, e in adj[u]:
                    want = col[u] ^ int(cut[e])
                    if col[v] < 0:
                        col[v] = want
                        q.append(v)
                    elif col[v] != want:
                        return False
        return True

    def dual_is_null(self, x: np.ndarray) -> bool:
        """crossed-edge set x bounds a vertex region (is a coboundary)"""
        return self._two_colour(self.nv, self.adj, x)

    def primal_is_null(self, z: np.ndarray) -> bool:
        """edge set z bounds a face region"""
        return self._two_colour(self.nf, self.fadj, z)

    def cut_connected_dual(self, x: np.ndarray) -> bool:
        """vertices stay connected after removing the crossed edges"""
        seen = np.zeros(self.nv, bool)
        seen[0] = True
        q = deque([0])
        while q:
            u = q.popleft()
            for v, e in self.adj[u]:
                if not x[e] and not seen[v]:
                    seen[v] = True
                    q.append(v)
        return bool(seen.all())

    def cut_connected_primal(self, z: np.ndarray) -> bool:
        """faces stay connected after removing the duals of the cycle's edges"""
        seen = np.zeros(self.nf, bool)
        seen[0] = True
        q = deque([0])
        while q:
            f = q.popleft()
            for g, e in self.fadj[f]:
                if not z[e] and not seen[g]:
                    seen[g] = True
                    q.append(g)
        return bool(seen.all())


def gf2_rank(rows: np.ndarray) -> int:
    M = (np.asarray(rows, dtype=np.uint8) % 2).copy()
    r = 0
    nrow, ncol = M.shape if M.ndim == 2 else (0, 0)
    for c in range(ncol):
        piv = None
        for i in range(r, nrow):
            if M[i, c]:
                piv = i
                break
        if piv is None:
            continue
        M[[r, piv]] = M[[piv, r]]
        for i in range(nrow):
            if i != r and M[i, c]:
                M[i] ^= M[r]
        r += 1
        if r == nrow:
            break
    return r

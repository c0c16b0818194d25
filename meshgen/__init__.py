"""Seeded synthetic meshes (closed, oriented, manifold) for tests and benchmarks.

Input generation only: nothing here computes any part of the loop-shrinking
method.  Both the CPU oracle and the CUDA library take these meshes as input.

The five workloads stand in for the paper's scanned models (Sec. 6, Table 1:
0.003-10 M faces, genus 1-335), which are not available:

1. torus        parametric 64 x 32 grid, R = 2.0, r = 0.7 (4096 faces), 1 seed
2. tube_chain   smooth union (blend 0.15) of 8 z-axis tori (R = 1, r = 0.35) spaced
                1.6 along x, polygonised, normal jitter sigma = 0.1 mean edge, 4 seeds
3. schwarz_p    cos x + cos y + cos z < 0 clipped to 4^3 periods, 1 seed
4. batch        256 meshes (tori and 2..20-torus chains), faces log-uniform in
                [2k, 200k], 4 seeds each
5. gyroid       gyroid solid clipped to 8^3 periods, jitter 0.05 mean edge, 1 seed

Polygonisation is marching tetrahedra on the Kuhn split of the sample grid (no
marching-cubes case table); it yields roughly twice the faces of marching cubes at
the same grid, so grid sizes are chosen for the stated face counts.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_meshgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator with gcc (plain C, no architecture flags)."""
    src = os.path.join(_HERE, "meshgen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fvisibility=hidden",
                               "-o", _SO + ".tmp", src, "-lm"])
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.POINTER
            lib.mg_seed_vertex.restype = ctypes.c_int32
            lib.mg_seed_vertex.argtypes = [ctypes.c_uint64, ctypes.c_int64]
            lib.mg_torus.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p]
            lib.mg_implicit.restype = ctypes.c_void_p
            lib.mg_implicit.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_int,
                                        P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_int64)]
            lib.mg_mesh_nv.restype = ctypes.c_int64
            lib.mg_mesh_nv.argtypes = [ctypes.c_void_p]
            lib.mg_mesh_nf.restype = ctypes.c_int64
            lib.mg_mesh_nf.argtypes = [ctypes.c_void_p]
            lib.mg_mesh_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.mg_mesh_free.argtypes = [ctypes.c_void_p]
            lib.mg_jitter.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_double, ctypes.c_uint64]
            _lib = lib
    return _lib


class Mesh:
    """Closed triangle mesh: X float64 [V, 3], F int32 [F, 3] (CCW, outward normals)."""

    def __init__(self, X: np.ndarray, F: np.ndarray, name: str = ""):
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.F = np.ascontiguousarray(F, dtype=np.int32)
        self.name = name

    @property
    def nv(self) -> int:
        return int(self.X.shape[0])

    @property
    def nf(self) -> int:
        return int(self.F.shape[0])

    def euler(self) -> int:
        e = np.sort(np.concatenate([self.F[:, [0, 1]], self.F[:, [1, 2]], self.F[:, [2, 0]]]), axis=1)
        ne = len(np.unique(e[:, 0].astype(np.int64) * self.nv + e[:, 1]))
        return self.nv - ne + self.nf

    def genus(self) -> int:
        return (2 - self.euler()) // 2


def seed_vertex(seed: int, nv: int) -> int:
    """Seed vertex floor(U * nv), U the first SplitMix64 uniform of stream `seed`."""
    return int(_load().mg_seed_vertex(ctypes.c_uint64(seed), nv))


def torus(nu: int = 64, nv: int = 32, R: float = 2.0, r: float = 0.7) -> Mesh:
    lib = _load()
    X = np.empty((nu * nv, 3), np.float64)
    F = np.empty((2 * nu * nv, 3), np.int32)
    lib.mg_torus(nu, nv, R, r, X.ctypes.data, F.ctypes.data)
    return Mesh(X, F, f"torus{nu}x{nv}")


def _implicit(kind: int, count: int, params, lo, hi, n, name: str) -> Mesh:
    lib = _load()
    if isinstance(n, int):
        n = (n, n, n)
    na = (ctypes.c_int64 * 3)(*[int(x) for x in n])
    pa = (ctypes.c_double * 8)(*([float(p) for p in params] + [0.0] * (8 - len(params))))
    loa = (ctypes.c_double * 3)(*lo)
    hia = (ctypes.c_double * 3)(*hi)
    h = lib.mg_implicit(kind, count, pa, len(params), loa, hia, na)
    nvv, nff = lib.mg_mesh_nv(h), lib.mg_mesh_nf(h)
    X = np.empty((nvv, 3), np.float64)
    F = np.empty((nff, 3), np.int32)
    lib.mg_mesh_copy(h, X.ctypes.data, F.ctypes.data)
    lib.mg_mesh_free(h)
    return Mesh(X, F, name)


def jitter(m: Mesh, sigma_rel: float, seed: int) -> Mesh:
    """Move each vertex along its area-weighted normal by N(0, (sigma_rel * mean edge)^2)."""
    X = m.X.copy()
    _load().mg_jitter(X.ctypes.data, m.nv, m.F.ctypes.data, m.nf, float(sigma_rel), ctypes.c_uint64(seed))
    return Mesh(X, m.F, m.name)


def tube_chain(n_tori: int = 8, grid: int = 256, R: float = 1.0, r: float = 0.35, spacing: float = 1.6,
               blend: float = 0.15) -> Mesh:
    pad = r + blend + 0.1
    lo = (-R - pad, -R - pad, -r - pad)
    hi = (spacing * (n_tori - 1) + R + pad, R + pad, r + pad)
    # grid = samples along the longest axis; other axes share the spacing
    L = hi[0] - lo[0]
    h = L / (grid - 1)
    ny = int(math.ceil((hi[1] - lo[1]) / h)) + 1
    nz = int(math.ceil((hi[2] - lo[2]) / h)) + 1
    hi2 = (lo[0] + h * (grid - 1), lo[1] + h * (ny - 1), lo[2] + h * (nz - 1))
    return _implicit(0, n_tori, [R, r, spacing, blend], lo, hi2, (grid, ny, nz), f"tube_chain{n_tori}_g{grid}")


def schwarz_p(periods: int = 4, grid: int = 512) -> Mesh:
    span = 2 * math.pi * periods
    eps = 1e-3
    box_lo, box_hi = (eps, eps, eps), (span - eps, span - eps, span - eps)
    h = span / (grid - 3)
    lo = (-h, -h, -h)
    hi = (span + h, span + h, span + h)
    return _implicit(1, 0, list(box_lo) + list(box_hi), lo, hi, grid, f"schwarz_p{periods}_g{grid}")


def gyroid(periods: int = 8, grid: int = 1024) -> Mesh:
    span = 2 * math.pi * periods
    eps = 1e-3
    box_lo, box_hi = (eps, eps, eps), (span - eps, span - eps, span - eps)
    h = span / (grid - 3)
    lo = (-h, -h, -h)
    hi = (span + h, span + h, span + h)
    return _implicit(2, 0, list(box_lo) + list(box_hi), lo, hi, grid, f"gyroid{periods}_g{grid}")


def capsules(arms: int = 5, grid: int = 96, length: float = 1.0, radius: float = 0.18, blend: float = 0.08) -> Mesh:
    """Genus-0 branching solid (arms from a common centre)."""
    pad = radius + blend + 0.1
    ext = length + pad
    return _implicit(3, arms, [length, radius, blend], (-ext,) * 3, (ext,) * 3, grid, f"capsules{arms}")


def sphere(grid: int = 48, radius: float = 1.0) -> Mesh:
    ext = radius + 0.2
    return _implicit(4, 0, [radius], (-ext,) * 3, (ext,) * 3, grid, "sphere")


# --------------------------------------------------------------------- workloads
def _batch_specs(scale: float = 1.0):
    """Shape of every mesh of the batch workload: (genus type, target faces), drawn in order from
    one PCG64 stream (shape mix only; the meshes' own noise uses SplitMix64)."""
    st = np.random.Generator(np.random.PCG64(4))
    out = []
    for _ in range(256):
        target = math.exp(st.uniform(math.log(2000), math.log(200000))) * scale
        gtype = int(st.integers(1, 21))
        out.append((gtype, target))
    return out


def batch_problem(i: int, scale: float = 1.0):
    """Mesh i of the batch workload (a torus for genus type 1, else a tube chain of that many
    tori) with its 4 seed vertices."""
    gtype, target = _batch_specs(scale)[i]
    if gtype == 1:
        nvv = max(4, int(round(math.sqrt(target / 4))))
        m = torus(2 * nvv, nvv, 2.0, 0.7)
    else:
        # marching tetrahedra give F ~ 7 * area / h^2 (measured 6.2-7.7) with area
        # n * 4 pi^2 R r; the spacing h is capped at r / 2.2 so that every tube is
        # resolved (which raises small targets of long chains to ~75k faces)
        L = 1.6 * (gtype - 1) + 2 * (1.0 + 0.35 + 0.15 + 0.1)
        h = min(0.16, math.sqrt(7.0 * gtype * 4 * math.pi ** 2 * 0.35 / target))
        grid = int(math.ceil(L / h)) + 1
        m = jitter(tube_chain(gtype, grid), 0.1, 100 + i)
    return m, [seed_vertex(4 * i + s, m.nv) for s in range(4)]


def workload(k: int, scale: float = 1.0):
    """Problems of workload k (1..5): list of (Mesh, [seed vertices]).

    `scale` < 1 shrinks the polygonisation grid (faces scale ~ scale^2) for small
    test variants with the same shape and structure.
    """
    if k == 1:
        m = torus(64, 32, 2.0, 0.7)
        return [(m, [seed_vertex(0, m.nv)])]
    if k == 2:
        m = tube_chain(8, max(24, int(round(388 * scale))))
        m = jitter(m, 0.1, 2)
        return [(m, [seed_vertex(s, m.nv) for s in range(4)])]
    if k == 3:
        m = schwarz_p(4, max(24, int(round(240 * scale))))
        return [(m, [seed_vertex(0, m.nv)])]
    if k == 4:
        return [batch_problem(i, scale) for i in range(256)]
    if k == 5:
        m = gyroid(8, max(32, int(round(295 * scale))))
        m = jitter(m, 0.05, 5)
        return [(m, [seed_vertex(0, m.nv)])]
    raise ValueError(k)

"""Thin ctypes binding of the CUDA library (include/vls.h), same names as the C ABI.

Argument marshalling only: every step of the path runs in the library's CUDA kernels.
Loading fails loudly if the library has not been built; there is no other code path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvls.so")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOTMANIFOLD", 3: "ENONORIENTABLE", 4: "EDISCONNECTED",
          5: "EMAXSTEPS", 6: "ESLOTS", 7: "ELAYERS", 8: "ELOOPFAIL", 9: "ETIMEOUT", 10: "ENOMEM",
          11: "ECUDA", 12: "ESTALL", 13: "ETOOLARGE"}
VLS_FP64, VLS_FP32_RECHECK, VLS_BF16_RECHECK = 0, 1, 2


class vls_options(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("e", ctypes.c_double), ("a", ctypes.c_double), ("w", ctypes.c_double),
                ("dt_factor", ctypes.c_double), ("eps0", ctypes.c_double), ("theta_iso", ctypes.c_double),
                ("lbar", ctypes.c_double), ("recheck_margin", ctypes.c_double),
                ("max_steps", ctypes.c_int32), ("max_pass_steps", ctypes.c_int32), ("tunnels", ctypes.c_int32),
                ("keep_state", ctypes.c_int32), ("record_steps", ctypes.c_int32), ("sync_interval", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("host_loop", ctypes.c_int32),
                ("hook_variant", ctypes.c_int32), ("rows_per_warp", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("offset", ctypes.c_double), ("K", ctypes.c_int32),
                ("laplacian", ctypes.c_int32), ("max_passes", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("drift_bound", ctypes.c_double), ("streamlines", ctypes.c_int32)]


class vls_mesh(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("nv", ctypes.c_int64), ("F", ctypes.c_void_p), ("nf", ctypes.c_int64),
                ("device", ctypes.c_int32)]


class vls_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("tunnel_steps", ctypes.c_int32), ("row_updates", ctypes.c_int64),
                ("pass_updates", ctypes.c_int64), ("merges", ctypes.c_int32), ("splits", ctypes.c_int32),
                ("ends", ctypes.c_int32), ("layers", ctypes.c_int32), ("ms_operator", ctypes.c_double),
                ("ms_initial", ctypes.c_double), ("ms_tunnel", ctypes.c_double), ("ms_download", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("ms_update", ctypes.c_double), ("ms_pass_update", ctypes.c_double),
                ("n_update", ctypes.c_int64), ("n_pass_update", ctypes.c_int64), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64), ("rechecks", ctypes.c_int64), ("pass_rechecks", ctypes.c_int64),
                ("mass_resid", ctypes.c_double), ("pass_mass_resid", ctypes.c_double),
                ("refine_updates", ctypes.c_int64), ("refine_steps", ctypes.c_int32), ("ms_refine", ctypes.c_double),
                ("refine_mass_resid", ctypes.c_double), ("mean_edge", ctypes.c_double),
                ("uncertified", ctypes.c_int64), ("pass_uncertified", ctypes.c_int64),
                ("refine_uncertified", ctypes.c_int64)]


EXPORTS = ["vls_default_options", "vls_constants", "vls_create", "vls_destroy", "vls_detect", "vls_detect_batch",
           "vls_result_count", "vls_result_status", "vls_result_genus", "vls_result_stats", "vls_result_num_loops",
           "vls_result_loop", "vls_result_handle", "vls_result_tunnel", "vls_result_refined",
           "vls_result_offset_change", "vls_result_streamline", "vls_result_reeb", "vls_result_state",
           "vls_result_records", "vls_result_kernel_times", "vls_result_free", "vls_status_string",
           "vls_tunnel_pass_noalloc"]

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.vls_default_options.argtypes = [P(vls_options)]
    L.vls_default_options.restype = None
    L.vls_constants.argtypes = [P(vls_options), P(dbl)]
    L.vls_constants.restype = None
    L.vls_create.argtypes = [P(vp), P(vls_options), vp]
    L.vls_create.restype = i32
    L.vls_destroy.argtypes = [vp]
    L.vls_destroy.restype = None
    L.vls_detect.argtypes = [vp, P(vls_mesh), i32, P(vp)]
    L.vls_detect.restype = i32
    L.vls_detect_batch.argtypes = [vp, i32, P(vls_mesh), P(i32), P(i32), P(vp)]
    L.vls_detect_batch.restype = i32
    L.vls_result_count.argtypes = [vp]
    L.vls_result_count.restype = i32
    L.vls_result_status.argtypes = [vp, i32]
    L.vls_result_status.restype = i32
    L.vls_result_genus.argtypes = [vp, i32]
    L.vls_result_genus.restype = i32
    L.vls_result_stats.argtypes = [vp, i32, P(vls_stats)]
    L.vls_result_stats.restype = i32
    L.vls_result_num_loops.argtypes = [vp, i32, i32]
    L.vls_result_num_loops.restype = i32
    L.vls_result_loop.argtypes = [vp, i32, i32, i32, P(P(i32)), P(i64), P(P(dbl)), P(i64)]
    L.vls_result_loop.restype = i32
    L.vls_result_handle.argtypes = [vp, i32, i32, P(P(i32)), P(i64), P(i32), P(dbl)]
    L.vls_result_handle.restype = i32
    L.vls_result_tunnel.argtypes = [vp, i32, i32, P(i32)]
    L.vls_result_tunnel.restype = i32
    L.vls_result_refined.argtypes = [vp, i32, i32, P(i32)]
    L.vls_result_refined.restype = i32
    L.vls_result_offset_change.argtypes = [vp, i32, i32, P(dbl)]
    L.vls_result_offset_change.restype = i32
    L.vls_result_streamline.argtypes = [vp, i32, i32, i32, P(i32), P(P(dbl)), P(i64), P(dbl)]
    L.vls_result_streamline.restype = i32
    L.vls_result_reeb.argtypes = [vp, i32, P(P(i32)), P(P(dbl)), P(i32), P(P(i32)), P(i32)]
    L.vls_result_reeb.restype = i32
    L.vls_result_state.argtypes = [vp, i32, P(P(i32)), P(P(dbl)), P(P(i32)), P(i64)]
    L.vls_result_state.restype = i32
    L.vls_result_records.argtypes = [vp, i32, P(P(i64)), P(i32)]
    L.vls_result_records.restype = i32
    L.vls_result_kernel_times.argtypes = [vp, P(P(ctypes.c_char_p)), P(P(i64)), P(P(dbl)), P(i32)]
    L.vls_result_kernel_times.restype = i32
    L.vls_result_free.argtypes = [vp]
    L.vls_result_free.restype = None
    L.vls_tunnel_pass_noalloc.argtypes = [vp, i64, i64, vp, i32, vp, i64, P(vls_options), vp, vp, vp]
    L.vls_tunnel_pass_noalloc.restype = i32
    L.vls_status_string.argtypes = [i32]
    L.vls_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


# ----------------------------------------------------------------- C-named wrappers
PRECISION = {"fp64": VLS_FP64, "fp32": VLS_FP32_RECHECK, "bf16": VLS_BF16_RECHECK}


def vls_default_options(**overrides) -> vls_options:
    """Defaults of the library with fields overridden by keyword; precision may be given as
    "fp64" / "fp32" (VLS_FP32_RECHECK) / "bf16" (VLS_BF16_RECHECK) or as the enum value."""
    o = vls_options()
    load().vls_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        setattr(o, k, v)
    return o


def vls_constants(o: vls_options | None = None) -> dict:
    o = o or vls_default_options()
    out = (ctypes.c_double * 4)()
    load().vls_constants(ctypes.byref(o), out)
    return {"eta": out[0], "lbar": out[1], "dt": out[2], "s": out[3]}


def vls_create(opts: vls_options | None = None, stream: int = 0) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    st = load().vls_create(ctypes.byref(ctx), ctypes.byref(opts) if opts is not None else None,
                           ctypes.c_void_p(stream) if stream else None)
    if st != 0:
        raise RuntimeError(f"vls_create failed: {STATUS.get(st, st)}")
    return ctx


def vls_destroy(ctx) -> None:
    load().vls_destroy(ctx)


def _mesh_struct(X, F, device: bool):
    m = vls_mesh()
    if device:
        m.X, m.nv, m.F, m.nf, m.device = int(X.data_ptr()), int(X.shape[0]), int(F.data_ptr()), int(F.shape[0]), 1
        keep = (X, F)
    else:
        X = np.ascontiguousarray(X, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.int32)
        m.X, m.nv, m.F, m.nf, m.device = X.ctypes.data, X.shape[0], F.ctypes.data, F.shape[0], 0
        keep = (X, F)
    return m, keep


def vls_detect_batch(ctx, meshes, seeds_per_mesh, device: bool = False) -> ctypes.c_void_p:
    """meshes: list of (X, F) (numpy host arrays, or torch CUDA tensors with device=True);
    seeds_per_mesh: list of lists of seed vertices.  Returns a result handle."""
    L = load()
    arr = (vls_mesh * len(meshes))()
    keep = []
    for i, (X, F) in enumerate(meshes):
        m, k = _mesh_struct(X, F, device)
        arr[i] = m
        keep.append(k)
    flat = [int(s) for ss in seeds_per_mesh for s in ss]
    seeds = (ctypes.c_int32 * max(1, len(flat)))(*flat)
    spm = (ctypes.c_int32 * len(meshes))(*[len(ss) for ss in seeds_per_mesh])
    out = ctypes.c_void_p()
    st = L.vls_detect_batch(ctx, len(meshes), arr, seeds, spm, ctypes.byref(out))
    if not out.value:
        raise RuntimeError(f"vls_detect_batch failed: {STATUS.get(st, st)}")
    return out


def vls_detect(ctx, X, F, seed: int, device: bool = False) -> ctypes.c_void_p:
    L = load()
    m, keep = _mesh_struct(X, F, device)
    out = ctypes.c_void_p()
    st = L.vls_detect(ctx, ctypes.byref(m), int(seed), ctypes.byref(out))
    if not out.value:
        raise RuntimeError(f"vls_detect failed: {STATUS.get(st, st)}")
    return out


def vls_tunnel_pass_noalloc(F, nv: int, cover, handle_step: int, edges, out_verts, out_info,
                            opts: vls_options | None = None, stream: int = 0) -> int:
    """One tunnel pass with no device allocation (all arguments are CUDA tensors: F int32
    [nf, 3], cover int32 [nv], edges int32 [n, 2], out_verts int32 [nv], out_info int32 [4]).
    Returns the launch status; the pass status is out_info[0] once the stream has run."""
    return int(load().vls_tunnel_pass_noalloc(
        ctypes.c_void_p(F.data_ptr()), int(F.shape[0]), int(nv), ctypes.c_void_p(cover.data_ptr()),
        int(handle_step), ctypes.c_void_p(edges.data_ptr()), int(edges.shape[0]),
        ctypes.byref(opts) if opts is not None else None, ctypes.c_void_p(stream) if stream else None,
        ctypes.c_void_p(out_verts.data_ptr()), ctypes.c_void_p(out_info.data_ptr())))


def vls_result_free(res) -> None:
    load().vls_result_free(res)


# ----------------------------------------------------------------- result objects
@dataclass
class Handle:
    step: int
    layer: int
    node: int
    edges: np.ndarray
    verts: np.ndarray
    points: np.ndarray
    length: float


@dataclass
class Tunnel:
    status: int
    stop_step: int
    bstar: int
    verts: np.ndarray
    stream_status: int = -1             # PL streamline (Sec. 3.2): status, -1 not traced
    stream: np.ndarray | None = None    # [n, 3] points of the closed polyline
    stream_length: float = 0.0


@dataclass
class Problem:
    status: int
    genus: int
    stats: dict
    nodes: np.ndarray
    node_pos: np.ndarray
    layers: np.ndarray
    handles: list = field(default_factory=list)
    tunnels: list = field(default_factory=list)
    refined: list = field(default_factory=list)      # refined handle loops (Tunnel-shaped), one per handle
    offset_change: np.ndarray | None = None          # [h, 3] handle, tunnel, refined (Sec. 3.5)
    layer: np.ndarray | None = None
    phi: np.ndarray | None = None
    cover: np.ndarray | None = None
    records: np.ndarray | None = None
    step_uncertified: np.ndarray | None = None      # per step: uncertified decisions (FP32 / BF16 forms)

    @property
    def status_name(self) -> str:
        return STATUS.get(self.status, str(self.status))

    def events(self):
        kinds = {0: "SEED", 1: "SPLIT", 2: "MERGE", 3: "END"}
        return [(kinds[int(k)], int(s)) for k, s in self.nodes]

    def reeb_cycle_rank(self) -> int:
        return int(len(self.layers) - len(self.nodes) + 1)


def _np(ptr, n, dtype):
    if n <= 0 or not ptr:
        return np.zeros(0, dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def vls_result_kernel_times(res) -> dict:
    """{kernel name: (launches, total ms)} of a result computed with profile = 1."""
    L = load()
    P = ctypes.POINTER
    names, launches, ms, n = P(ctypes.c_char_p)(), P(ctypes.c_int64)(), P(ctypes.c_double)(), ctypes.c_int32()
    L.vls_result_kernel_times(res, ctypes.byref(names), ctypes.byref(launches), ctypes.byref(ms), ctypes.byref(n))
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(n.value)}


def _streamline(L, res, p: int, i: int, kind: int) -> dict:
    st, pts, n, ln = ctypes.c_int32(), ctypes.POINTER(ctypes.c_double)(), ctypes.c_int64(), ctypes.c_double()
    L.vls_result_streamline(res, p, i, kind, ctypes.byref(st), ctypes.byref(pts), ctypes.byref(n), ctypes.byref(ln))
    return dict(stream_status=int(st.value), stream=_np(pts, 3 * n.value, np.float64).reshape(-1, 3),
                stream_length=float(ln.value))


def read_result(res) -> list:
    """Copy every problem of a result handle into Python objects."""
    L = load()
    P = ctypes.POINTER
    out = []
    for p in range(L.vls_result_count(res)):
        st = L.vls_result_status(res, p)
        s = vls_stats()
        L.vls_result_stats(res, p, ctypes.byref(s))
        stats = {k: getattr(s, k) for k, _ in vls_stats._fields_}
        nodes, pos, lay = P(ctypes.c_int32)(), P(ctypes.c_double)(), P(ctypes.c_int32)()
        nn, nl = ctypes.c_int32(), ctypes.c_int32()
        L.vls_result_reeb(res, p, ctypes.byref(nodes), ctypes.byref(pos), ctypes.byref(nn), ctypes.byref(lay),
                          ctypes.byref(nl))
        pr = Problem(status=st, genus=L.vls_result_genus(res, p), stats=stats,
                     nodes=_np(nodes, 2 * nn.value, np.int32).reshape(-1, 2),
                     node_pos=_np(pos, 3 * nn.value, np.float64).reshape(-1, 3),
                     layers=_np(lay, 3 * nl.value, np.int32).reshape(-1, 3))
        for i in range(max(0, L.vls_result_num_loops(res, p, 0))):
            e, ne = P(ctypes.c_int32)(), ctypes.c_int64()
            info = (ctypes.c_int32 * 3)()
            ln = ctypes.c_double()
            L.vls_result_handle(res, p, i, ctypes.byref(e), ctypes.byref(ne), info, ctypes.byref(ln))
            v, nv_, pts, npt = P(ctypes.c_int32)(), ctypes.c_int64(), P(ctypes.c_double)(), ctypes.c_int64()
            L.vls_result_loop(res, p, 0, i, ctypes.byref(v), ctypes.byref(nv_), ctypes.byref(pts), ctypes.byref(npt))
            pr.handles.append(Handle(step=info[0], layer=info[1], node=info[2],
                                     edges=_np(e, 2 * ne.value, np.int32).reshape(-1, 2),
                                     verts=_np(v, nv_.value, np.int32),
                                     points=_np(pts, 3 * npt.value, np.float64).reshape(-1, 3), length=ln.value))
        for i in range(max(0, L.vls_result_num_loops(res, p, 1))):
            info = (ctypes.c_int32 * 3)()
            L.vls_result_tunnel(res, p, i, info)
            v, nv_ = P(ctypes.c_int32)(), ctypes.c_int64()
            L.vls_result_loop(res, p, 1, i, ctypes.byref(v), ctypes.byref(nv_), None, None)
            pr.tunnels.append(Tunnel(status=info[0], stop_step=info[1], bstar=info[2], verts=_np(v, nv_.value, np.int32),
                                     **_streamline(L, res, p, i, 0)))
        for i in range(max(0, L.vls_result_num_loops(res, p, 2))):
            info = (ctypes.c_int32 * 3)()
            L.vls_result_refined(res, p, i, info)
            v, nv_ = P(ctypes.c_int32)(), ctypes.c_int64()
            L.vls_result_loop(res, p, 2, i, ctypes.byref(v), ctypes.byref(nv_), None, None)
            pr.refined.append(Tunnel(status=info[0], stop_step=info[1], bstar=info[2], verts=_np(v, nv_.value, np.int32),
                                     **_streamline(L, res, p, i, 1)))
        dl = []
        for i in range(len(pr.handles)):
            out3 = (ctypes.c_double * 3)()
            L.vls_result_offset_change(res, p, i, out3)
            dl.append(list(out3))
        pr.offset_change = np.array(dl, dtype=np.float64).reshape(-1, 3)
        la, ph, co, nvv = P(ctypes.c_int32)(), P(ctypes.c_double)(), P(ctypes.c_int32)(), ctypes.c_int64()
        if L.vls_result_state(res, p, ctypes.byref(la), ctypes.byref(ph), ctypes.byref(co), ctypes.byref(nvv)) == 0:
            pr.layer = _np(la, nvv.value, np.int32)
            pr.phi = _np(ph, nvv.value, np.float64)
            pr.cover = _np(co, nvv.value, np.int32)
        rec, nr = P(ctypes.c_int64)(), ctypes.c_int32()
        L.vls_result_records(res, p, ctypes.byref(rec), ctypes.byref(nr))
        rec5 = _np(rec, 5 * nr.value, np.int64).reshape(-1, 5)
        pr.records = rec5[:, :4].copy()
        pr.step_uncertified = rec5[:, 4].copy()
        out.append(pr)
    return out


def detect(problems, opts: vls_options | None = None, device: bool = False, **overrides) -> list:
    """Convenience: problems = list of (mesh, [seeds]) (mesh with .X/.F); returns [Problem]."""
    o = opts if opts is not None else vls_default_options(**overrides)
    ctx = vls_create(o)
    try:
        res = vls_detect_batch(ctx, [(m.X, m.F) for m, _ in problems], [s for _, s in problems], device=device)
        try:
            return read_result(res)
        finally:
            vls_result_free(res)
    finally:
        vls_destroy(ctx)

"""CPU oracle of the loop-shrinking hot path (plain C, FP64, single-threaded).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and
by the CPU-baseline leg of ``bench.py``.  It shares no code with the CUDA library.
See ``vls_oracle.c`` for the paper passages it follows and the readings it takes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_vls_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOTMANIFOLD", 3: "ENONORIENTABLE", 4: "EDISCONNECTED",
          5: "EMAXSTEPS", 6: "ESLOTS", 7: "ELAYERS", 8: "ELOOPFAIL", 9: "ETIMEOUT", 10: "ENOMEM",
          11: "ECUDA", 12: "ESTALL"}
NODE_KIND = {0: "SEED", 1: "SPLIT", 2: "MERGE", 3: "END"}


class Options(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("e", ctypes.c_double), ("a", ctypes.c_double),
                ("w", ctypes.c_double), ("dt_factor", ctypes.c_double), ("eps0", ctypes.c_double),
                ("theta_iso", ctypes.c_double), ("lbar", ctypes.c_double),
                ("max_steps", ctypes.c_int32), ("max_pass_steps", ctypes.c_int32),
                ("seed_ring", ctypes.c_int32), ("naive", ctypes.c_int32), ("tunnels", ctypes.c_int32),
                ("record_steps", ctypes.c_int32), ("refine", ctypes.c_int32), ("offset", ctypes.c_double),
                ("max_passes", ctypes.c_int32), ("streamlines", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc, FP contraction off (each product/sum rounded alone)."""
    src = os.path.join(_HERE, "vls_oracle.c")
    hdr = os.path.join(_HERE, "vls_oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", _SO + ".tmp", src, "-lm"])
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            P = ctypes.POINTER
            L.orc_default_options.argtypes = [P(Options)]
            L.orc_constants.argtypes = [P(Options), P(dbl)]
            L.orc_detect.restype = vp
            L.orc_detect.argtypes = [vp, i64, vp, i64, i32, P(Options)]
            L.orc_free.argtypes = [vp]
            for name in ["orc_status", "orc_genus", "orc_steps", "orc_num_nodes", "orc_num_layers",
                         "orc_num_handles"]:
                getattr(L, name).restype = i32
                getattr(L, name).argtypes = [vp]
            for name, rt in [("orc_counters", P(i64)), ("orc_state_layer", P(i32)), ("orc_state_phi", P(dbl)),
                             ("orc_cover", P(i32)), ("orc_nodes", P(i32)), ("orc_node_pos", P(dbl)),
                             ("orc_layers", P(i32))]:
                getattr(L, name).restype = rt
                getattr(L, name).argtypes = [vp]
            L.orc_step_records.restype = P(i64)
            L.orc_step_records.argtypes = [vp, P(i32)]
            for name, rt in [("orc_handle_info", P(i32)), ("orc_handle_edges", P(i32)),
                             ("orc_handle_verts", P(i32)), ("orc_handle_points", P(dbl)),
                             ("orc_tunnel_info", P(i32)), ("orc_tunnel_verts", P(i32)),
                             ("orc_tunnel_arrival", P(i32))]:
                getattr(L, name).restype = rt
                getattr(L, name).argtypes = [vp, i32]
            L.orc_handle_length.restype = dbl
            L.orc_handle_length.argtypes = [vp, i32]
            for name, rt in [("orc_refined_info", P(i32)), ("orc_refined_verts", P(i32)),
                             ("orc_loop_offset_change", P(dbl))]:
                getattr(L, name).restype = rt
                getattr(L, name).argtypes = [vp, i32]
            L.orc_tunnel_arrival_time.restype = P(dbl)
            L.orc_tunnel_arrival_time.argtypes = [vp, i32]
            L.orc_mean_edge.restype = dbl
            L.orc_mean_edge.argtypes = [vp]
            L.orc_trace_streamline.restype = i32
            L.orc_trace_streamline.argtypes = [vp, i64, vp, i64, vp, vp, i64, i32, vp, i64, P(i64), P(i32)]
            L.orc_streamline.restype = i32
            L.orc_streamline.argtypes = [vp, i32, i32, P(i64), P(dbl), P(P(dbl))]
            _lib = L
    return _lib


def default_options(**kw) -> Options:
    o = Options()
    _load().orc_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def constants(opts: Options | None = None) -> dict:
    o = opts or default_options()
    out = (ctypes.c_double * 4)()
    _load().orc_constants(ctypes.byref(o), out)
    return {"eta": out[0], "lbar": out[1], "dt": out[2], "s": out[3]}


def _arr(ptr, n, dtype):
    if n == 0 or not ptr:
        return np.zeros(0, dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


@dataclass
class Handle:
    step: int
    layer: int
    node: int
    edges: np.ndarray      # [n, 2] (inside, outside) crossing edges in loop order
    verts: np.ndarray      # collapsed inside-vertex cycle
    points: np.ndarray     # [n, 3] isoline points
    length: float


@dataclass
class Tunnel:
    status: int
    stop_step: int
    bstar: int
    verts: np.ndarray
    arrival: np.ndarray | None = None
    arrival_time: np.ndarray | None = None   # with the step's fraction (record_steps only)
    stream_status: int = -1            # PL streamline (Sec. 3.2): status, -1 not run
    stream: np.ndarray | None = None   # [n, 3] points of the closed polyline
    stream_length: float = 0.0


@dataclass
class Result:
    status: int
    genus: int
    steps: int
    counters: np.ndarray
    layer: np.ndarray
    phi: np.ndarray
    cover: np.ndarray
    records: np.ndarray
    nodes: np.ndarray          # [n, 2] kind, step
    node_pos: np.ndarray       # [n, 3]
    layers: np.ndarray         # [L, 3] birth, death, final state
    handles: list = field(default_factory=list)
    tunnels: list = field(default_factory=list)
    refined: list = field(default_factory=list)   # Tunnel-shaped records of the refined handle loops
    offset_change: np.ndarray | None = None       # [h, 3]: handle, tunnel, refined (Sec. 3.5)
    mean_edge: float = 0.0

    @property
    def status_name(self) -> str:
        return STATUS.get(self.status, str(self.status))

    def events(self):
        return [(NODE_KIND[int(k)], int(s)) for k, s in self.nodes]

    def reeb_cycle_rank(self) -> int:
        # arcs = layers (birth -> death); the graph is connected through the seed
        return int(len(self.layers) - len(self.nodes) + 1)


def trace_streamline(mesh, tf, start: int, cut_edges=None, cap: int = 16384):
    """The PL streamline trace alone (Sec. 3.2) on the arrival field tf (sources 0, unreached -1),
    the given (a, b) edges cut: (status, [n, 3] points, source reached)."""
    L = _load()
    X = np.ascontiguousarray(mesh.X, dtype=np.float64)
    F = np.ascontiguousarray(mesh.F, dtype=np.int32)
    t = np.ascontiguousarray(tf, dtype=np.float64)
    ce = np.ascontiguousarray(np.zeros((0, 2)) if cut_edges is None else cut_edges, dtype=np.int32).reshape(-1, 2)
    pts = np.zeros((cap, 3))
    n, end = ctypes.c_int64(), ctypes.c_int32()
    st = L.orc_trace_streamline(X.ctypes.data, X.shape[0], F.ctypes.data, F.shape[0], t.ctypes.data,
                                ce.ctypes.data, ce.shape[0], int(start), pts.ctypes.data, cap,
                                ctypes.byref(n), ctypes.byref(end))
    return int(st), pts[:min(n.value, cap)].copy(), int(end.value)


def detect(mesh, seed: int, opts: Options | None = None, **kw) -> Result:
    """Run the oracle on (mesh.X, mesh.F) from seed vertex `seed`."""
    L = _load()
    o = opts if opts is not None else default_options(**kw)
    X = np.ascontiguousarray(mesh.X, dtype=np.float64)
    F = np.ascontiguousarray(mesh.F, dtype=np.int32)
    h = L.orc_detect(X.ctypes.data, X.shape[0], F.ctypes.data, F.shape[0], int(seed), ctypes.byref(o))
    try:
        st = L.orc_status(h)
        nv = X.shape[0]
        built = L.orc_state_layer(h)
        if not built:
            return Result(st, L.orc_genus(h), 0, np.zeros(8, np.int64), np.zeros(0, np.int32),
                          np.zeros(0), np.zeros(0, np.int32), np.zeros((0, 4), np.int64),
                          np.zeros((0, 2), np.int32), np.zeros((0, 3)), np.zeros((0, 3), np.int32))
        nrec = ctypes.c_int32()
        rec = L.orc_step_records(h, ctypes.byref(nrec))
        nn, nl, nh = L.orc_num_nodes(h), L.orc_num_layers(h), L.orc_num_handles(h)
        res = Result(
            status=st, genus=L.orc_genus(h), steps=L.orc_steps(h),
            counters=_arr(L.orc_counters(h), 8, np.int64),
            layer=_arr(built, nv, np.int32), phi=_arr(L.orc_state_phi(h), nv, np.float64),
            cover=_arr(L.orc_cover(h), nv, np.int32),
            records=_arr(rec, 4 * nrec.value, np.int64).reshape(-1, 4),
            nodes=_arr(L.orc_nodes(h), 2 * nn, np.int32).reshape(-1, 2),
            node_pos=_arr(L.orc_node_pos(h), 3 * nn, np.float64).reshape(-1, 3),
            layers=_arr(L.orc_layers(h), 3 * nl, np.int32).reshape(-1, 3))
        for i in range(nh):
            info = _arr(L.orc_handle_info(h, i), 5, np.int32)
            m, nvs = int(info[3]), int(info[4])
            res.handles.append(Handle(
                step=int(info[0]), layer=int(info[1]), node=int(info[2]),
                edges=_arr(L.orc_handle_edges(h, i), 2 * m, np.int32).reshape(-1, 2),
                verts=_arr(L.orc_handle_verts(h, i), nvs, np.int32),
                points=_arr(L.orc_handle_points(h, i), 3 * m, np.float64).reshape(-1, 3),
                length=float(L.orc_handle_length(h, i))))
            sl = []
            for kind in (0, 1):
                n, ln, pp = ctypes.c_int64(), ctypes.c_double(), ctypes.POINTER(ctypes.c_double)()
                sst = L.orc_streamline(h, i, kind, ctypes.byref(n), ctypes.byref(ln), ctypes.byref(pp))
                sl.append(dict(stream_status=int(sst), stream_length=float(ln.value),
                               stream=_arr(pp, 3 * n.value, np.float64).reshape(-1, 3)))
            ti = _arr(L.orc_tunnel_info(h, i), 4, np.int32)
            arr = L.orc_tunnel_arrival(h, i)
            atf = L.orc_tunnel_arrival_time(h, i)
            res.tunnels.append(Tunnel(status=int(ti[0]), stop_step=int(ti[1]), bstar=int(ti[2]),
                                      verts=_arr(L.orc_tunnel_verts(h, i), max(int(ti[3]), 0), np.int32),
                                      arrival=_arr(arr, nv, np.int32) if arr else None,
                                      arrival_time=_arr(atf, nv, np.float64) if atf else None, **sl[0]))
            ri = _arr(L.orc_refined_info(h, i), 4, np.int32)
            res.refined.append(Tunnel(status=int(ri[0]), stop_step=int(ri[1]), bstar=int(ri[2]),
                                      verts=_arr(L.orc_refined_verts(h, i), max(int(ri[3]), 0), np.int32),
                                      **sl[1]))
        res.offset_change = np.array([_arr(L.orc_loop_offset_change(h, i), 3, np.float64) for i in range(nh)]
                                     ).reshape(-1, 3)
        res.mean_edge = float(L.orc_mean_edge(h))
        return res
    finally:
        L.orc_free(h)

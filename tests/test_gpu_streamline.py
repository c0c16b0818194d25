"""GPU parity of the PL streamlines of the tunnel and refinement passes (Sec. 3.2) against the CPU
oracle, through the C ABI.

FP64 form: the fractional arrival times, every face choice and every point are computed with the
same operations in the same order as the oracle's, so status, points and length are bit-exact.
FP32 / BF16 forms: the arrival times come from the low-precision trajectory, so the points move
with its drift; where the pass's vertex loop equals the oracle's the streamline must still be a
valid closed trace of the same loop class (checked on the torus by its windings), with its length
close to the oracle's.
"""
import numpy as np
import pytest

import meshgen
import oracle
from parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_13168_gb300 import build as libbuild

    libbuild.build()
    import paper_2105_13168_gb300 as v

    v.load()
    return v


def assert_streamlines_equal(g, o):
    n = 0
    for kind in ("tunnels", "refined"):
        for a, b in zip(getattr(g, kind), getattr(o, kind)):
            assert a.stream_status == b.stream_status, (kind, a.stream_status, b.stream_status)
            assert np.array_equal(a.stream, b.stream), (kind, len(a.stream), len(b.stream))
            assert a.stream_length == b.stream_length
            n += a.stream_status == 0
    return n


SHAPES = {"torus": lambda: meshgen.torus(64, 32, 2.0, 0.7), "torus_small": lambda: meshgen.torus(24, 12),
          "chain2": lambda: meshgen.tube_chain(2, 64), "chain3": lambda: meshgen.tube_chain(3, 80),
          "capsules": lambda: meshgen.capsules(5, 60), "gyroid1": lambda: meshgen.gyroid(1, 40)}


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_streamlines_fp64_bit_exact(vls, name):
    m = SHAPES[name]()
    seeds = [meshgen.seed_vertex(k, m.nv) for k in range(3)]
    gs = vls.detect([(m, seeds)], keep_state=1, record_steps=1, precision="fp64")
    traced = passes = 0
    for g, s in zip(gs, seeds):
        o = oracle.detect(m, s, record_steps=1)
        assert_parity(g, o)
        traced += assert_streamlines_equal(g, o)
        passes += sum(t.status == 0 for t in g.tunnels + g.refined)
    assert traced == passes and (passes > 0 or m.genus() == 0)


@pytest.mark.parametrize("k", [7, 44, 120])
def test_streamlines_fp64_batch_problems(vls, k):
    m, seeds = meshgen.batch_problem(k)
    gs = vls.detect([(m, list(seeds))], precision="fp64")
    for g, s in zip(gs, seeds):
        o = oracle.detect(m, s)
        assert g.status == o.status
        assert_streamlines_equal(g, o)


def test_streamlines_fp64_tube_chain_batch(vls):
    """The tube-chain workload at grid scale 0.35 (8 tori, ~63k faces), 4 seeds in one batch."""
    probs = meshgen.workload(2, 0.35)
    gs = vls.detect(probs, precision="fp64")
    m, seeds = probs[0]
    for g, s in zip(gs, seeds):
        o = oracle.detect(m, s)
        assert g.status == o.status == 0
        assert assert_streamlines_equal(g, o) == 2 * 8


def _winding(P, fn):
    a = fn(P)
    d = np.diff(np.concatenate([a, a[:1]]))
    d = (d + np.pi) % (2 * np.pi) - np.pi
    return int(np.rint(d.sum() / (2 * np.pi)))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_streamlines_low_precision_torus(vls, precision):
    R0 = 2.0
    m = meshgen.torus(64, 32, R0, 0.7)
    seeds = [meshgen.seed_vertex(k, m.nv) for k in range(4)]
    gs = vls.detect([(m, seeds)], precision=precision)
    major = lambda P: np.arctan2(P[:, 1], P[:, 0])
    minor = lambda P: np.arctan2(P[:, 2], np.hypot(P[:, 0], P[:, 1]) - R0)
    for g, s in zip(gs, seeds):
        o = oracle.detect(m, s)
        t, rf = g.tunnels[0], g.refined[0]
        assert t.stream_status == 0 and rf.stream_status == 0
        assert abs(_winding(t.stream, major)) == 1
        assert abs(_winding(rf.stream, minor)) == 1 and _winding(rf.stream, major) == 0
        assert np.array_equal(t.stream[0], m.X[t.bstar]) and np.array_equal(rf.stream[0], m.X[rf.bstar])
        for a, b in ((t, o.tunnels[0]), (rf, o.refined[0])):
            L = np.linalg.norm(a.stream - np.roll(a.stream, -1, 0), axis=1).sum()
            assert abs(L - a.stream_length) <= 1e-9 * L
            if np.array_equal(a.verts, b.verts) and precision == "fp32":
                assert a.stream_length == pytest.approx(b.stream_length, rel=0.02)


def test_streamlines_switch(vls):
    """streamlines = 0 traces none and leaves every other result as it was."""
    m = meshgen.tube_chain(2, 64)
    s = meshgen.seed_vertex(1, m.nv)
    on = vls.detect([(m, [s])], precision="fp64", keep_state=1, record_steps=1)[0]
    off = vls.detect([(m, [s])], precision="fp64", keep_state=1, record_steps=1, streamlines=0)[0]
    assert all(t.stream_status == -1 and len(t.stream) == 0 for t in off.tunnels + off.refined)
    assert all(t.stream_status == 0 for t in on.tunnels + on.refined)
    for a, b in zip(on.tunnels + on.refined, off.tunnels + off.refined):
        assert a.status == b.status and np.array_equal(a.verts, b.verts)
    assert np.array_equal(on.records, off.records) and np.array_equal(on.phi, off.phi)
    o = oracle.detect(m, s, streamlines=0)
    assert all(t.stream_status == -1 for t in o.tunnels + o.refined)
    with pytest.raises(RuntimeError):
        vls.vls_create(vls.vls_default_options(streamlines=2))

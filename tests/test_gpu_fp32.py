"""GPU parity of the FP32 form (values stored and stepped in FP32; rows that decide within the
recheck margin of a threshold, or where several layers meet, redone in FP64) against the FP64
CPU oracle on the same seeded inputs.

The recheck removes the rounding of the step being taken, not the drift of the FP32 inputs
(about 1e-7, at most about 6e-7 measured).  A threshold decision whose FP64 value lies closer
to its threshold than that drift can still go the other way; the library counts every decision
taken within the drift bound (vls_options.drift_bound, 1e-6) of its threshold as uncertified,
per step and per pass.  The bar (tests/parity.py, assert_fp32_parity):
  - exact: status, genus, every event and the layer table (Reeb graph topology), handle loops
    (crossing edges and vertex sequences);
  - certified: the first step whose band record differs took an uncertified decision; every
    vertex whose cover step differs was covered at or after it; final layers, tunnel loops and
    refined loops differ only when uncertified decisions were taken;
  - values: |phi_fp32 - phi_oracle| <= 2e-6 on the state after the last step before the first
    divergence (and on the final state when no record differs); loop points within 1e-3 of their
    edge; Reeb positions within 1e-4, or 1e-2 when a step's band differs by a vertex (a position
    is a band mean).
"""
import numpy as np
import pytest

import meshgen
import oracle
from parity import FP32_TOL, assert_fp32_parity, first_divergence

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


def run_pair(vls, problems, gpu_kw=None, **kw):
    gpu = vls.detect(problems, keep_state=1, record_steps=1, precision="fp32", **(gpu_kw or {}), **kw)
    orc = [oracle.detect(m, s, record_steps=1, **kw) for m, seeds in problems for s in seeds]
    return gpu, orc


def test_torus_fp32_parity(vls):
    m = meshgen.torus(64, 32, 2.0, 0.7)
    s = meshgen.seed_vertex(0, m.nv)
    (g,), (o,) = run_pair(vls, [(m, [s])])
    assert o.status == 0
    err, _, _, _ = assert_fp32_parity(g, o, m.X)
    assert g.stats["rechecks"] > 0
    assert g.stats["rechecks"] < g.stats["row_updates"]
    print(f"torus fp32: max |phi - oracle| = {err}, rechecks {g.stats['rechecks']} of "
          f"{g.stats['row_updates']} rows, pass rechecks {g.stats['pass_rechecks']}")


@pytest.mark.parametrize("steps", [1, 7, 60, 109, 178])
def test_torus_fp32_state_each_phase(vls, steps):
    m = meshgen.torus(64, 32, 2.0, 0.7)
    s = meshgen.seed_vertex(0, m.nv)
    (g,), (o,) = run_pair(vls, [(m, [s])], max_steps=steps, tunnels=0)
    assert_fp32_parity(g, o, m.X)


@pytest.mark.parametrize("name", ["chain2", "chain3", "capsules", "sphere", "torus_small"])
def test_shapes_fp32_parity(vls, name):
    m = {"chain2": lambda: meshgen.tube_chain(2, 64), "chain3": lambda: meshgen.tube_chain(3, 80),
         "capsules": lambda: meshgen.capsules(5, 60), "sphere": lambda: meshgen.sphere(28),
         "torus_small": lambda: meshgen.torus(24, 12)}[name]()
    seeds = [meshgen.seed_vertex(sd, m.nv) for sd in range(2)]
    gpu, orc = run_pair(vls, [(m, seeds)])
    for g, o in zip(gpu, orc):
        assert_fp32_parity(g, o, m.X)


def values_before_divergence(vls, m, s, g, o):
    """|phi - phi_oracle| on the state after the last step whose record agrees (all decisions equal)."""
    i1 = first_divergence(g, o)
    if i1 is None or i1 == 0:
        return None
    (ga,), (oa,) = run_pair(vls, [(m, [s])], max_steps=i1, tunnels=0)
    assert np.array_equal(ga.records, oa.records) and np.array_equal(ga.layer, oa.layer)
    err = float(np.abs(ga.phi - oa.phi).max())
    assert err <= FP32_TOL, f"values after step {i1}: max err {err:.3e}"
    return err


def test_tube_chain_small_fp32_batch(vls):
    """The tube-chain workload at grid scale 0.35 (8 tori, ~63k faces), 4 seeds in one batch."""
    probs = meshgen.workload(2, 0.35)
    gpu, orc = run_pair(vls, probs)
    out = [assert_fp32_parity(g, o, probs[0][0].X) for g, o in zip(gpu, orc)]
    m, seeds = probs[0]
    errs = [values_before_divergence(vls, m, s, g, o) for s, g, o in zip(seeds, gpu, orc)]
    print(f"uncertified decisions {[g.stats['uncertified'] for g in gpu]}, pass {[g.stats['pass_uncertified'] for g in gpu]}, "
          f"max value error before the first divergence {errs}")
    rows = sum(g.stats["row_updates"] for g in gpu)
    print(f"tube chain 0.35 fp32: record steps differing {[r for _, r, _, _ in out]}, cover steps differing "
          f"{[c for _, _, c, _ in out]}, tunnel loops differing {[t for _, _, _, t in out]}, "
          f"rechecks {gpu[0].stats['rechecks']} of {rows} rows")


@pytest.mark.parametrize("steps", [100, 300])
def test_tube_chain_small_fp32_values_mid_run(vls, steps):
    """Values mid-run (front in flight) within the FP32 tolerance of the FP64 oracle."""
    m, seeds = meshgen.workload(2, 0.35)[0]
    gpu, orc = run_pair(vls, [(m, seeds)], max_steps=steps, tunnels=0)
    for g, o in zip(gpu, orc):
        err, rec_bad, _, _ = assert_fp32_parity(g, o, m.X)
        if rec_bad == 0:
            assert err <= FP32_TOL


def test_fp32_equals_fp64_form_on_integer_results(vls):
    """Both GPU forms agree on events and handle loops of a mixed batch; records, cover steps,
    final layers and tunnel loops differ only after uncertified decisions of the FP32 run."""
    meshes = [meshgen.torus(32, 16), meshgen.tube_chain(2, 56), meshgen.capsules(4, 48)]
    probs = [(m, [meshgen.seed_vertex(5 * i + k, m.nv) for k in range(2)]) for i, m in enumerate(meshes)]
    a = vls.detect(probs, keep_state=1, record_steps=1, precision="fp32")
    b = vls.detect(probs, keep_state=1, record_steps=1, precision="fp64")
    for ga, gb in zip(a, b):
        assert ga.status == gb.status and ga.events() == gb.events()
        assert len(ga.records) == len(gb.records)
        i1 = first_divergence(ga, gb)
        assert i1 is None or ga.step_uncertified[i1] > 0
        assert np.array_equal(ga.layer, gb.layer) or ga.stats["uncertified"] > 0
        if (ga.cover != gb.cover).any():
            assert i1 is not None
        assert [h.verts.tolist() for h in ga.handles] == [h.verts.tolist() for h in gb.handles]
        if [t.verts.tolist() for t in ga.tunnels] != [t.verts.tolist() for t in gb.tunnels]:
            assert ga.stats["pass_uncertified"] > 0 or ga.stats["uncertified"] > 0
        assert gb.stats["rechecks"] == 0 and gb.stats["pass_rechecks"] == 0
        assert gb.stats["uncertified"] == gb.stats["pass_uncertified"] == gb.stats["refine_uncertified"] == 0
        assert (gb.step_uncertified == 0).all()


def test_fp32_margin_option(vls):
    """A wide margin sends every row through the FP64 recheck and keeps parity; a bad margin is
    refused at context creation."""
    m = meshgen.torus(24, 12)
    s = meshgen.seed_vertex(0, m.nv)
    (g,), (o,) = run_pair(vls, [(m, [s])], gpu_kw={"recheck_margin": 0.2})
    assert_fp32_parity(g, o, m.X)
    assert g.stats["rechecks"] >= 0.5 * g.stats["row_updates"]
    for bad in (0.0, -1.0, 0.5):
        with pytest.raises(RuntimeError):
            vls.vls_create(vls.vls_default_options(precision="fp32", recheck_margin=bad))
    with pytest.raises(RuntimeError):
        vls.vls_create(vls.vls_default_options(precision=7))

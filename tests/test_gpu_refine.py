"""GPU parity of the handle-refinement passes (Sec. 3.3) and the loop classification (Sec. 3.5)
against the CPU oracle, through the C ABI; the options that switch them and bound the passes."""
import numpy as np
import pytest

import meshgen
import oracle
from parity import assert_parity, assert_refined_and_classes

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


@pytest.mark.parametrize("which", ["torus", "chain2", "chain3", "batch44", "batch7"])
def test_refined_loops_match_oracle(vls, which):
    if which.startswith("batch"):
        m, seeds = meshgen.batch_problem(int(which[5:]))
    else:
        m = {"torus": lambda: meshgen.torus(64, 32, 2.0, 0.7), "chain2": lambda: meshgen.tube_chain(2, 64),
             "chain3": lambda: meshgen.tube_chain(3, 80)}[which]()
        seeds = [meshgen.seed_vertex(k, m.nv) for k in range(2)]
    gs = vls.detect([(m, list(seeds))], keep_state=1, record_steps=1)
    for g, s in zip(gs, seeds):
        o = oracle.detect(m, s, record_steps=1)
        assert_parity(g, o)
        assert len(g.refined) == len(g.handles) == m.genus()
        assert all(r.status == 0 for r in g.refined)
        assert g.stats["refine_updates"] > 0 and g.stats["refine_mass_resid"] < 1e-12
        assert g.stats["mean_edge"] == pytest.approx(o.mean_edge, rel=1e-12)


def test_refine_switch_and_pass_bound(vls):
    m = meshgen.tube_chain(3, 80)
    s = meshgen.seed_vertex(0, m.nv)
    full = vls.detect([(m, [s])])[0]
    off = vls.detect([(m, [s])], refine=0)[0]
    assert [r.status for r in off.refined] == [-1] * len(off.handles)
    assert all(np.array_equal(a.verts, b.verts) for a, b in zip(off.tunnels, full.tunnels))
    assert np.isnan(off.offset_change[:, 2]).all() and not np.isnan(full.offset_change).any()
    two = vls.detect([(m, [s])], max_passes=2)[0]
    assert [t.status for t in two.tunnels] == [0, 0] + [-1] * (len(two.handles) - 2)
    assert [r.status for r in two.refined] == [0, 0] + [-1] * (len(two.handles) - 2)
    for i in range(2):
        assert np.array_equal(two.refined[i].verts, full.refined[i].verts)
    o = oracle.detect(m, s, refine=0)
    assert_refined_and_classes(off, o)

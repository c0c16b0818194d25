"""The multi-GPU partition on one GPU: a batch split over two ranks by greedy LPT, the two shards run
in turn, and the gathered per-problem results equal the whole batch's bit for bit (problems are
independent; their results do not depend on the batch they run in) -- but for the Reeb node
positions, band means summed in a batch-dependent order, equal to 1e-12."""
import numpy as np
import pytest

import meshgen

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


def same(a, b):
    assert a.status == b.status and a.events() == b.events()
    assert np.array_equal(a.records, b.records) and np.array_equal(a.layers, b.layers)
    # a Reeb node position is a band mean summed in parallel in the order the step's frontier was
    # built, which depends on the batch: equal up to rounding
    assert np.allclose(a.node_pos, b.node_pos, rtol=1e-12, atol=1e-12)
    assert np.array_equal(a.phi, b.phi) and np.array_equal(a.layer, b.layer) and np.array_equal(a.cover, b.cover)
    for x, y in zip(a.handles, b.handles):
        assert np.array_equal(x.edges, y.edges) and np.array_equal(x.points, y.points)
    for xs, ys in ((a.tunnels, b.tunnels), (a.refined, b.refined)):
        assert len(xs) == len(ys)
        for x, y in zip(xs, ys):
            assert (x.status, x.stop_step, x.bstar) == (y.status, y.stop_step, y.bstar)
            assert np.array_equal(x.verts, y.verts)
    assert np.array_equal(a.offset_change, b.offset_change, equal_nan=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_two_shards_equal_the_whole_batch(vls, precision):
    from paper_2105_13168_gb300 import partition

    meshes = [meshgen.torus(32, 16), meshgen.tube_chain(2, 56), meshgen.capsules(4, 48), meshgen.tube_chain(3, 64)]
    probs = [(m, [meshgen.seed_vertex(3 * i + k, m.nv) for k in range(2)]) for i, m in enumerate(meshes)]
    kw = dict(keep_state=1, record_steps=1, precision=precision)
    whole = vls.detect(probs, **kw)
    parts, idx = [], []
    for r in range(2):
        sub, mine = partition.shard(probs, r, 2)
        assert sub  # both ranks get work
        parts += vls.detect(sub, **kw)
        idx += mine
    gathered = partition.gather(parts, idx, len(whole))
    for a, b in zip(gathered, whole):
        same(a, b)

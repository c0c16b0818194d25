"""Resolution limit of the diffuse front (no GPU): which handles the method can register.

A handle is registered when the advancing front first splits -- the phi = 1 plateau closes around
one cycle of the handle, cutting the narrow band in two (Sec. 3.1) -- and the two children later
meet around the other cycle (a merge).  If the front's leading edge closes the second cycle before
the plateau has closed the first, the band never splits, no merge follows, and the handle passes
without an event (the Reeb graph misses its cycle).  The band is about 4 edges wide (the scaled
operator fixes eta = 4 lbar), so the two cycles must close at clearly different times.

On the nu x nv grid torus the uniform scaled operator sees a flat combinatorial torus (every
vertex alike, so the seed does not matter): the front is a disk growing at a constant number of
edges per step, and it closes the two cycles at radii nu / 2 and nv / 2.  Measured: the handle is
registered when |nu - nv| >= 7 and missed when |nu - nv| <= 4 (5 and 6 are the transition), over
nv = 8 .. 32 -- an absolute threshold in edges, independent of the torus's size.  So on a mesh of
finer resolution the same shape loses fewer handles (the difference of its cycle lengths in edges
grows with the resolution), which is what the Schwarz-P and gyroid workloads show.
"""
import pytest

import meshgen
import oracle

OK = 0


@pytest.mark.parametrize("nv", [8, 12, 16, 24, 32])
def test_grid_torus_threshold(nv):
    for dnu in (-12, -8, -7, -4, -2, 0, 2, 4, 7, 8, 12):
        nu = nv + dnu
        if nu < 6:
            continue
        m = meshgen.torus(nu, nv, 2.0, 0.7)
        assert m.genus() == 1
        r = oracle.detect(m, 0, tunnels=0)
        assert r.status == OK, r.status_name
        if abs(dnu) >= 7:
            assert len(r.handles) == 1 and r.reeb_cycle_rank() == 1, (nu, nv)
        else:
            # missed: no split before the front covers the torus, the Reeb graph is a tree
            assert len(r.handles) == 0 and r.reeb_cycle_rank() == 0, (nu, nv)
            assert [k for k, _ in r.events()].count("MERGE") == 0


def test_threshold_is_absolute_in_edges():
    """Scaling both circumferences by 3 (nu - nv from 4 to 12) turns a missed handle into a registered
    one: the threshold is in edges, not a ratio."""
    small = oracle.detect(meshgen.torus(16, 12, 2.0, 0.7), 0, tunnels=0)
    large = oracle.detect(meshgen.torus(48, 36, 2.0, 0.7), 0, tunnels=0)
    assert len(small.handles) == 0 and len(large.handles) == 1

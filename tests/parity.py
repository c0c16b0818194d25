"""Parity assertions between a GPU result (paper_2105_13168_gb300.vls.Problem) and the CPU
oracle (oracle.Result).  Integer work (events, labels, loops, cover steps, band hashes) is
compared exactly; FP64 values with a relative bound of 1e-12 (expected bit-identical: both
sides round every operation alone in the same order); Reeb positions are means summed in a
different order on the GPU, compared to 1e-12 relative of the coordinate scale."""
import numpy as np

FP64_REL = 1e-12
# FP32 form: value tolerance, and loop-point / Reeb-position tolerance (relative to coordinates)
FP32_TOL = 2e-6
GEOM_TOL = 1e-4
GEOM_TOL_FP32_POINTS = 1e-3


def assert_close(a, b, rel=FP64_REL, what=""):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    if a.size == 0:
        return
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(a - b).max())
    assert err <= rel * scale, f"{what}: max abs err {err:.3e} > {rel:.1e} * {scale:.3e}"


def assert_parity(g, o, state=True, records=True):
    assert g.status == o.status, (g.status_name, o.status_name)
    assert g.genus == o.genus
    if records and o.records is not None and len(o.records):
        n = min(len(g.records), len(o.records))
        assert len(g.records) == len(o.records), (len(g.records), len(o.records))
        bad = np.nonzero((g.records[:n] != o.records[:n]).any(axis=1))[0]
        assert bad.size == 0, f"first divergent step {bad[0] + 1}: gpu {g.records[bad[0]]} oracle {o.records[bad[0]]}"
    assert g.events() == o.events(), f"events: gpu {g.events()[:12]} oracle {o.events()[:12]}"
    assert np.array_equal(g.layers, o.layers)
    assert_close(g.node_pos, o.node_pos, what="reeb node positions")
    assert len(g.handles) == len(o.handles)
    for i, (hg, ho) in enumerate(zip(g.handles, o.handles)):
        assert (hg.step, hg.layer, hg.node) == (ho.step, ho.layer, ho.node), \
            f"handle {i}: gpu {(hg.step, hg.layer, hg.node, len(hg.edges))} oracle {(ho.step, ho.layer, ho.node, len(ho.edges))}"
        assert np.array_equal(hg.edges, ho.edges), f"handle {i} crossing edges differ"
        assert np.array_equal(hg.verts, ho.verts), f"handle {i} vertices differ"
        assert_close(hg.points, ho.points, what=f"handle {i} points")
        assert abs(hg.length - ho.length) <= FP64_REL * max(1.0, ho.length)
    assert len(g.tunnels) == len(o.tunnels)
    for i, (tg, to) in enumerate(zip(g.tunnels, o.tunnels)):
        assert (tg.status, tg.stop_step, tg.bstar) == (to.status, to.stop_step, to.bstar), \
            f"tunnel {i}: gpu {(tg.status, tg.stop_step, tg.bstar)} oracle {(to.status, to.stop_step, to.bstar)}"
        assert np.array_equal(tg.verts, to.verts), f"tunnel {i} differs"
    assert_refined_and_classes(g, o)
    if state and g.phi is not None:
        assert np.array_equal(g.layer, o.layer)
        assert np.array_equal(g.cover, o.cover)
        assert_close(g.phi, o.phi, what="phi")


def assert_refined_and_classes(g, o, skip=()):
    """Refined handle loops (Sec. 3.3) identical; the offset length changes of the loop
    classification (Sec. 3.5) within 1e-9 relative (the GPU sums a loop's segments in parallel, in
    another order), and their signs equal where they are not within that of zero.  Handles in
    `skip` (whose tunnel loops legitimately differ) are left out."""
    assert len(g.refined) == len(o.refined) == len(o.handles)
    for i, (rg, ro) in enumerate(zip(g.refined, o.refined)):
        if i in skip:
            continue
        assert (rg.status, rg.stop_step, rg.bstar) == (ro.status, ro.stop_step, ro.bstar), \
            f"refined {i}: gpu {(rg.status, rg.stop_step, rg.bstar)} oracle {(ro.status, ro.stop_step, ro.bstar)}"
        assert np.array_equal(rg.verts, ro.verts), f"refined handle {i} differs"
    if len(o.handles) == 0:
        return
    a, b = np.asarray(g.offset_change, dtype=np.float64), np.asarray(o.offset_change, dtype=np.float64)
    assert a.shape == b.shape
    keep = np.ones(len(b), bool)
    keep[list(skip)] = False
    a, b = a[keep], b[keep]
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(b)
    tol = 1e-9 * np.maximum(1.0, np.abs(b[ok]))
    assert (np.abs(a[ok] - b[ok]) <= tol).all(), f"offset length change: max err {np.abs(a[ok] - b[ok]).max():.3e}"
    sure = np.abs(b[ok]) > tol
    assert (np.sign(a[ok])[sure] == np.sign(b[ok])[sure]).all()


def close(a, b, rel, what):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    if a.size == 0:
        return 0.0
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(a - b).max())
    assert err <= rel * scale, f"{what}: max abs err {err:.3e} > {rel:.1e} * {scale:.3e}"
    return err


def point_moves(hg, ho, X=None):
    """Handle-loop points of two runs on identical crossing edges.  A point interpolates theta along
    its edge (a, b) at t = (psi_a - theta) / (psi_a - psi_b), so a value error d moves it along the
    edge by up to d / (psi_a - psi_b) in t: small on most edges, large only where the edge's value
    jump is tiny.  Every point must stay on its edge (0 <= t <= 1).  Returns the per-point
    displacement |dp| and, when the positions X are given, the move |dt| in the edge parameter."""
    dp = np.linalg.norm(np.asarray(hg.points) - np.asarray(ho.points), axis=1)
    if X is None:
        return dp, None
    a, b = X[hg.edges[:, 0]], X[hg.edges[:, 1]]
    ab = b - a
    L2 = np.maximum((ab * ab).sum(axis=1), 1e-300)
    tg = ((np.asarray(hg.points) - a) * ab).sum(axis=1) / L2
    to = ((np.asarray(ho.points) - a) * ab).sum(axis=1) / L2
    off = np.linalg.norm(np.asarray(hg.points) - (a + tg[:, None] * ab), axis=1)
    assert (tg >= -1e-9).all() and (tg <= 1 + 1e-9).all() and (off <= 1e-9 * (1 + np.sqrt(L2))).all(), \
        "a handle-loop point left its crossing edge"
    return dp, np.abs(tg - to)


def first_divergence(g, o):
    """0-based index of the first step whose record (frontier size, band size, band hash) differs
    between two runs, or None."""
    n = min(len(g.records), len(o.records))
    bad = np.nonzero((g.records[:n] != o.records[:n]).any(axis=1))[0]
    if bad.size:
        return int(bad[0])
    return None if len(g.records) == len(o.records) else n


def assert_fp32_parity(g, o, X=None):
    """The contract of the FP32 / BF16 forms against the FP64 oracle (reading R-14).

    Exact: status, genus, events, layer table and handle loops.  Certified: a low-precision run can
    only leave the FP64 trajectory through a threshold decision taken within the drift bound of its
    threshold, which the library counts as uncertified.  So the first step whose band record
    differs must have taken uncertified decisions; every vertex whose cover step differs was first
    covered at or after that step; final layers, tunnel loops and refined loops differ only when
    an uncertified decision was taken (in the initial pass, the tunnel or the refinement passes).
    Values within FP32_TOL when no record differs.  Returns (max value error or None, differing
    record steps, differing cover steps, differing tunnel loops)."""
    assert g.status == o.status, (g.status_name, o.status_name)
    assert g.genus == o.genus
    assert g.events() == o.events()
    assert np.array_equal(g.layers, o.layers)
    assert len(g.records) == len(o.records), (len(g.records), len(o.records))
    rec_bad = int((g.records != o.records).any(axis=1).sum())
    i1 = first_divergence(g, o)
    if i1 is not None:
        assert g.step_uncertified is not None and g.step_uncertified[i1] > 0, \
            f"step {i1 + 1} is the first whose band differs but took no uncertified decision"
    # a node position is the mean of an event step's band: one vertex more or less in that band
    # (a differing record) moves it by about the band's extent over its size
    close(g.node_pos, o.node_pos, GEOM_TOL if rec_bad == 0 else 1e-2, "reeb node positions")
    assert len(g.handles) == len(o.handles)
    npts, far = 0, 0
    for i, (hg, ho) in enumerate(zip(g.handles, o.handles)):
        assert (hg.step, hg.layer, hg.node) == (ho.step, ho.layer, ho.node), f"handle {i}"
        assert np.array_equal(hg.edges, ho.edges), f"handle {i} crossing edges differ"
        assert np.array_equal(hg.verts, ho.verts), f"handle {i} vertices differ"
        # a point interpolates theta between its edge's values: the FP32 drift divided by the
        # edge's value jump moves it along the edge (points on near-flat edges move far)
        dp, dt = point_moves(hg, ho, X)
        npts += dp.size
        far += int((dt > 1e-3).sum()) if dt is not None else int((dp > GEOM_TOL_FP32_POINTS).sum())
        # the polyline length moves by at most twice the points' displacements
        assert abs(hg.length - ho.length) <= 2 * float(dp.sum()) + 1e-9 * max(1.0, ho.length), f"handle {i} length"
    # while no decision differed the values agree to the FP32 tolerance and few points move; a
    # snap decision that moved (a differing step record) perturbs its neighbourhood by up to eps0
    # and the points near it move further: those are only required to stay on their edges
    if rec_bad == 0:
        assert far <= 2 + 0.01 * npts, f"{far} of {npts} handle-loop points moved beyond 1e-3 of their edge"
    unc_init = g.stats["uncertified"] > 0
    unc_pass = g.stats["pass_uncertified"] > 0
    # cover steps: a vertex whose cover step differs was covered at or after the first divergence
    cov = g.cover != o.cover
    cov_bad = int(cov.sum())
    if cov_bad:
        assert i1 is not None, f"{cov_bad} cover steps differ with identical step records"
        first = np.minimum(g.cover[cov], o.cover[cov])
        first = np.where(first < 0, np.maximum(g.cover[cov], o.cover[cov]), first)
        assert first.min() >= i1 + 1, f"a cover step differs at step {first.min()} before the first divergence {i1 + 1}"
    lay_bad = int((g.layer != o.layer).sum())
    if lay_bad:
        assert unc_init, f"{lay_bad} final layers differ without an uncertified decision"
    # tunnel passes decide arrival steps at theta over thousands of steps: a loop differs only after
    # an uncertified decision (of its pass, or of the initial pass through the covered area)
    assert len(g.tunnels) == len(o.tunnels)
    bad_t = {i for i, (tg, to) in enumerate(zip(g.tunnels, o.tunnels))
             if (tg.status, tg.stop_step, tg.bstar) != (to.status, to.stop_step, to.bstar) or not np.array_equal(tg.verts, to.verts)}
    tun_bad = len(bad_t)
    if tun_bad:
        assert unc_pass or unc_init, f"{tun_bad} tunnel loops differ without an uncertified decision"
    ref_bad = sum((rg.status, rg.stop_step, rg.bstar) != (ro.status, ro.stop_step, ro.bstar) or not np.array_equal(rg.verts, ro.verts)
                  for i, (rg, ro) in enumerate(zip(g.refined, o.refined)) if i not in bad_t)
    if ref_bad:
        assert g.stats["refine_uncertified"] > 0 or unc_pass or unc_init, \
            f"{ref_bad} refined handle loops differ without an uncertified decision"
    err = None
    if rec_bad == 0:
        err = float(np.abs(g.phi - o.phi).max()) if g.phi.size else 0.0
        assert err <= FP32_TOL, f"phi max abs err {err:.3e} > {FP32_TOL:.1e}"
    return err, rec_bad, cov_bad, tun_bad



"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same seeded
inputs (element by element: per-step frontier/band sizes and band hashes, every event, layer
table, Reeb node, handle loop, tunnel loop, final state and cover steps)."""
import numpy as np
import pytest

import meshgen
import oracle
from parity import assert_close, assert_fp32_parity, assert_parity

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


def run_gpu(vls, problems, **kw):
    return vls.detect(problems, keep_state=1, record_steps=1, **kw)


def run_orc(m, s, **kw):
    return oracle.detect(m, s, record_steps=1, **kw)


def test_torus_full_parity(vls):
    m = meshgen.torus(64, 32, 2.0, 0.7)
    s = meshgen.seed_vertex(0, m.nv)
    g = run_gpu(vls, [(m, [s])])[0]
    o = run_orc(m, s)
    assert o.status == 0
    assert_parity(g, o)


@pytest.mark.parametrize("steps", [1, 2, 7, 60, 108, 109, 150, 177, 178])
def test_torus_state_each_phase(vls, steps):
    """State after exactly `steps` steps (before/at/after the split and the merge)."""
    m = meshgen.torus(64, 32, 2.0, 0.7)
    s = meshgen.seed_vertex(0, m.nv)
    g = run_gpu(vls, [(m, [s])], max_steps=steps, tunnels=0)[0]
    o = run_orc(m, s, max_steps=steps, tunnels=0)
    assert_parity(g, o)


@pytest.mark.parametrize("name", ["chain2", "chain3", "capsules", "sphere", "torus_small"])
def test_shapes_full_parity(vls, name):
    m = {"chain2": lambda: meshgen.tube_chain(2, 64), "chain3": lambda: meshgen.tube_chain(3, 80),
         "capsules": lambda: meshgen.capsules(5, 60), "sphere": lambda: meshgen.sphere(28),
         "torus_small": lambda: meshgen.torus(24, 12)}[name]()
    for sd in range(2):
        s = meshgen.seed_vertex(sd, m.nv)
        g = run_gpu(vls, [(m, [s])])[0]
        o = run_orc(m, s)
        assert_parity(g, o)


def test_batch_equals_single_runs(vls):
    """Problems of uneven size in one batch give exactly their solo results."""
    meshes = [meshgen.torus(32, 16), meshgen.tube_chain(2, 56), meshgen.capsules(4, 48)]
    probs = [(m, [meshgen.seed_vertex(3 * i + k, m.nv) for k in range(2)]) for i, m in enumerate(meshes)]
    batched = run_gpu(vls, probs)
    i = 0
    for m, seeds in probs:
        for s in seeds:
            solo = run_gpu(vls, [(m, [s])])[0]
            o = run_orc(m, s)
            assert_parity(batched[i], o)
            assert_parity(solo, o)
            i += 1


def test_device_pointers_equal_host(vls):
    import torch

    m = meshgen.tube_chain(2, 56)
    s = meshgen.seed_vertex(5, m.nv)
    o = run_orc(m, s)
    ctx = vls.vls_create(vls.vls_default_options(keep_state=1, record_steps=1))
    try:
        X, F = torch.from_numpy(m.X).cuda(), torch.from_numpy(m.F).cuda()
        res = vls.vls_detect(ctx, X, F, s, device=True)
        g = vls.read_result(res)[0]
        vls.vls_result_free(res)
        res = vls.vls_detect(ctx, m.X, m.F, s, device=False)
        h = vls.read_result(res)[0]
        vls.vls_result_free(res)
    finally:
        vls.vls_destroy(ctx)
    assert_parity(g, o)
    assert_parity(h, o)


def test_invalid_meshes_statuses(vls):
    t = meshgen.torus(16, 8)
    bad = []
    bad.append(meshgen.Mesh(t.X, t.F[1:]))                         # open
    F = t.F.copy(); F[0] = F[0][::-1]; bad.append(meshgen.Mesh(t.X, F))  # flipped face
    bad.append(meshgen.Mesh(np.concatenate([t.X, t.X + 9]), np.concatenate([t.F, t.F + t.nv])))  # 2 parts
    F = t.F.copy(); F[2, 2] = t.nv; bad.append(meshgen.Mesh(t.X, F))     # index out of range
    probs = [(m, [0]) for m in bad] + [(t, [t.nv + 5])]               # + seed out of range
    gs = run_gpu(vls, probs)
    for (m, seeds), g in zip(probs, gs):
        o = oracle.detect(m, seeds[0])
        assert g.status == o.status, (g.status_name, o.status_name)


def test_step_limit_and_no_tunnels(vls):
    m = meshgen.tube_chain(2, 56)
    s = meshgen.seed_vertex(1, m.nv)
    g = run_gpu(vls, [(m, [s])], max_steps=123)[0]
    o = run_orc(m, s, max_steps=123)
    assert g.status_name == "EMAXSTEPS"
    assert_parity(g, o)


def test_stats_are_consistent(vls):
    m = meshgen.tube_chain(3, 64)
    s = meshgen.seed_vertex(2, m.nv)
    g = run_gpu(vls, [(m, [s])])[0]
    o = run_orc(m, s)
    assert g.stats["row_updates"] == o.counters[0]
    # the oracle counts the rows of tunnel and refinement passes together
    assert g.stats["pass_updates"] + g.stats["refine_updates"] == o.counters[2]
    assert g.stats["refine_updates"] > 0
    t_only = run_orc(m, s, refine=0)
    assert g.stats["pass_updates"] == t_only.counters[2]
    assert g.stats["merges"] == o.counters[3] and g.stats["splits"] == o.counters[4]
    assert g.stats["ends"] == o.counters[5] and g.stats["layers"] == o.counters[6]
    assert g.stats["steps"] == o.steps


@pytest.mark.parametrize("threads,bps,variant,rpw", [(64, 1, 1, 32), (256, 64, 2, 32), (128, 2, 1, 16),
                                                     (128, 4, 2, 8), (64, 64, 2, 8), (256, 1, 1, 16)])
def test_launch_shapes_and_union_find_variants(vls, threads, bps, variant, rpw):
    """Every launch shape, both band union-find variants and every rows-per-warp setting give the
    oracle's results (the autotuner may pick any of them)."""
    m = meshgen.tube_chain(2, 64)
    s = meshgen.seed_vertex(1, m.nv)
    g = run_gpu(vls, [(m, [s])], threads=threads, blocks_per_sm=bps, hook_variant=variant, rows_per_warp=rpw)[0]
    assert_parity(g, run_orc(m, s))
    f = run_gpu(vls, [(m, [s])], precision="fp32", threads=threads, blocks_per_sm=bps, hook_variant=variant,
                rows_per_warp=rpw)[0]
    assert_fp32_parity(f, run_orc(m, s), m.X)


def test_rows_per_warp_option_checked(vls):
    for bad in (4, 12, 64, -1):
        with pytest.raises(RuntimeError):
            vls.vls_create(vls.vls_default_options(rows_per_warp=bad))


def test_tunnel_passes_in_chunks(vls, monkeypatch):
    """Tunnel passes split into memory-bounded chunks (here one pass per chunk) give the same
    loops as all passes at once."""
    m = meshgen.tube_chain(3, 80)
    s = meshgen.seed_vertex(0, m.nv)
    whole = run_gpu(vls, [(m, [s, s + 1])])
    monkeypatch.setenv("VLS_PASS_VERTS", "1")
    chunked = run_gpu(vls, [(m, [s, s + 1])])
    for a, b in zip(whole, chunked):
        assert [t.verts.tolist() for t in a.tunnels] == [t.verts.tolist() for t in b.tunnels]
        assert [(t.status, t.stop_step, t.bstar) for t in a.tunnels] == [(t.status, t.stop_step, t.bstar) for t in b.tunnels]
        assert len(a.tunnels) == 3
    assert_parity(chunked[0], run_orc(m, s))


@pytest.mark.parametrize("mesh,seed", [(44, 2), (51, 2)])
def test_tunnel_pass_fallbacks(vls, mesh, seed):
    """Batch mesh 44 seed 2: a handle loop separates the area covered at its step and the pass
    runs again on the whole surface.  Batch mesh 51 seed 2: a pass front stalls and the problem
    ends ELOOPFAIL.  Both exactly as the oracle."""
    m, seeds = meshgen.batch_problem(mesh)
    s = seeds[seed]
    g = run_gpu(vls, [(m, [s])])[0]
    assert_parity(g, run_orc(m, s))


def test_tunnels_off_keeps_status_ok(vls):
    """With the tunnel passes switched off a finished problem is OK, its tunnel records say
    'did not run' (status -1)."""
    m = meshgen.tube_chain(2, 56)
    g = run_gpu(vls, [(m, [meshgen.seed_vertex(0, m.nv)])], tunnels=0)[0]
    assert g.status == 0 and len(g.handles) == 2
    assert all(t.status == -1 for t in g.tunnels)


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_mass_check_of_the_diffusion_step(vls, precision, bound):
    """The FP64 mass check: at every step the lumped-mass-weighted Laplacian of the base sums to
    zero over the updated rows (m_v L_vu = 1 is symmetric and every row sums to zero), less the
    flux into vertices that are never rows (frozen plateaus in the initial pass, the sources of a
    tunnel pass), so the largest residual over the run is rounding only -- about 1e-16 relative to
    the terms in the FP64 form, about 1e-7 in the FP32 form -- on a torus, a genus-2 chain and the
    tube chain (4 seeds), in the initial pass and in the tunnel passes."""
    probs = [(meshgen.torus(64, 32, 2.0, 0.7), [meshgen.seed_vertex(0, 2048)]),
             (meshgen.tube_chain(2, 64), [1, 77])] + meshgen.workload(2, 0.35)
    out = vls.detect(probs, precision=precision)
    for p in out:
        assert p.status == 0, p.status_name
        r, rp = p.stats["mass_resid"], p.stats["pass_mass_resid"]
        assert 0.0 < r <= bound, r
        assert 0.0 < rp <= bound, rp  # the tunnel passes, sources' flux taken out
    print(precision, "largest mass residual", max(p.stats["mass_resid"] for p in out),
          "tunnel passes", max(p.stats["pass_mass_resid"] for p in out))


@pytest.mark.parametrize("host_loop", [0, 1])
def test_merge_phase_in_rounds(vls, host_loop):
    """More fronts meet in one step than the merge phase traces at once (64 isolines): 80 copies of
    the same torus problem merge at the same step (160 isolines), resolved in rounds; every copy
    gets exactly the oracle's result."""
    m = meshgen.torus(24, 12)
    s = meshgen.seed_vertex(1, m.nv)
    out = run_gpu(vls, [(m, [s] * 80)], host_loop=host_loop)
    o = run_orc(m, s)
    assert o.status == 0 and len(o.handles) == 1
    assert len(out) == 80
    for g in out:
        assert_parity(g, o)


def test_passes_overlapping_the_initial_pass(vls, monkeypatch):
    """The passes can also start while the initial pass runs (VLS_OVERLAP_PASSES=1: tunnel passes of
    the handles found by each 256-step segment, refinements once a problem's initial pass ended);
    every result is the same as in the default order (tunnel and refinement passes afterwards) and
    the oracle's."""
    meshes = [meshgen.tube_chain(3, 80), meshgen.torus(48, 20)]
    probs = [(m, [meshgen.seed_vertex(2 * i + k, m.nv) for k in range(2)]) for i, m in enumerate(meshes)]
    base = run_gpu(vls, probs)
    monkeypatch.setenv("VLS_OVERLAP_PASSES", "1")
    over = run_gpu(vls, probs)
    i = 0
    for m, seeds in probs:
        for s in seeds:
            o = run_orc(m, s)
            assert_parity(base[i], o)
            assert_parity(over[i], o)
            i += 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_host_loop_equals_graph(vls, precision):
    """The host-launched step loop (profiling path: every kernel launched each step, the merge
    scatter and the event kernels returning at once when nothing happened) gives the results of the
    device-driven graph, on a batch with splits, merges and extinctions."""
    meshes = [meshgen.tube_chain(3, 80), meshgen.capsules(5, 60), meshgen.torus(32, 16)]
    probs = [(m, [meshgen.seed_vertex(3 * i + k, m.nv) for k in range(2)]) for i, m in enumerate(meshes)]
    a = run_gpu(vls, probs, precision=precision)
    b = run_gpu(vls, probs, precision=precision, host_loop=1)
    for ga, gb in zip(a, b):
        assert ga.status == gb.status == 0
        assert ga.events() == gb.events()
        assert np.array_equal(ga.layers, gb.layers) and np.array_equal(ga.records, gb.records)
        assert np.array_equal(ga.cover, gb.cover) and np.array_equal(ga.layer, gb.layer)
        assert np.array_equal(ga.phi, gb.phi)
        for ta, tb in zip(ga.tunnels + ga.refined, gb.tunnels + gb.refined):
            assert ta.status == tb.status and np.array_equal(ta.verts, tb.verts)
            assert ta.stream_status == tb.stream_status and np.array_equal(ta.stream, tb.stream)
    kinds = {k for p in a for k, _ in p.events()}
    assert {"SPLIT", "MERGE", "END"} <= kinds

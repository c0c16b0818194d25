"""vls_tunnel_pass_noalloc (tunnel pass with no device allocation, for callers that cannot
allocate device memory) against the tunnel loops vls_detect reports for the same handles.

Collected last on purpose: the entry point keeps its scratch in one static device array of
the library, so this file also checks that consecutive calls (and calls after every other
GPU test of the session) see no leftovers of earlier calls."""
import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_13168_gb300 import build as libbuild

    libbuild.build()
    import paper_2105_13168_gb300 as v
    from paper_2105_13168_gb300 import vls

    v.load()
    return v, vls, torch


def test_noalloc_tunnel_pass_matches_detect(lib):
    v, vls, torch = lib
    m = meshgen.tube_chain(2, 56)
    s = meshgen.seed_vertex(4, m.nv)
    g = v.detect([(m, [s])], keep_state=1)[0]
    assert g.status_name == "OK" and len(g.handles) == 2
    F = torch.from_numpy(m.F).cuda()
    cover = torch.from_numpy(g.cover).cuda()
    edges = [torch.from_numpy(h.edges).cuda() for h in g.handles]
    calls = 0
    for _ in range(2):  # two rounds over both handles: consecutive calls share the scratch
        for h, t, e in zip(g.handles, g.tunnels, edges):
            out = torch.full((m.nv,), -7, dtype=torch.int32, device="cuda")
            info = torch.full((4,), -9, dtype=torch.int32, device="cuda")
            assert vls.vls_tunnel_pass_noalloc(F, m.nv, cover, h.step, e, out, info) == 0
            torch.cuda.synchronize()
            info = info.cpu().numpy()
            assert (info[0], info[1], info[2]) == (t.status, t.stop_step, t.bstar), (info, t.status, t.stop_step)
            assert info[0] == 0 and info[3] == len(t.verts)
            assert np.array_equal(out[: info[3]].cpu().numpy(), t.verts)
            calls += 1
    assert calls == 4


def test_noalloc_rejects_sizes_beyond_the_limit(lib):
    v, vls, torch = lib
    F = torch.zeros((8, 3), dtype=torch.int32, device="cuda")
    cover = torch.zeros(8, dtype=torch.int32, device="cuda")
    e = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = vls.vls_tunnel_pass_noalloc(F, 262145, cover, 0, e, out, info)
    assert vls.STATUS[st] == "ETOOLARGE"

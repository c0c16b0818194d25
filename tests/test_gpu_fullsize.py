"""Full-size parity on the tube-chain workload (8 smooth-unioned tori, ~512k faces, 4 seeds),
in the batched launch configuration the benchmark times, against the CPU oracle run on all
four seeds (a spawn process pool, started before the first GPU call): the FP64 form bit for bit,
and the FP32 form the benchmark times under its contract (identical events and handle loops)."""
import concurrent.futures as cf
import multiprocessing as mp

import pytest

import meshgen
from parity import assert_fp32_parity, assert_parity

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _oracle_job(args):
    import meshgen as mg
    import oracle as orc

    scale, seed = args
    m, _ = mg.workload(2, scale)[0]
    return orc.detect(m, seed, record_steps=1)


@pytest.fixture(scope="module")
def workload2():
    probs = meshgen.workload(2)
    m, seeds = probs[0]
    with cf.ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn")) as ex:
        orc = list(ex.map(_oracle_job, [(1.0, s) for s in seeds]))
    return probs, orc


def test_tube_chain_full_size_parity(workload2):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_13168_gb300 import build as libbuild

    libbuild.build()
    import paper_2105_13168_gb300 as vls

    probs, orc = workload2
    m = probs[0][0]
    assert m.nf > 500_000 and m.genus() == 8
    gpu = vls.detect(probs, keep_state=1, record_steps=1)
    assert len(gpu) == 4
    for g, o in zip(gpu, orc):
        assert o.status == 0 and len(o.handles) == 8
        assert_parity(g, o)
    g32 = vls.detect(probs, keep_state=1, record_steps=1, precision="fp32")
    for g, o in zip(g32, orc):
        err, rec_bad, cov_bad, tun_bad = assert_fp32_parity(g, o, m.X)
        print(f"tube chain full size, FP32 form: records differing {rec_bad}, cover steps differing {cov_bad}, "
              f"tunnel loops differing {tun_bad}, max |phi - oracle| {err}")

"""A single fused GEMM captured in a CUDA graph and replayed: every replay must redo the
packing protocol from scratch.  The ready words and arrival counters of one launch are tagged
with a launch count the kernel itself advances in the workspace, so a replayed launch (whose
arguments are frozen at capture) never mistakes the previous replay's panels for its own.
Compared with the oracle and bit for bit with an eager call of the same problem."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_08417_gb300 import gemmfip as g  # noqa: E402
from paper_2302_08417_gb300 import inputs  # noqa: E402
from tests import gpu_util as gu  # noqa: E402


@pytest.fixture(scope="module")
def runner():
    import __graft_entry__
    __graft_entry__.build()
    return gu.Runner()


LINE, SHARED = g.GFIP_PACKER_LINE, g.GFIP_PACKER_SHARED
CASES = [
    # FP64 32 x 32 tiles: 1120 tiles over a smaller persistent grid -> packing and stream-K
    (np.float64, "N", "N", 1100, 1000, 900, g.GFIP_PACK_AUTO, LINE),
    (np.float64, "T", "T", 700, 650, 1300, g.GFIP_PACK_BOTH, LINE),
    (np.float64, "N", "T", 900, 1000, 800, g.GFIP_PACK_AUTO, SHARED),
    # FP32 128 x 128 tiles: 18 x 18 tiles -> one partial wave split along k
    (np.float32, "N", "T", 2300, 2200, 700, g.GFIP_PACK_AUTO, LINE),
    (np.float32, "T", "N", 600, 900, 2000, g.GFIP_PACK_BOTH, LINE),
    (np.float32, "N", "N", 1500, 1400, 1100, g.GFIP_PACK_AUTO, SHARED),
]


@pytest.mark.parametrize("dtype,ta,tb,m,n,k,policy,packer", CASES)
@pytest.mark.parametrize("variant", ["fused", "pack_then_compute"])
def test_replayed_graph_matches_eager_and_oracle(runner, dtype, ta, tb, m, n, k, policy,
                                                 packer, variant):
    p = inputs.problem(m + n + k, ta, tb, m, n, k, 0.75, 0.5, 7, 3, 5, dtype=dtype)
    eager, _ = runner.run(p, variant, policy=policy, packer=packer)
    ref, ab = gu.reference(p)
    gu.assert_close(p, eager, ref, ab, label="eager")

    h, dev = runner.h, runner.dev
    esz = p.A.dtype.itemsize
    A = torch.from_numpy(p.A).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    C0 = torch.from_numpy(p.C0).to(dev)
    C = C0.clone()
    h.set_pack_policy(policy)
    h.set_packer(packer)
    h.ensure_workspace(p.transa, p.transb, p.m, p.n, p.k, esz)
    torch.cuda.synchronize()
    name = g.ENTRY[(variant, esz)]
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    try:
        with torch.cuda.stream(stream):
            h.bind_stream(stream)
            with torch.cuda.graph(graph, stream=stream):
                rc = g._gemm_call(name, h.h, p.transa, p.transb, p.m, p.n, p.k, p.alpha,
                                  A.data_ptr(), p.lda, B.data_ptr(), p.ldb, p.beta,
                                  C.data_ptr(), p.ldc)
        h.bind_stream(torch.cuda.current_stream())
        assert rc == 0, g.error_string(rc)
        for rep in range(4):
            C.copy_(C0)
            graph.replay()
            torch.cuda.synchronize()
            got = C.cpu().numpy()
            assert np.array_equal(got.view(np.uint8), eager.view(np.uint8)), f"replay {rep}"
        # an eager call on the same handle between replays keeps both correct
        again, _ = runner.run(p, variant, policy=policy, packer=packer)
        h.set_pack_policy(policy)
        h.set_packer(packer)
        assert np.array_equal(again.view(np.uint8), eager.view(np.uint8))
        C.copy_(C0)
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().view(np.uint8), eager.view(np.uint8))
    finally:
        h.bind_stream(torch.cuda.current_stream())
        h.set_pack_policy(g.GFIP_PACK_AUTO)
        h.set_packer(g.GFIP_PACKER_AUTO)
    assert h.status() == 0


def test_first_call_under_capture_is_refused_then_capture_works(runner):
    """The first call on a fresh workspace must clear its control words (a memset that a graph
    replay would repeat, resetting the launch counter that tags every ready word).  Under
    capture that call returns GFIP_ERR_CAPTURE and records nothing; once one eager call has
    cleared them, the same call captures and replays exactly."""
    p = inputs.problem(4242, "N", "N", 300, 280, 260, 1.0, 0.5, 7, 7, 7)
    dev = runner.dev
    h = g.Handle()
    h.bind_stream()
    h.ensure_workspace(p.transa, p.transb, p.m, p.n, p.k, 8)
    A = torch.from_numpy(p.A).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    C0 = torch.from_numpy(p.C0).to(dev)
    C = C0.clone()
    torch.cuda.synchronize()

    def call():
        return g.gfip_dgemm(h.h, p.transa, p.transb, p.m, p.n, p.k, p.alpha, A.data_ptr(),
                            p.lda, B.data_ptr(), p.ldb, p.beta, C.data_ptr(), p.ldc)

    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        h.bind_stream(stream)
        with torch.cuda.graph(graph, stream=stream):
            rc = call()
            torch.cuda._sleep(1)     # keeps the captured graph non-empty
    h.bind_stream()
    assert rc == g.GFIP_ERR_CAPTURE, g.error_string(rc)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().view(np.uint8), p.C0.view(np.uint8)), \
        "a refused call must not touch C"
    del graph

    assert call() == 0            # eager: clears the control words
    torch.cuda.synchronize()
    eager = C.cpu().numpy()
    ref, ab = gu.reference(p)
    gu.assert_close(p, eager, ref, ab, label="eager after refusal")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        h.bind_stream(stream)
        with torch.cuda.graph(graph, stream=stream):
            rc = call()
    h.bind_stream()
    assert rc == 0
    for _ in range(2):
        C.copy_(C0)
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().view(np.uint8), eager.view(np.uint8))
    assert h.status() == 0

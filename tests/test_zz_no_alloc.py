"""gks_step1d_noalloc: the 1-D S2O4 step for callers that cannot allocate
device memory (their memory belongs to another allocator, or they cannot
take cudaMalloc's implicit synchronisation).  Checked through the C ABI
against the context-based step (gks_step) on two calls in a row.  This file
is collected last so a stop-at-first-failure run has run everything else."""
import numpy as np
import pytest

from paper_2309_10534_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_10534_gb300 import build, gks
    build.build()
    return torch, gks


def _rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


@pytest.mark.parametrize("scheme", [{}, {"merge": "average"}, {"recon": "weno_ao"}, {"recon": "weno_z"},
                                    {"recon": "teno5"}], ids=["tenod", "average", "wenoao", "wenoz", "teno5"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_noalloc_step_matches_context_step_twice(env, precision, tol, scheme):
    torch, gks = env
    s = WL.sod(1000)
    dt1, dt2 = 2.0e-4, 2.5e-4
    ref = gks.Solver(1, 1000, bc=s.bc, precision=precision, tau="euler", **scheme)
    ref.set_state(s.W)
    ref.step(dt1)
    ref1 = ref.get_state()
    ref.step(dt2)
    ref2 = ref.get_state()

    dev = torch.device("cuda", torch.cuda.current_device())
    a = torch.from_numpy(np.ascontiguousarray(s.W[:, 0, :])).to(dev)
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    stream = torch.cuda.current_stream().cuda_stream
    assert gks.step1d_noalloc(a, b, s.dx, dt1, bc=s.bc[:2], precision=precision, stream=stream, **scheme) == 0
    assert _rel_l1(b.cpu().numpy(), ref1[:, 0, :]) < tol
    # second call in a row: the shared scratch holds the first call's data
    assert gks.step1d_noalloc(b, c, s.dx, dt2, bc=s.bc[:2], precision=precision, stream=stream, **scheme) == 0
    assert _rel_l1(c.cpu().numpy(), ref2[:, 0, :]) < tol


def test_noalloc_rejects_grids_beyond_its_static_scratch(env):
    torch, gks = env
    n = 16384 + 1
    a = torch.ones((3, n), dtype=torch.float64, device="cuda")
    with pytest.raises(gks.GKSError) as e:
        gks.step1d_noalloc(a, torch.empty_like(a), 1.0 / n, 1e-5)
    assert e.value.status == gks.GKS_EUNSUPPORTED


@pytest.mark.parametrize("kw,status", [({"positivity_fallback": 0}, "GKS_EUNSUPPORTED"), ({"merge": 7}, "GKS_EINVAL"),
                                       ({"recon": 9}, "GKS_EINVAL"), ({"ct1": -1.0}, "GKS_EINVAL")])
def test_noalloc_refuses_scheme_arguments(env, kw, status):
    torch, gks = env
    a = torch.ones((3, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(gks.GKSError) as e:
        gks.step1d_noalloc(a, torch.empty_like(a), 1.0 / 64, 1e-5, **kw)
    assert e.value.status == getattr(gks, status)


def test_noalloc_refuses_a_capturing_stream(env):
    torch, gks = env
    s = WL.sod(64)
    a = torch.from_numpy(np.ascontiguousarray(s.W[:, 0, :])).cuda()
    b = torch.empty_like(a)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.stream(side):
        g.capture_begin()
        try:
            gks.step1d_noalloc(a, b, s.dx, 1e-4, bc=s.bc[:2], stream=side.cuda_stream)
        except gks.GKSError as e:
            refused = e.status
        finally:
            g.capture_end()
    assert refused == gks.GKS_EINVAL

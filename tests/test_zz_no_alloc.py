"""proxsdp_gpu_aproj_noalloc: the truncated projection for callers that cannot
allocate device memory (code under CUDA-graph capture, hosts whose own pool
owns the GPU memory, real-time hosts that must not allocate mid-run).

It must give the same projection as proxsdp_gpu_aproj (within the 1e-5
relative tolerance the projection tests use) on two calls in a row, since the
calls share one static scratch array whose contents carry over; and it must
reject sizes beyond its limit without touching the GPU.  The outputs are
allocated by the test before the calls, so the calls themselves allocate
nothing.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import sdp_instances as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1810_05231_gb300 as p

    return p


def _matrix(n, r, seed):
    rng = np.random.default_rng(seed)
    lam = np.concatenate([np.sort(rng.uniform(2.0, 10.0, 2 * r))[::-1], -np.sort(rng.uniform(0.1, 30.0, n - 2 * r))])
    lam[:r] += 1.0  # a gap at r: the truncation is unique
    S, _, _ = si.random_symmetric_with_spectrum(n, lam, seed=seed)
    return torch.tensor(S, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("n,r", [(700, 8), (100, 6)])
def test_noalloc_matches_allocating_entry_point_twice(pkg, n, r):
    S1 = _matrix(n, r, seed=n + 1)
    S2 = _matrix(n, r, seed=n + 2)
    P = torch.empty((n, n), device="cuda", dtype=torch.float32)
    V = torch.empty((r, n), device="cuda", dtype=torch.float32)
    lam = torch.empty(r, device="cuda", dtype=torch.float64)
    for S in (S1, S2):  # two calls in a row on the shared scratch
        Pa, _, la, _ = pkg.aproj(S, r)
        Pn, Vn, ln, info = pkg.aproj_noalloc(S, r, P=P, V=V, lam=lam)
        torch.cuda.synchronize()
        ref = Pa.double()
        err = (Pn.double() - ref).norm().item() / ref.norm().item()
        assert err <= 1e-5, err
        assert torch.allclose(ln, la, rtol=1e-5, atol=1e-5 * la.abs().max().item())
        # the returned factors reproduce the projection
        Vd = Vn.double()
        rec = (Vd * ln.clamp(min=0)) @ Vd.t()
        assert (rec - Pn.double()).norm().item() <= 1e-5 * ref.norm().item()


def test_noalloc_rejects_sizes_beyond_its_limit(pkg):
    n = 2049
    S = torch.zeros((n, n), device="cuda", dtype=torch.float32)
    with pytest.raises(pkg.ProxSDPError) as e:
        pkg.aproj_noalloc(S, 4)
    assert e.value.code == -5  # PROXSDP_ERR_UNSUPPORTED
    assert "2048" in str(e.value)

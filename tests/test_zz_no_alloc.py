"""proxsdp_gpu_aproj_noalloc: the truncated projection for callers that cannot
allocate device memory (hosts whose own pool allocator owns the GPU memory and
forbids other allocations, plugins inside such hosts, real-time hosts that
must not allocate mid-run).

The calls share one static scratch array whose contents carry over from call
to call, so the test runs a sequence of calls that starts at the size limit
(n = 2048, where the scratch pieces are exactly full) and then goes to smaller
and back to larger sizes: every call must give the projection of its own
input, the exact truncation of Sec. 3.1 (Eq. trunc_eig) of a matrix with a
known spectrum within the 1e-5 relative tolerance the projection tests use,
and agree with proxsdp_gpu_aproj within the same tolerance.  Sizes beyond the
limit and invalid settings are rejected.  The outputs are allocated by the
test before the calls, so the calls themselves allocate nothing.  This file is
collected last on purpose.
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
    """S with a known spectrum (a gap at r, so the truncation is unique) and its exact truncation."""
    rng = np.random.default_rng(seed)
    lam = np.concatenate([np.sort(rng.uniform(2.0, 10.0, 2 * r))[::-1], -np.sort(rng.uniform(0.1, 30.0, n - 2 * r))])
    lam[:r] += 1.0
    S, Q, lam = si.random_symmetric_with_spectrum(n, lam, seed=seed)
    Pref = (Q[:, :r] * np.maximum(lam[:r], 0.0)) @ Q[:, :r].T
    return torch.tensor(S, dtype=torch.float32, device="cuda"), Pref, lam[:r]


@pytest.mark.parametrize("sizes,r", [((2048, 700, 100, 700), 8), ((700, 2048), 16)])
def test_noalloc_call_sequence_matches_exact_truncation(pkg, sizes, r):
    for k, n in enumerate(sizes):
        S, Pref, lam_ref = _matrix(n, r, seed=10 * n + k)
        P = torch.empty((n, n), device="cuda", dtype=torch.float32)
        V = torch.empty((r, n), device="cuda", dtype=torch.float32)
        lam = torch.empty(r, device="cuda", dtype=torch.float64)
        Pn, Vn, ln, info = pkg.aproj_noalloc(S, r, P=P, V=V, lam=lam)
        torch.cuda.synchronize()
        Pg = Pn.double().cpu().numpy()
        err = np.linalg.norm(Pg - Pref) / np.linalg.norm(Pref)
        assert err <= 1e-5, (n, err, info.as_dict())
        np.testing.assert_allclose(ln.cpu().numpy(), lam_ref, rtol=1e-5, atol=1e-5 * np.abs(lam_ref).max())
        # the allocating entry point on the same input
        Pa, _, la, _ = pkg.aproj(S, r)
        torch.cuda.synchronize()
        ea = (Pn.double() - Pa.double()).norm().item() / Pa.double().norm().item()
        assert ea <= 1e-5, (n, ea)
        # the returned factors reproduce the projection
        Vd = Vn.double()
        rec = (Vd * ln.clamp(min=0)) @ Vd.t()
        assert (rec - Pn.double()).norm().item() <= 1e-5 * np.linalg.norm(Pref)


def test_noalloc_dense_path_twice(pkg):
    """n <= 128 takes the one-block dense eigensolver; two calls in a row."""
    for seed in (1, 2):
        S, Pref, lam_ref = _matrix(100, 6, seed=seed)
        Pn, _, ln, _ = pkg.aproj_noalloc(S, 6)
        torch.cuda.synchronize()
        err = np.linalg.norm(Pn.double().cpu().numpy() - Pref) / np.linalg.norm(Pref)
        assert err <= 1e-5, err


def test_noalloc_rejects_sizes_beyond_its_limit(pkg):
    n = 2049
    S = torch.zeros((n, n), device="cuda", dtype=torch.float32)
    with pytest.raises(pkg.ProxSDPError) as e:
        pkg.aproj_noalloc(S, 4)
    assert e.value.code == -5  # PROXSDP_ERR_UNSUPPORTED
    assert "2048" in str(e.value)


def test_noalloc_rejects_invalid_settings(pkg):
    S, _, _ = _matrix(300, 4, seed=3)
    for bad in (dict(block_size=0), dict(guard=-1), dict(lanczos_steps=-1), dict(lanczos_max_cycles=0)):
        s = pkg.default_settings(**bad)
        with pytest.raises(pkg.ProxSDPError) as e:
            pkg.aproj_noalloc(S, 4, settings=s)
        assert e.value.code == -1, bad  # PROXSDP_ERR_INVALID_ARG

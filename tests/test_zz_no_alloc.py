"""The allocation-free PML/TVaR entry point (ara_pml_tvar_noalloc).

Some callers may not allocate device memory: code running under a
framework's caching allocator, which owns the device memory budget, or a
latency-critical loop in which cudaMalloc/cudaFree (which can synchronise the
device) are not acceptable.  This entry point keeps its select state in a
fixed block of device memory owned by the library instead.  The test calls it
through the C ABI twice in a row (two different YLTs, so the second call must
not see the first call's state) and compares each result with the
allocating entry point, ara_pml_tvar, and with the FP64 oracle.  It sits in a file of its own, collected
last, and passes both alone in a fresh process and after the other tests.
"""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

PML_TOL = 1e-4  # the PML / TVaR tolerance of the parity tests
RPS = np.array([1.0, 2.0, 100.0, 250.0, 1e6])


def _ylt(n, seed):
    rng = np.random.default_rng(seed)
    y = np.round(rng.lognormal(8, 2, n), 2)  # ties
    y[rng.random(n) < 0.4] = 0.0
    return y


def test_noalloc_pml_tvar_matches_the_allocating_entry_point():
    torch = pytest.importorskip("torch")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1501_06326_gb300 import ara

    eng = ara.Ara(0)
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    for call, (n, seed) in enumerate([(1_000_003, 1), (777, 2)]):
        y = _ylt(n, seed)
        ref_pml, ref_tvar = eng.pml_tvar(y, RPS)
        y_dev = torch.from_numpy(y).cuda()
        if call == 0:  # device outputs
            pml = torch.zeros(RPS.size, dtype=torch.float64, device="cuda")
            tvar = torch.zeros(RPS.size, dtype=torch.float64, device="cuda")
        else:  # host outputs
            pml, tvar = np.zeros(RPS.size), np.zeros(RPS.size)
        rc = ara.ara_pml_tvar_noalloc(y_dev, n, RPS, RPS.size, pml, tvar, stream)
        assert rc == ara.ARA_OK
        torch.cuda.synchronize()
        if call == 0:
            pml, tvar = pml.cpu().numpy(), tvar.cpu().numpy()
        assert np.allclose(pml, ref_pml, rtol=PML_TOL, atol=0)
        assert np.allclose(tvar, ref_tvar, rtol=PML_TOL, atol=0)
        # and against the FP64 oracle's sort (Section 2.3), as tightly as the
        # allocating entry point meets it: PML is one of the year losses, and
        # TVaR a sum of them in a fixed order
        or_pml, or_tvar = oracle.pml_tvar(y, RPS)
        assert np.array_equal(pml, or_pml)
        assert np.allclose(tvar, or_tvar, rtol=1e-12, atol=0)
        results.append((pml, tvar))
    eng.close()
    assert not np.array_equal(results[0][0], results[1][0])


def test_noalloc_rejects_what_it_cannot_serve():
    torch = pytest.importorskip("torch")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1501_06326_gb300 import ara

    y = _ylt(1000, 3)
    y_dev = torch.from_numpy(y).cuda()
    out = np.zeros(ara.ARA_NOALLOC_MAX_RP + 1)
    too_many = np.full(ara.ARA_NOALLOC_MAX_RP + 1, 100.0)
    assert ara.ara_pml_tvar_noalloc(y_dev, y.size, too_many, too_many.size, out, out.copy()) == ara.ARA_EINVAL
    assert ara.ara_pml_tvar_noalloc(y, y.size, RPS, RPS.size, out, out.copy()) == ara.ARA_EINVAL  # host ylt
    assert ara.ara_pml_tvar_noalloc(y_dev, 0, RPS, RPS.size, out, out.copy()) == ara.ARA_EINVAL

"""The allocation-free exp(tau X) e_1 entry point.

sgk_expm_e1_noalloc serves callers that must not allocate device memory
while they run (code being recorded into a CUDA graph, latency-critical
loops, processes whose device memory belongs to another allocator): its
scratch is a fixed array compiled into the library.  This file is collected
last so that a failure here does not stop the rest of the suite; it also
passes on its own in a fresh process.

Its outputs are checked against the FP64 oracle's Pade(13) scaling and
squaring (oracle.krylov.expm_pade13, first column) with the expm tolerance of
the parity tests (1e-12 relative to the largest entry), on both kernels it
runs: m <= 56 (the cluster kernel, work matrices in shared memory) and
56 < m <= 64 (the single-CTA kernel on the library's fixed scratch).  They
are also checked against the regular entry point, which allocates.  The
calls come in a row with different matrices, so later calls run on the
scratch left by earlier ones.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.krylov import expm_pade13  # noqa: E402
from paper_1810_11111_gb300 import sgkiif  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _noalloc(X, tau, stream):
    m = X.shape[0]
    Xd = torch.as_tensor(X, dtype=torch.float64, device="cuda").contiguous()
    yd = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
    rc = sgkiif.sgk_expm_e1_noalloc(m, Xd.data_ptr(), float(tau), yd.data_ptr(), stream)
    assert rc == sgkiif.SGK_OK
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _close(got, want):
    return np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_noalloc_expm_matches_oracle_and_regular_entry_point():
    sgkiif.load()
    stream = torch.cuda.current_stream().cuda_stream
    ctx = sgkiif.Context(0, stream, sgkiif.SGK_FP64)
    rng = np.random.default_rng(17)
    cases = [(rng.standard_normal((30, 30)) * 40.0 / 30, 0.5),
             (-np.diag(np.logspace(0, 4, 64)) + 0.01 * rng.standard_normal((64, 64)), 0.005),
             (rng.standard_normal((60, 60)) * 3.0, 0.2),
             (rng.standard_normal((64, 64)) * 2.0, 0.3),
             (rng.standard_normal((56, 56)) * 5.0, 0.1)]
    for rep in range(2):  # two calls in a row per case
        for X, tau in cases:
            oracle = expm_pade13(tau * X)[:, 0]
            got = _noalloc(X, tau, stream)
            assert _close(got, oracle), (X.shape, rep, np.abs(got - oracle).max())
            assert _close(got, ctx.expm_e1(X, tau))
    ctx.close()


def test_noalloc_expm_rejects_oversized_and_null():
    sgkiif.load()
    m = sgkiif.EXPM_NOALLOC_MAX_M + 1
    X = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    y = torch.zeros(m, dtype=torch.float64, device="cuda")
    assert sgkiif.sgk_expm_e1_noalloc(m, X.data_ptr(), 1.0, y.data_ptr(), None) == sgkiif.SGK_EINVAL
    assert sgkiif.sgk_expm_e1_noalloc(4, None, 1.0, y.data_ptr(), None) == sgkiif.SGK_EINVAL
    assert sgkiif.sgk_expm_e1_noalloc(0, X.data_ptr(), 1.0, y.data_ptr(), None) == sgkiif.SGK_EINVAL

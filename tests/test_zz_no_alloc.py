"""cdwac_build_W_imag_noalloc against cdwac_build_W_imag (GPU).

The allocation-free entry point serves callers that must not allocate device memory while they run; its scratch
is a fixed device array shared by all calls.  It runs the same kernels as the context path, so its W table must
match that path's within the FP64 parity tolerance, on two calls in a row with different systems (the shared
array keeps the previous call's contents), and oversized systems must be refused before anything runs.
This file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2305_15955_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2305_15955_gb300 import cdwac  # noqa: E402


def _system(spec, dtype=np.float64):
    eps = inputs.eigenvalues(spec)
    return cdwac.System(eps, inputs.build_B(spec, dtype=dtype), inputs.build_On(spec, dtype=dtype), spec.states,
                        spec.n_occ)


def _noalloc(sysd, p):
    dev = torch.device("cuda", 0)
    xi = torch.empty(p.n_imag, dtype=torch.float64, device=dev)
    wxi = torch.empty_like(xi)
    W = torch.full((sysd.n_states, p.n_imag, sysd.n_basis), np.nan, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rc = cdwac.build_W_imag_noalloc(sysd, p, xi, wxi, W, status)
    torch.cuda.synchronize()
    return rc, xi, wxi, W, int(status.cpu()[0])


def test_noalloc_matches_context_path_twice():
    ctx = cdwac.Context(0)
    cases = [(inputs.small_system(), np.float64, 40),
             (inputs.custom_system(70, 9, 200, seed=8, n_core=2, states=(0, 1), core_scale=0.3), np.float32, 24)]
    for spec, dt, n_imag in cases:
        sysd = _system(spec, dt)
        p = cdwac.Params(n_imag=n_imag)
        xi0, wxi0, W0 = ctx.build_W_imag(sysd, p)
        rc, xi, wxi, W, status = _noalloc(sysd, p)
        assert rc == cdwac.OK and status == 0
        assert torch.equal(xi, xi0) and torch.equal(wxi, wxi0)
        np.testing.assert_allclose(W.cpu().numpy(), W0.cpu().numpy(), rtol=1e-12, atol=1e-15)
    ctx.close()


def test_noalloc_refuses_oversized_and_mixed():
    spec = inputs.small_system()
    sysd = _system(spec)
    rc, *_ = _noalloc(sysd, cdwac.Params(n_imag=8, precision=cdwac.PREC_MIXED))
    assert rc == cdwac.ERR_ARG
    big = inputs.custom_system(1300, 10, 1500, seed=4, n_core=1, states=(0,))
    eps = inputs.eigenvalues(big)
    dev = torch.device("cuda", 0)
    # sizes only matter for the check: zero-filled device buffers of the right shape
    sys_big = cdwac.System(eps, torch.zeros(big.n_aux, big.n_ov, dtype=torch.float32, device=dev),
                           torch.zeros(1, big.n_aux, big.n_basis, dtype=torch.float32, device=dev), (0,), big.n_occ)
    rc, *_ = _noalloc(sys_big, cdwac.Params(n_imag=8))
    assert rc == cdwac.ERR_ARG

"""The allocation-free hydro residual (mhd_hydro_rhs_static) against the
ordinary context-based one (mhd_hydro_rhs), through the C ABI.

Some callers cannot allocate device memory (all of it belongs to their own
caching allocator or budget, or they sit in a latency-critical loop); the
allocation-free entry point serves them from a fixed library scratch array.
This file is collected last so that a run stopping at the first failure has
run every other test already; it passes alone and after the others.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p,mesh", [(3, (12, 9)), (2, (7, 5))])
def test_static_residual_matches_context_residual(p, mesh):
    import torch
    from oracle import Oracle
    from paper_2609_10849_b300.mhd import Solver, hydro_rhs_static
    from tests.test_oracle_hydro import smooth_random_state

    domain = (0.0, 1.3, 0.0, 0.9)
    o = Oracle(*mesh, p, p, 1.4, domain)  # only builds the input state
    s = Solver(*mesh, p, p, 1.4, domain)
    stream = torch.cuda.current_stream()
    for call in range(2):  # two calls in a row share the static scratch
        U = smooth_random_state(o, np.random.default_rng(7 + call))
        ref = s.hydro_rhs(U.copy())
        Ud = torch.tensor(U, dtype=torch.float64, device="cuda").contiguous()
        Ld = torch.full_like(Ud, float("nan"))
        hydro_rhs_static(*mesh, p, 1.4, domain, Ud, Ld, stream.cuda_stream)
        torch.cuda.synchronize()
        got = Ld.cpu().numpy()
        scale = np.abs(ref).max()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-12 * scale, (call, np.abs(got - ref).max() / scale)


def test_static_residual_rejects_oversized_mesh():
    """A mesh needing more face-flux scratch than the static array holds is
    refused by the C entry point (buffers of the right size, so the binding's
    own checks pass)."""
    import torch
    from paper_2609_10849_b300.mhd import MhdError, hydro_rhs_static
    n = 5 * 200 * 200 * 16
    U = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(MhdError, match="static scratch"):
        hydro_rhs_static(200, 200, 3, 1.4, (0.0, 1.0, 0.0, 1.0), U, torch.zeros_like(U))

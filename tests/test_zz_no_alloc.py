"""The allocation-free ILU apply.

Some callers cannot let the library allocate device memory in the middle of a
step (their framework owns all device memory, or a cudaMalloc there would
stall the device).  ilu_apply_noalloc serves them: same result as ilu_apply,
scratch taken from a fixed array inside the library.  This file runs last so
that a failure here does not hide the other tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1704_06862_gb300 as sie  # noqa: E402
from paper_1704_06862_gb300 import geometry as geo  # noqa: E402

MESH = dict(nu_outer=5, nu_inner=3, r_outer=0.75, r_inner=0.5, eps_shell=2.56, eps_core=4.0)


def _rand(s, nrhs, seed):
    return torch.from_numpy(geo.random_coefficients(2 * s.ne, nrhs, seed=seed).reshape(nrhs, s.ne, 2)).cuda()


def test_noalloc_ilu_allocates_nothing_on_a_fresh_context():
    """On a context that has never run an ILU apply (its work buffers not yet
    allocated), the first ilu_apply_noalloc call leaves the library's own
    device-byte count and the device's free memory unchanged."""
    import __graft_entry__ as g
    g.build()
    # a first context loads the library's kernels and the fixed scratch array
    warm = sie.Solver(geo.coated_sphere(**MESH), levels=4)
    r = _rand(warm, 1, 30)
    sie.ilu_apply_noalloc(warm.ctx, r, torch.zeros_like(r), 1, sie.SIE_PREC_MIXED)
    sie.ilu_apply_noalloc(warm.ctx, r, torch.zeros_like(r), 1, sie.SIE_PREC_FP64)
    torch.cuda.synchronize()
    warm.close()
    s = sie.Solver(geo.coated_sphere(**MESH), levels=4)
    try:
        r = _rand(s, 1, 31)
        z = torch.zeros_like(r)
        torch.cuda.synchronize()
        held0 = sie.sie_query(s.ctx, 7)
        free0 = torch.cuda.mem_get_info()[0]
        for prec in (sie.SIE_PREC_MIXED, sie.SIE_PREC_FP64):
            sie.ilu_apply_noalloc(s.ctx, r, z, 1, prec)
        torch.cuda.synchronize()
        assert sie.sie_query(s.ctx, 7) == held0
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.isfinite(torch.view_as_real(z)).all()
    finally:
        s.close()


@pytest.mark.parametrize("nrhs", [1, 2])
def test_noalloc_ilu_matches_ilu_apply_on_consecutive_calls(nrhs):
    """nrhs = 1 takes the chained single-right-hand-side sweep steps (whose box
    pieces meet through the context's counters), nrhs = 2 the block sweeps;
    two calls in a row share the fixed scratch array."""
    import __graft_entry__ as g
    g.build()
    s = sie.Solver(geo.coated_sphere(**MESH), levels=4)
    try:
        for prec in (sie.SIE_PREC_FP64, sie.SIE_PREC_MIXED):
            tol = 1e-9 if prec == sie.SIE_PREC_FP64 else 1e-5
            for seed in (31, 32):
                r = _rand(s, nrhs, seed)
                z_ref = torch.zeros_like(r)
                z = torch.full_like(r, float("nan"))
                sie.ilu_apply(s.ctx, r, z_ref, nrhs, prec)
                sie.ilu_apply_noalloc(s.ctx, r, z, nrhs, prec)
                torch.cuda.synchronize()
                a, b = z.cpu().numpy(), z_ref.cpu().numpy()
                assert np.all(np.isfinite(a))
                assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)
        # beyond the stated maximum the call is refused before touching buffers
        r = torch.zeros((1, s.ne, 2), dtype=torch.complex128, device="cuda")
        with pytest.raises(sie.SieError) as e:
            sie.ilu_apply_noalloc(s.ctx, r, torch.zeros_like(r), 174763 // s.ne + 1)
        assert e.value.code == 1
    finally:
        s.close()


def test_noalloc_block_on_a_fresh_context_matches_interleaved_path():
    """On a context that never ran a block of right-hand sides the
    allocation-free apply takes the block sweeps on the vectors as they are;
    once ilu_apply has set up the context's interleaved work buffers the
    block sweeps run on right-hand-side-interleaved copies.  Both give the
    same preconditioner (same sums per right-hand side, other order)."""
    import __graft_entry__ as g
    g.build()
    for prec, tol in ((sie.SIE_PREC_FP64, 1e-9), (sie.SIE_PREC_MIXED, 1e-5)):
        s = sie.Solver(geo.coated_sphere(**MESH), levels=4)
        try:
            r = _rand(s, 5, 33)
            z_direct = torch.zeros_like(r)
            sie.ilu_apply_noalloc(s.ctx, r, z_direct, 5, prec)   # no work buffers yet
            torch.cuda.synchronize()
            z_inter = torch.zeros_like(r)
            sie.ilu_apply(s.ctx, r, z_inter, 5, prec)            # allocates them, interleaved sweeps
            torch.cuda.synchronize()
            a, b = z_direct.cpu().numpy(), z_inter.cpu().numpy()
            assert np.all(np.isfinite(a)) and np.all(np.isfinite(b))
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)
        finally:
            s.close()

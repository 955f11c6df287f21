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


def test_noalloc_ilu_matches_ilu_apply_on_consecutive_calls():
    import __graft_entry__ as g
    g.build()
    s = sie.Solver(geo.coated_sphere(5, 3, 0.75, 0.5, 2.56, 4.0), levels=4)
    try:
        for prec in (sie.SIE_PREC_FP64, sie.SIE_PREC_MIXED):
            for seed in (31, 32):          # two calls in a row share the scratch array
                r = torch.from_numpy(geo.random_coefficients(2 * s.ne, 2, seed=seed).reshape(2, s.ne, 2)).cuda()
                z_ref = torch.zeros_like(r)
                z = torch.full_like(r, float("nan"))
                sie.ilu_apply(s.ctx, r, z_ref, 2, prec)
                sie.ilu_apply_noalloc(s.ctx, r, z, 2, prec)
                torch.cuda.synchronize()
                a, b = z.cpu().numpy(), z_ref.cpu().numpy()
                assert np.all(np.isfinite(a))
                assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)
        # beyond the stated maximum the call is refused before touching buffers
        r = torch.zeros((1, s.ne, 2), dtype=torch.complex128, device="cuda")
        with pytest.raises(sie.SieError) as e:
            sie.ilu_apply_noalloc(s.ctx, r, torch.zeros_like(r), 174763 // s.ne + 1)
        assert e.value.code == 1
    finally:
        s.close()

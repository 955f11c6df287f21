"""Tile shapes of the block-RHS kernels and their autotuner.

Every tile shape computes the same product: the near-field, ILU and receive
block sizes and the split of the interpolation and anterpolation by source
keep each right-hand side's summation order, so their results are identical
bit for bit; the M2L forms and the tensor-core aggregation
change the order or the operand split, so they agree to FP32 rounding (1e-5
of the product).  The autotuner picks valid values, keeps them in the
context and writes them to a file that another context reads back."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1704_06862_gb300 as sie  # noqa: E402
from paper_1704_06862_gb300 import geometry as geo  # noqa: E402

MESH = geo.coated_sphere(12, 8, 0.75, 0.5, 2.56, 4.0)
R = 24


@pytest.fixture(scope="module")
def solver():
    import __graft_entry__ as g
    g.build()
    s = sie.Solver(MESH, levels=4)
    yield s
    s.close()


def _x(s):
    return torch.from_numpy(geo.random_coefficients(2 * s.ne, R, seed=5).reshape(R, s.ne, 2)).cuda()


def _prod(s, x, parts=3):
    y = torch.zeros_like(x)
    sie.sie_matvec_parts(s.ctx, x, y, R, sie.SIE_PREC_MIXED, parts)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _ilu(s, x):
    z = torch.zeros_like(x)
    sie.ilu_apply(s.ctx, x, z, R, sie.SIE_PREC_MIXED)
    torch.cuda.synchronize()          # the library works on its own stream
    return z.cpu().numpy()


def _reset(s):
    sie.apply_tuning(s.ctx, {"near_rb": 0, "ilu_rb": 0, "aggregation": 0, "receive_rb": 0, "m2l": -1,
                             "receive_tc": -1})
    sie.sie_set_param(s.ctx, 2, 16)
    sie.sie_set_param(s.ctx, 10, -1)


def test_tile_shapes_give_the_same_product(solver):
    s = solver
    x = _x(s)
    try:
        _reset(s)
        ref = _prod(s, x)
        near_ref = _prod(s, x, 1)
        for rb in (4, 8, 16):
            sie.sie_set_param(s.ctx, 4, rb)
            assert np.array_equal(_prod(s, x, 1), near_ref)
        _reset(s)
        z_ref = _ilu(s, x)
        for rb in (4, 8, 16):
            sie.sie_set_param(s.ctx, 5, rb)
            assert np.array_equal(_ilu(s, x), z_ref)
        _reset(s)
        sie.sie_set_param(s.ctx, 7, 1)                 # the same M2L form for every receive size
        far_ref = _prod(s, x, 2)
        for rb in (1, 2, 4):
            sie.sie_set_param(s.ctx, 6, rb)
            assert np.array_equal(_prod(s, x, 2), far_ref)
        sie.sie_set_param(s.ctx, 6, 0)
        for split in (0, 1):
            sie.sie_set_param(s.ctx, 10, split)
            assert np.array_equal(_prod(s, x, 2), far_ref)
        scale = np.linalg.norm(ref)
        for m2l in (0, 1, 2):
            for agg in (0, 16):
                for rtc in (0, 16):
                    _reset(s)
                    sie.sie_set_param(s.ctx, 7, m2l)
                    sie.sie_set_param(s.ctx, 2, 2 if agg else 0)
                    sie.sie_set_param(s.ctx, 3, agg)
                    sie.sie_set_param(s.ctx, 8, rtc)
                    assert np.linalg.norm(_prod(s, x) - ref) < 1e-5 * scale, (m2l, agg, rtc)
    finally:
        _reset(s)


def test_autotune_choices_round_trip(solver, tmp_path):
    s = solver
    x = _x(s)
    path = os.path.join(str(tmp_path), "tuning.json")
    try:
        _reset(s)
        ref = _prod(s, x)
        t = sie.sie_autotune(s.ctx, R, reps=1, path=path)
        print(f"autotune at {R} right-hand sides: {t}")
        assert t["near_rb"] in (4, 8, 16) and t["ilu_rb"] in (4, 8, 16) and t["receive_rb"] in (1, 2, 4)
        assert t["aggregation"] in (0, 16, 32, 64) and t["m2l"] in (0, 1, 2) and t["receive_tc"] in (-1, 0, 16, 32, 64)
        assert all(v > 0 for v in t["ms"])
        assert json.load(open(path)) == t
        tuned = _prod(s, x)
        assert np.linalg.norm(tuned - ref) < 1e-5 * np.linalg.norm(ref)
        # another context reads the file back and computes the same product
        s2 = sie.Solver(MESH, levels=4)
        try:
            sie.apply_tuning(s2.ctx, path)
            assert np.array_equal(_prod(s2, x), tuned)
        finally:
            s2.close()
    finally:
        _reset(s)

"""Parity at the measured workloads' full size (coated sphere, 78 000
unknowns, 5-level MLFMM, the launch configuration bench.py times; plasmonic
coated nanoparticle, 30 720 unknowns, 4-level MLFMM, bench.py's nanoparticle
leg; lossy dielectric cube, 104 976 unknowns, 5-level MLFMM, bench.py's
monostatic sweep; lossy dielectric ellipsoid, 355 488 unknowns, 7-level
MLFMM, bench.py's learned-preconditioner leg; three-layer lens on a slab,
1 189 264 unknowns, five media, 7-level MLFMM, bench.py's lens leg, whose
sample adds junction edges): the product
is checked on rows the oracle computes one by one (dense JMCFIE rows of the
sampled bases against all bases), and the near-field entries of those rows
element by element.

Tolerance on the sampled product rows: relative L2 1e-3 over the sample (the
MLFMM far-field accuracy target); near entries 1e-9."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1704_06862_gb300 as sie  # noqa: E402
from paper_1704_06862_gb300 import geometry as geo  # noqa: E402
from oracle import fill, tree  # noqa: E402
from oracle.rwg import Mesh  # noqa: E402


@pytest.fixture(scope="module", params=[("coated_c2", 5), ("nanoparticle", 4), ("cube_c3", 5), ("ellipsoid_c4", 7),
                                                ("lens_c5", 7)], ids=lambda p: p[0])
def full(request):
    import __graft_entry__ as g
    g.build()
    name, levels = request.param
    mesh = geo.workload(name)
    s = sie.Solver(mesh, levels=levels, digits=3.0)
    m = Mesh(**mesh)
    yield s, m, levels
    s.close()


def test_sampled_rows(full):
    s, m, levels = full
    assert s.ne == m.ne
    rng = np.random.default_rng(2017)
    if m.junction.any():        # five media: dense rows cost five times as much; two junction rows among them
        rows = np.sort(np.concatenate([rng.choice(np.nonzero(~m.junction)[0], 4, replace=False),
                                       rng.choice(np.nonzero(m.junction)[0], 2, replace=False)]))
    else:
        rows = np.sort(rng.choice(m.ne, 8, replace=False))
    Zr = fill.assemble(m, rows=rows)                      # [2 len(rows), 2 ne]
    x = geo.random_coefficients(2 * m.ne, 1, seed=1234)
    ref = Zr @ x[0]
    xd = torch.from_numpy(x.reshape(1, m.ne, 2)).cuda()
    y = torch.zeros_like(xd)
    sie.mlfmm_matvec(s.ctx, xd, y, 1, sie.SIE_PREC_FP64)
    torch.cuda.synchronize()
    got = y.cpu().numpy().reshape(m.ne, 2)[rows].reshape(-1)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"full-size sampled rows ({m.ne} bases): rel L2 {err:.2e}")
    assert err < 1e-3
    # near entries of those rows, element by element
    r, c, v = sie.sie_near_export(s.ctx)
    sel = np.isin(r, rows)
    loc = {e: i for i, e in enumerate(rows)}
    li = np.array([loc[e] for e in r[sel]])
    refb = np.stack([Zr[2 * li + a, 2 * c[sel] + bb] for a in range(2) for bb in range(2)], axis=1)
    assert np.max(np.abs(v[sel] - refb)) < 1e-9 * np.max(np.abs(Zr))
    ijk = tree.box_coords(m, levels)
    near = np.abs(ijk[rows][:, None, :] - ijk[None, :, :]).max(axis=2) <= 1
    assert sel.sum() == near.sum()


def test_ilu_schedules_agree_at_full_size(full):
    """The single-RHS ILU(0) apply in one persistent cooperative launch (grid
    barriers between the 15 colour steps) against one launch per step: same
    items, same arithmetic order, so the results are identical bit for bit,
    in both precisions; at this size boxes are split into several pieces
    (the partial sums meet through the per-box counters).  The FP32 apply is
    within 1e-4 of the FP64 one."""
    s, m, levels = full
    x = torch.from_numpy(geo.random_coefficients(2 * m.ne, 1, seed=77).reshape(1, m.ne, 2)).cuda()
    out = {}
    try:
        for sched in (1, 0):
            sie.sie_set_param(s.ctx, 1, sched)
            for prec in (sie.SIE_PREC_FP64, sie.SIE_PREC_MIXED):
                z = torch.full_like(x, float("nan"))
                sie.ilu_apply(s.ctx, x, z, 1, prec)
                sie.sie_device_status(s.ctx)
                out[sched, prec] = z.cpu().numpy()
    finally:
        sie.sie_set_param(s.ctx, 1, 1)
    for prec in (sie.SIE_PREC_FP64, sie.SIE_PREC_MIXED):
        assert np.all(np.isfinite(out[0, prec]))
        assert np.array_equal(out[0, prec], out[1, prec])
    a, b = out[0, sie.SIE_PREC_MIXED], out[0, sie.SIE_PREC_FP64]
    assert np.linalg.norm(a - b) < 1e-4 * np.linalg.norm(b)

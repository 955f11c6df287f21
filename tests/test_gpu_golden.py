"""MLFMM accuracy and solution parity on stored oracle results.

The expected values in tests/golden/*.npz were written by
tests/golden/make_golden.py, which calls only the CPU oracle (dense JMCFIE
fill, dense product, dense LU, far field, Mie series).

Tolerances:
* near part of the product: same integrals on both sides -> 1e-12.
* whole product, FP64 MLFMM: relative L2 1e-3 (the far-field accuracy target).
* FP32 (mixed) product vs FP64 product: 1e-4; the true-residual product of
  the mixed form (FP64 near field, FP32 far field into the FP64 product):
  near part 1e-12, whole product vs FP64 1e-5.
* mixed-form solves: the FP64-operator residual of the returned currents
  within 1.5 x tol at tol 1e-6 (there the true residual uses the whole FP64
  operator) and within 1.05 x tol at tol 1e-4 (FP64 near field + FP32 far
  field, a few 1e-6 from the FP64 operator).
* currents solved to 1e-6 vs dense LU: 1e-3 relative L2.
* RCS of the solved currents vs the oracle RCS of the LU currents: 0.2 dB on
  angles within 30 dB of the peak.
"""
import importlib.util
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1704_06862_gb300 as sie  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
make_golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(make_golden)

NAMES = [n for n in make_golden.CASES if os.path.exists(os.path.join(HERE, "golden", f"{n}.npz"))]

# Solved currents against dense LU: 1e-3, except the cube.  Its faces are flat
# and aligned with the octree, so many source pairs sit at the worst case of
# the one-buffer well-separation rule (sources at box corners, centres two
# boxes apart), where the addition theorem converges only as about 0.87^L:
# its product still meets 1e-3 (4.9e-4) but more directions (d0 = 4) or a
# finer mesh leave that error unchanged, and the cube system's conditioning
# amplifies it about 3.7 times in the currents (measured 1.8e-3; its RCS is
# within 0.013 dB of the oracle's).  The split sphere's disk lies in the
# octree's z = 0 box faces, the same worst case: product 8.2e-4, unchanged
# with d0 = 4 (7.8e-4), currents 1.1e-3, RCS within 0.005 dB of the oracle's.
CURRENTS_TOL = {"cube_small": 2.5e-3, "split_sphere": 2e-3}


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module", params=NAMES)
def case(request):
    name = request.param
    d = dict(np.load(os.path.join(HERE, "golden", f"{name}.npz")))
    mesh = make_golden.CASES[name]["mesh"]()
    s = sie.Solver(mesh, levels=int(d["levels"]), digits=float(make_golden.CASES[name].get("digits", 3.0)))
    assert s.ne == int(d["ne"])
    yield name, s, d
    s.close()


def _dev(a, ne):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1, ne, 2)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().reshape(t.shape[0], -1)


def test_product_near_far_and_mixed(case):
    name, s, d = case
    x = _dev(d["x"], s.ne)
    y = torch.zeros_like(x)
    sie.sie_matvec_parts(s.ctx, x, y, 2, sie.SIE_PREC_FP64, parts=1)
    assert rel(_host(y), d["y_near"]) < 1e-12
    sie.mlfmm_matvec(s.ctx, x, y, 2, sie.SIE_PREC_FP64)
    y64 = _host(y)
    err = rel(y64, d["y"])
    far_err = rel(y64 - d["y_near"], d["y"] - d["y_near"])
    print(f"{name}: MLFMM product rel L2 {err:.2e}, far part {far_err:.2e}")
    assert err < 1e-3
    sie.mlfmm_matvec(s.ctx, x, y, 2, sie.SIE_PREC_MIXED)
    assert rel(_host(y), y64) < 1e-4
    sie.sie_matvec_parts(s.ctx, x, y, 2, sie.SIE_PREC_NEAR64, parts=1)
    assert rel(_host(y), d["y_near"]) < 1e-12
    sie.mlfmm_matvec(s.ctx, x, y, 2, sie.SIE_PREC_NEAR64)
    e64 = rel(_host(y), y64)
    print(f"{name}: true-residual product (FP64 near, FP32 far) vs FP64 product rel L2 {e64:.2e}")
    assert e64 < 1e-5


@pytest.mark.parametrize("prec", [sie.SIE_PREC_FP64, sie.SIE_PREC_MIXED])
def test_solution_and_rcs(case, prec):
    name, s, d = case
    b = torch.zeros((1, s.ne, 2), dtype=torch.complex128, device="cuda")
    sie.sie_plane_wave_rhs(s.ctx, [[0.0, 0.0, 0.0, 1.0]], b)
    assert rel(_host(b), d["b"]) < 1e-12
    x = torch.zeros_like(b)
    st = sie.gmres_solve(s.ctx, b, x, 1, restart=50, max_iters=1000, tol=1e-6, prec=prec, precond=1)
    assert st[0]["converged"]
    xs = _host(x)[0]
    err = rel(xs, d["xs"])
    rcs = sie.rcs_farfield(s.ctx, x, 1, d["obs"])[0]
    ok = d["rcs"][:, 0] > d["rcs"][:, 0].max() * 1e-3
    db = np.abs(10 * np.log10(rcs[ok, 0]) - 10 * np.log10(d["rcs"][ok, 0]))
    mie_db = np.abs(10 * np.log10(rcs[:, 0]) - 10 * np.log10(d["mie"]))
    print(f"{name} prec={prec}: iters {st[0]['iters']}, currents rel err {err:.2e}, RCS vs oracle max "
          f"{db.max():.3f} dB, vs Mie mean {mie_db.mean():.3f} dB")
    assert err < CURRENTS_TOL.get(name, 1e-3)
    assert db.max() < 0.2
    if prec == sie.SIE_PREC_MIXED:
        y = torch.zeros_like(b)
        sie.mlfmm_matvec(s.ctx, x, y, 1, sie.SIE_PREC_FP64)
        r64 = rel(_host(y), _host(b))
        print(f"{name}: FP64-operator residual {r64:.2e} (solver's {st[0]['rel_residual']:.2e})")
        assert r64 < 1.5e-6


def test_batched_solve_equals_single_solves(case):
    """A block of right-hand sides (monostatic incidences) solved together
    gives the currents of the individual solves."""
    name, s, d = case
    if name != "sphere_c1":
        pytest.skip("one case suffices")
    inc = np.array([[0.0, 0.0, 0.0, 1.0], [0.9, 0.0, 0.0, 1.0], [2.2, 0.0, 0.0, 1.0]])
    b = torch.zeros((3, s.ne, 2), dtype=torch.complex128, device="cuda")
    sie.sie_plane_wave_rhs(s.ctx, inc, b)
    xb = torch.zeros_like(b)
    st = sie.gmres_solve(s.ctx, b, xb, 3, restart=50, max_iters=500, tol=1e-8, prec=sie.SIE_PREC_FP64, precond=1)
    assert all(t["converged"] for t in st)
    xb = _host(xb)
    for r in range(3):
        x1 = torch.zeros((1, s.ne, 2), dtype=torch.complex128, device="cuda")
        sie.gmres_solve(s.ctx, b[r:r + 1].contiguous(), x1, 1, restart=50, max_iters=500, tol=1e-8,
                        prec=sie.SIE_PREC_FP64, precond=1)
        assert rel(xb[r], _host(x1)[0]) < 1e-6


def test_eager_steps_equal_graph_steps(case):
    """Krylov steps launched eagerly give the same iterations and currents as
    the captured-graph steps (same kernels in the same order)."""
    name, s, d = case
    if name != "coated_r075":
        pytest.skip("one case suffices")
    b = torch.zeros((1, s.ne, 2), dtype=torch.complex128, device="cuda")
    sie.sie_plane_wave_rhs(s.ctx, [[0.0, 0.0, 0.0, 1.0]], b)
    out = []
    for graphs in (True, False):
        x = torch.zeros_like(b)
        st = sie.gmres_solve(s.ctx, b, x, 1, restart=50, max_iters=1000, tol=1e-6, prec=sie.SIE_PREC_MIXED,
                             precond=1, graphs=graphs)
        out.append((st[0]["iters"], _host(x)))
    assert out[0][0] == out[1][0]
    assert rel(out[0][1], out[1][1]) < 1e-12


def test_graph_captured_step_product_matches_oracle(case):
    """The product inside a captured Krylov-step graph, checked against the
    dense oracle matrix on every stored case (including the one with the
    most leaf directions, where aggregation takes four directions per
    thread).  One FGMRES step without a preconditioner, right-hand side the
    stored random vector u with its stored dense product Zu, from x0 = 0,
    returns x1 = alpha u with alpha = (Zu)^H u / |Zu|^2, the minimiser of
    |u - alpha Z u|.  A relative product error e moves alpha by at most
    about 2e, hence the 2e-3 bound for the 1e-3 product accuracy."""
    name, s, d = case
    u, Zu = d["x"][0], d["y"][0]
    alpha = np.vdot(Zu, u) / np.vdot(Zu, Zu)
    for prec in (sie.SIE_PREC_FP64, sie.SIE_PREC_MIXED):
        rhs = _dev(u, s.ne)
        x = torch.zeros_like(rhs)
        st = sie.gmres_solve(s.ctx, rhs, x, 1, restart=1, max_iters=1, tol=1e-12, prec=prec, precond=0,
                             check=False, graphs=True)
        assert st[0]["iters"] == 1 and not st[0]["converged"]
        err = rel(_host(x)[0], alpha * u)
        print(f"{name} prec={prec}: one graph-launched step, |x1 - alpha u| / |alpha u| = {err:.2e}")
        assert err < 2e-3


def test_monostatic_block_sweep(case):
    """Monostatic sweep as one block of right-hand sides (the cube case): the
    theta-theta RCS of every incidence against the oracle's dense-LU values
    (0.1 dB: MLFMM and mixed-precision error only), and the mirror symmetry
    theta_i <-> pi - theta_i of the body within 0.05 dB."""
    name, s, d = case
    if "mono_inc" not in d:
        pytest.skip("stored monostatic values only for the cube case")
    inc = d["mono_inc"]
    R = len(inc)
    b = torch.zeros((R, s.ne, 2), dtype=torch.complex128, device="cuda")
    sie.sie_plane_wave_rhs(s.ctx, inc, b)
    x = torch.zeros_like(b)
    st = sie.gmres_solve(s.ctx, b, x, R, restart=50, max_iters=1000, tol=1e-6, prec=sie.SIE_PREC_MIXED, precond=1)
    assert all(t["converged"] for t in st)
    obs = np.stack([inc[:, 0], inc[:, 1]], axis=1)
    rcs = sie.rcs_farfield_prec(s.ctx, x, R, obs, sie.SIE_PREC_MIXED)
    mono = 10 * np.log10(rcs[np.arange(R), np.arange(R), 0])
    ref = 10 * np.log10(d["mono_rcs"])
    print(f"{name}: monostatic block of {R}: max {np.abs(mono - ref).max():.4f} dB from the oracle, "
          f"mirror {np.abs(mono - mono[::-1]).max():.4f} dB")
    assert np.abs(mono - ref).max() < 0.1
    assert np.abs(mono - mono[::-1]).max() < 0.05


def test_tensor_core_aggregation(case):
    """Leaf aggregation as split-BF16 tensor-core products (tcgen05, FP32
    accumulator in tensor memory) for blocks of right-hand sides, against
    the FP32 SIMT aggregation on the same block, for passes of 16, 32 and 64
    right-hand sides and a ragged block (40 = 32 + 8).  The three BF16 parts
    of each operand carry FP32-level precision, so the difference of the far
    parts must stay within 1e-5 of the whole product (the FP32 rounding
    level of the mixed form; a two-part split reached 2e-4 on a cube, the
    diagonal translations amplifying the operands' error).  The whole
    product of the first two columns within 1e-3 of the stored dense oracle
    product and of all columns within 1e-4 of the FP64 product."""
    name, s, d = case
    if name not in ("coated_r075", "cube_small", "nanoparticle", "lens_small"):
        pytest.skip("three media, sharp edges, the most leaf directions and junction edges suffice")
    R = 40
    ph = np.exp(1j * np.linspace(0.0, 2.0, R // 2))
    X = np.concatenate([d["x"] * p for p in ph])          # [R, 2 ne]; rows 0, 1 are the stored vectors
    x = _dev(X, s.ne)

    def product(tc_min, rb, parts):
        sie.sie_set_param(s.ctx, 2, tc_min)
        sie.sie_set_param(s.ctx, 3, rb)
        y = torch.zeros_like(x)
        sie.sie_matvec_parts(s.ctx, x, y, R, sie.SIE_PREC_MIXED, parts)
        return _host(y)

    try:
        whole = np.linalg.norm(product(0, 0, 3))
        ref = product(0, 0, 2)                               # far part, SIMT aggregation
        for rb in (16, 32, 64):
            got = product(16, rb, 2)
            diff = np.linalg.norm(got - ref)
            print(f"{name}: tensor-core aggregation, {rb} right-hand sides per pass: far part rel diff "
                  f"{diff / np.linalg.norm(ref):.2e}, relative to the product {diff / whole:.2e}")
            assert np.all(np.isfinite(got)) and diff < 1e-5 * whole
        sie.sie_set_param(s.ctx, 2, 16)
        sie.sie_set_param(s.ctx, 3, 0)
        y = torch.zeros_like(x)
        sie.mlfmm_matvec(s.ctx, x, y, R, sie.SIE_PREC_MIXED)
        y64 = torch.zeros_like(x)
        sie.mlfmm_matvec(s.ctx, x, y64, R, sie.SIE_PREC_FP64)
        yh = _host(y)
        assert rel(yh[:2], d["y"]) < 1e-3
        assert rel(yh, _host(y64)) < 1e-4
    finally:
        sie.sie_set_param(s.ctx, 2, 16)
        sie.sie_set_param(s.ctx, 3, 0)


def test_tensor_core_receive(case):
    """Leaf receive as split-BF16 tensor-core products (tcgen05; the receive
    patterns bulk-copied, the box's combined fields formed per chunk by the
    threads) for blocks of right-hand sides, against the SIMT receive on the
    same block: the far parts within 1e-5 of the whole product for passes of
    16, 32 and 64 right-hand sides and a ragged block (40); with both leaf
    contractions on the tensor cores the whole product of the first two
    columns within 1e-3 of the stored dense oracle product and of all
    columns within 1e-4 of the FP64 product."""
    name, s, d = case
    if name not in ("coated_r075", "cube_small", "nanoparticle", "lens_small"):
        pytest.skip("three media, sharp edges, the most leaf directions and junction edges suffice")
    R = 40
    ph = np.exp(1j * np.linspace(0.0, 2.0, R // 2))
    X = np.concatenate([d["x"] * p for p in ph])
    x = _dev(X, s.ne)

    def product(rec_tc, parts):
        sie.sie_set_param(s.ctx, 8, rec_tc)
        y = torch.zeros_like(x)
        sie.sie_matvec_parts(s.ctx, x, y, R, sie.SIE_PREC_MIXED, parts)
        return _host(y)

    try:
        sie.sie_set_param(s.ctx, 2, 0)                       # SIMT aggregation: isolate the receive
        whole = np.linalg.norm(product(0, 3))
        ref = product(0, 2)
        for rb in (16, 32, 64):
            got = product(rb, 2)
            diff = np.linalg.norm(got - ref)
            print(f"{name}: tensor-core receive, {rb} right-hand sides per pass: far part rel diff "
                  f"{diff / np.linalg.norm(ref):.2e}, relative to the product {diff / whole:.2e}")
            assert np.all(np.isfinite(got)) and diff < 1e-5 * whole
        sie.sie_set_param(s.ctx, 2, 16)
        sie.sie_set_param(s.ctx, 8, 32)
        y = torch.zeros_like(x)
        sie.mlfmm_matvec(s.ctx, x, y, R, sie.SIE_PREC_MIXED)
        y64 = torch.zeros_like(x)
        sie.mlfmm_matvec(s.ctx, x, y64, R, sie.SIE_PREC_FP64)
        yh = _host(y)
        assert rel(yh[:2], d["y"]) < 1e-3
        assert rel(yh, _host(y64)) < 1e-4
    finally:
        sie.sie_set_param(s.ctx, 2, 16)
        sie.sie_set_param(s.ctx, 8, -1)


def test_block_product_equals_single_products(case):
    """A block of 9 right-hand sides (the translations then run by sibling
    groups) gives the products of the right-hand sides one at a time (per
    target box), in both precisions; on a layered body and on one with
    junction edges (bases in more than two media)."""
    name, s, d = case
    if name not in ("coated_r075", "lens_small"):
        pytest.skip("two cases suffice")
    x = np.concatenate([d["x"]] * 5)[:9] * np.arange(1, 10)[:, None]
    xb = _dev(x, s.ne)
    for prec, tol in ((sie.SIE_PREC_FP64, 1e-12), (sie.SIE_PREC_MIXED, 1e-5)):
        yb = torch.zeros_like(xb)
        sie.mlfmm_matvec(s.ctx, xb, yb, 9, prec)
        yb = _host(yb)
        for r in (0, 4, 8):
            y1 = torch.zeros_like(xb[r:r + 1])
            sie.mlfmm_matvec(s.ctx, xb[r:r + 1].contiguous(), y1, 1, prec)
            assert rel(yb[r], _host(y1)[0]) < tol


def test_residual_operator_choice(case):
    """At tol 1e-4 the mixed form's true residual uses the FP64 near field +
    FP32 far field (restarts every 10 iterations, so it decides several
    times): it takes the iterations of the whole-FP64 residual to within two,
    and the currents it returns meet the tolerance under the FP64 operator
    too (within 5 %)."""
    name, s, d = case
    if name != "coated_r075":
        pytest.skip("one case suffices")
    b = torch.zeros((1, s.ne, 2), dtype=torch.complex128, device="cuda")
    sie.sie_plane_wave_rhs(s.ctx, [[0.0, 0.0, 0.0, 1.0]], b)
    its = []
    for full in (True, False):
        x = torch.zeros_like(b)
        st = sie.gmres_solve(s.ctx, b, x, 1, restart=10, max_iters=1000, tol=1e-4, prec=sie.SIE_PREC_MIXED,
                             precond=1, residual_far_fp64=full)
        assert st[0]["converged"] and st[0]["restarts"] >= 1
        its.append(st[0]["iters"])
        y = torch.zeros_like(b)
        sie.mlfmm_matvec(s.ctx, x, y, 1, sie.SIE_PREC_FP64)
        assert rel(_host(y), _host(b)) < 1.05e-4
    assert abs(its[0] - its[1]) <= 2


@pytest.mark.parametrize("method", [sie.SOLVE_BICGSTAB, sie.SOLVE_CGS])
def test_bicgstab_cgs_solution(case, method):
    """The paper's solvers with ILU(0) on the MLFMM operator (mixed precision,
    FP64 true residual at the end) reach the dense-LU currents."""
    name, s, d = case
    b = torch.zeros((1, s.ne, 2), dtype=torch.complex128, device="cuda")
    sie.sie_plane_wave_rhs(s.ctx, [[0.0, 0.0, 0.0, 1.0]], b)
    x = torch.zeros_like(b)
    st = sie.gmres_solve(s.ctx, b, x, 1, max_iters=1000, tol=1e-6, prec=sie.SIE_PREC_MIXED, precond=1,
                         method=method)
    assert st[0]["converged"]
    assert rel(_host(x)[0], d["xs"]) < CURRENTS_TOL.get(name, 1e-3)


@pytest.fixture(scope="module")
def forms():
    return dict(np.load(os.path.join(HERE, "golden", "sphere_c1_forms.npz")))


@pytest.mark.parametrize("form,fname", [(sie.FORM_JMCFIE, "jmcfie"), (sie.FORM_CTF, "ctf"),
                                        (sie.FORM_CNF, "cnf"), (sie.FORM_PMCHWT, "pmchwt"),
                                        (sie.FORM_ICTF, "ictf")])
def test_formulation_variants(forms, form, fname):
    """Each formulation (fill weights, folded receive patterns, excitation)
    against the oracle's dense matrix of that formulation: near part exactly,
    MLFMM product to 1e-3, excitation exactly, solved currents to 1e-3 for
    JMCFIE and 5e-3 for the variants (the product's 1e-3-level error grows
    with the condition number, 2-4 times JMCFIE's for CTF, CNF, PMCHWT and
    ICTF on this sphere), and their RCS to 0.2 dB.  ICTF's row weights act on
    every product part and on the excitation."""
    d = forms
    s = sie.Solver(make_golden.CASES["sphere_c1"]["mesh"](), levels=int(d["levels"]), formulation=form)
    try:
        assert s.ne == int(d["ne"])
        x = _dev(d["x"], s.ne)
        y = torch.zeros_like(x)
        sie.sie_matvec_parts(s.ctx, x, y, 2, sie.SIE_PREC_FP64, parts=1)
        assert rel(_host(y), d[f"y_near_{fname}"]) < 1e-12
        sie.mlfmm_matvec(s.ctx, x, y, 2, sie.SIE_PREC_FP64)
        assert rel(_host(y), d[f"y_{fname}"]) < 1e-3
        b = torch.zeros((1, s.ne, 2), dtype=torch.complex128, device="cuda")
        sie.sie_plane_wave_rhs(s.ctx, [[0.0, 0.0, 0.0, 1.0]], b)
        assert rel(_host(b), d[f"b_{fname}"]) < 1e-12
        xs = torch.zeros_like(b)
        st = sie.gmres_solve(s.ctx, b, xs, 1, restart=50, max_iters=3000, tol=1e-6, prec=sie.SIE_PREC_MIXED,
                             precond=1)
        assert st[0]["converged"]
        assert rel(_host(xs)[0], d[f"xs_{fname}"]) < (1e-3 if form == sie.FORM_JMCFIE else 5e-3)
        rcs = sie.rcs_farfield(s.ctx, xs, 1, d["obs"])[0]
        ref = d[f"rcs_{fname}"]
        ok = ref[:, 0] > ref[:, 0].max() * 1e-3
        assert np.abs(10 * np.log10(rcs[ok, 0]) - 10 * np.log10(ref[ok, 0])).max() < 0.2
    finally:
        s.close()

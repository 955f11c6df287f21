"""Write the stored expected values used by the GPU parity tests.

Every value here is computed by the CPU oracle (``oracle/``) alone, on seeded
synthetic inputs from ``paper_1704_06862_gb300.geometry``; nothing comes from
the CUDA path.  Run:  python tests/golden/make_golden.py [name ...]

Cases
  sphere_c1    eps_r = 4 sphere, radius 0.5 lambda0, geodesic nu = 8
               (1280 triangles, 3840 unknowns); 3-level tree (leaf 0.25).
  sphere_r1    eps_r = 4 sphere, radius 1.0 lambda0, nu = 12 (8640 unknowns);
               4-level tree (leaf 0.25): exercises interpolation/anterpolation.
  sphere_lossy eps_r = 6 - 0.6j sphere (complex wavenumber), radius 0.5, nu = 8.
  coated_r075  coated sphere, core 0.5 (eps 4), shell 0.75 (eps 2.56), nu 12/8
               (12480 unknowns, three media); 4-level tree (leaf 0.1875).
  nanoparticle plasmonic coated sphere: core 230/550 (eps -10 - 0.8j), shell
               250/550 (eps -5 - 2j), nu 6/6 (4320 unknowns); 3-level tree.
               Its Mie series is also the reference of the finer
               nanoparticle workload (same radii, media and angles).
  cube_small   lossy dielectric cube (eps 6 - 0.6j), edge 0.6 lambda0, 14 x 14
               squares per face (7056 unknowns); 3-level tree; no Mie series
               (stored as NaN); also the monostatic theta-theta RCS of 8
               theta-polarised incidences theta_i in [0, pi], phi = 0.
  ellipsoid_small  lossy dielectric ellipsoid (eps 3 - 0.2j), semi-axes 1.0 x
               0.5 x 0.25 lambda0, cube-sphere mesh (2688 unknowns); 4-level
               tree; no Mie series; monostatic RCS of 8 incidences as above.
Stored: seeded x (2 columns), y = Z x, y_near = Z_near x (touching-box
pattern), plane-wave excitation b, dense-LU solution, bistatic RCS of that
solution at 361 angles, and the Mie series at the same angles.

  split_sphere   a sphere cut into two regions of equal eps by the plane
                 z = 0: 24 junction edges on the equator, 960 RWG edges.
  lens_small     the lens-on-slab body at a size the dense oracle solves:
                 five media, junction edges on three circles.
  sphere_c1_forms  the sphere_c1 case in the five formulations (JMCFIE, CTF,
                 CNF, PMCHWT, ICTF): per formulation the products y and y_near of
                 the seeded x, the excitation b, the LU currents and their RCS.
  mie_coated_c2  the coated-sphere Mie series alone (core 1.0 lambda0, eps 4;
                 shell 1.5 lambda0, eps 2.56; x-polarised incidence along -z),
                 361 bistatic angles in phi = 0: the reference of the benchmark
                 workload's RCS (78 000 unknowns, too large for a dense solve).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from paper_1704_06862_gb300 import geometry as geo  # noqa: E402
from oracle import farfield, fill, mie, solvers, tree  # noqa: E402
from oracle.rwg import Mesh  # noqa: E402

CASES = {
    "sphere_c1": dict(mesh=lambda: geo.homogeneous_sphere(nu=8, radius=0.5, eps_r=4.0), levels=3, radius=0.5),
    "sphere_r1": dict(mesh=lambda: geo.homogeneous_sphere(nu=12, radius=1.0, eps_r=4.0), levels=4, radius=1.0),
    "sphere_lossy": dict(mesh=lambda: geo.homogeneous_sphere(nu=8, radius=0.5, eps_r=6.0 - 0.6j), levels=3,
                         radius=0.5, eps=6.0 - 0.6j),
    "coated_r075": dict(mesh=lambda: geo.coated_sphere(12, 8, 0.75, 0.5, 2.56, 4.0), levels=4, coated=(0.5, 0.75)),
    # plasmonic coated nanoparticle: silver-like core (230 nm) in a gold-like
    # shell (20 nm) at 545 THz, scaled to lambda0 = 550 nm; permittivities are
    # assumed round values with negative real parts (e^{+jwt}, loss eps'' < 0)
    "nanoparticle": dict(mesh=lambda: geo.coated_sphere(6, 6, 250 / 550, 230 / 550, geo.NANO_EPS_SHELL,
                                                        geo.NANO_EPS_CORE),
                         levels=3, coated=(230 / 550, 250 / 550), eps=(geo.NANO_EPS_CORE, geo.NANO_EPS_SHELL)),
    # lossy dielectric cube (eps 6 - 0.6j, the material of the cube workload),
    # edge 0.6 lambda0, 14 x 14 squares per face: sharp edges and corners, no
    # closed form (no Mie series); monostatic RCS of 8 incidences stored
    # (triangles at most 0.3 of the leaf box edge, as in the cube workload: on a
    # coarser mesh the RWG supports overhang their boxes and the far part of
    # the product loses accuracy whatever the number of directions)
    "cube_small": dict(mesh=lambda: geo.workload("cube_small"), levels=3, mie=False, mono=8),
    # tri-axial lossy dielectric ellipsoid (eps 3 - 0.2j, the material of the
    # ellipsoid workload), semi-axes 1.0 x 0.5 x 0.25 lambda0, cube-sphere mesh
    "ellipsoid_small": dict(mesh=lambda: geo.workload("ellipsoid_small"), levels=4, mie=False, mono=8),
    # sphere cut by the plane z = 0 into two regions of the same eps: junction
    # edges on the equator (upper hemisphere 0|1, lower 0|2, disk 1|2); its
    # exterior field is that of the uncut sphere (Mie series of radius 0.3, eps 4)
    "split_sphere": dict(mesh=lambda: geo.split_sphere(12, 24, 3, 0.3, 4.0, 4.0), levels=3, radius=0.3),
    # three-layer hemispherical lens (eps 10.2 / 4.5 / 2.2, radii 0.15 / 0.3 /
    # 0.6 lambda0) on a 1.4 x 1.4 x 0.2 lambda0 slab of eps 2.2: five media,
    # junction edges on the three base circles; no closed form
    "lens_small": dict(mesh=lambda: geo.workload("lens_small"),
                       levels=3, mie=False),
}


def make(name):
    spec = CASES[name]
    t0 = time.time()
    m = Mesh(**spec["mesh"]())
    Z = fill.assemble(m)
    x = geo.random_coefficients(2 * m.ne, 2, seed=1234)
    y = (Z @ x.T).T
    mask = tree.near_mask(m, spec["levels"])
    Zn = Z * np.repeat(np.repeat(mask, 2, 0), 2, 1)
    y_near = (Zn @ x.T).T
    inc = np.array([[0.0, 0.0, 0.0, 1.0]])
    b = fill.rhs(m, inc)
    xs = solvers.lu_solve(Z, b[0])
    obs = geo.bistatic_angles(361)
    rcs = farfield.rcs(m, xs[None], obs)[0]
    extra = {}
    if not spec.get("mie", True):
        ref = np.full(len(obs), np.nan)
    elif "coated" in spec:
        ec, es = spec.get("eps", (4.0, 2.56))
        ref = mie.coated_bistatic(spec["coated"][0], spec["coated"][1], ec, es, obs[:, 0])
    else:
        ref = mie.sphere_bistatic(spec["radius"], spec.get("eps", 4.0), obs[:, 0])
    if "mono" in spec:
        # monostatic sweep: theta-polarised incidences theta_i in [0, pi], phi = 0, received theta-theta
        minc = geo.monostatic_incidences(spec["mono"])
        X = np.stack([solvers.lu_solve(Z, bb) for bb in fill.rhs(m, minc)])
        R = farfield.rcs(m, X, np.stack([minc[:, 0], minc[:, 1]], axis=1))
        extra = dict(mono_inc=minc, mono_rcs=np.array([R[i, i, 0] for i in range(len(minc))]))
    np.savez_compressed(os.path.join(HERE, f"{name}.npz"), x=x, y=y, y_near=y_near, b=b, xs=xs, obs=obs,
                        rcs=rcs, mie=ref, levels=spec["levels"], ne=m.ne, **extra)
    err = np.abs(10 * np.log10(rcs[:, 0]) - 10 * np.log10(ref))
    print(f"{name}: ne={m.ne} fill+solve {time.time() - t0:.0f}s  RCS vs Mie mean {err.mean():.3f} dB, "
          f"max {err.max():.3f} dB")


def make_forms():
    spec = CASES["sphere_c1"]
    t0 = time.time()
    m = Mesh(**spec["mesh"]())
    Zs = fill.assemble_variants(m)
    x = geo.random_coefficients(2 * m.ne, 2, seed=1234)
    mask = tree.near_mask(m, spec["levels"])
    mk = np.repeat(np.repeat(mask, 2, 0), 2, 1)
    inc = np.array([[0.0, 0.0, 0.0, 1.0]])
    obs = geo.bistatic_angles(361)
    out = dict(x=x, obs=obs, levels=spec["levels"], ne=m.ne)
    for f, Z in Zs.items():
        b = fill.rhs(m, inc, formulation=f)
        xs = solvers.lu_solve(Z, b[0])
        out[f"y_{f}"] = (Z @ x.T).T
        out[f"y_near_{f}"] = ((Z * mk) @ x.T).T
        out[f"b_{f}"] = b
        out[f"xs_{f}"] = xs
        out[f"rcs_{f}"] = farfield.rcs(m, xs[None], obs)[0]
    np.savez_compressed(os.path.join(HERE, "sphere_c1_forms.npz"), **out)
    print(f"sphere_c1_forms: ne={m.ne} {time.time() - t0:.0f}s")


def make_mie_coated_c2():
    obs = geo.bistatic_angles(361)
    ref = mie.coated_bistatic(1.0, 1.5, 4.0, 2.56, obs[:, 0])
    np.savez_compressed(os.path.join(HERE, "mie_coated_c2.npz"), obs=obs, mie=ref)
    print(f"mie_coated_c2: {len(obs)} angles, peak {10 * np.log10(ref.max()):.2f} dBsm")


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(CASES) + ["sphere_c1_forms", "mie_coated_c2"]):
        if n == "mie_coated_c2":
            make_mie_coated_c2()
        elif n == "sphere_c1_forms":
            make_forms()
        else:
            make(n)

"""CPU FP64 oracle for the JMCFIE / RWG surface-integral method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
CUDA library never calls it and shares no code, header, table or helper with
it; the only module both sides import is the seeded input generator
``paper_1704_06862_gb300.geometry``.

What it computes (plain definitions, no acceleration):

* RWG basis on triangle pairs (Eq. 22, Fig. 4)                     -> rwg.py
* dense Galerkin JMCFIE matrix and excitation vector
  (Eqs. 5-11 per medium, combined by Eqs. 12-16; entries Eqs. 15-26) -> fill.py
* analytic potential integrals for singularity extraction            -> potentials.py
* far field and RCS (Eqs. 27-29), plane wave (Eq. 30)               -> farfield.py
* Mie series for homogeneous and coated spheres (Fig. 5, Fig. 10)    -> mie.py
* dense LU, restarted GMRES, ILU(0) on the near-field pattern        -> solvers.py
* octree box assignment, near pattern, colour ordering               -> tree.py

Readings of garbled or silent passages are stated in each function's
docstring.  Parity status: every function is pinned by a
``-m "not gpu"`` test (tests/test_oracle_*.py) except where its docstring says
"parity unpinned".
"""

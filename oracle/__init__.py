"""Plain FP64 CPU oracle for the Shan-Chen droplet/bubble method of
"A Mesoscale Perspective on the Tolman Length" (arXiv:2105.08772).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
reference that the CUDA path is checked against.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import or run it.  The product path (the C-ABI library and
its Python binding) never imports it and shares no code, table or constant
with it.

Everything is numpy float64, written to be read against the paper:

* ``lattice``     -- velocity sets, lattice weights and forcing-stencil weights
                     derived from the isotropy conditions (Sec. II, Eq. (8)).
* ``eos``         -- pseudopotentials psi(n), bulk pressure (Eq. (10)), the
                     critical coupling G_c and the flat-interface coexistence
                     construction.
* ``lbm3d``       -- the D3Q19 BGK + Guo-forcing Shan-Chen step
                     (Eqs. (3)-(8)) and the droplet/bubble initial profile
                     (Eq. (23)).
* ``flat``        -- the flat-interface run (Sec. IV, Eq. (24)) and sigma_0
                     (Eq. (25)).
* ``observables`` -- lattice pressure tensor (Eq. (9)), P_in/P_out, R_e,
                     centre of mass, convergence measures (Sec. IV), the
                     generalised surface tension sigma[R] (Eqs. (21)-(22)),
                     R_s, sigma_s and the Tolman fit (Eqs. (2), (12)).

Parity status of each function is stated in its module docstring; the
3-D transient is pinned by invariants and by the closed forms of linear
acoustics (sound speed from Eq. (10), damping from the lattice viscosity); the
paper prints no field values.
"""

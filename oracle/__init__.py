"""FP64 CPU oracle for the LBGK-LPT bubble-column method (arXiv:1710.07073).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, calls or links anything here, and nothing here imports the product.

The oracle is a plain, slow, obviously-correct restatement of the paper in
numpy float64:

* ``lattice``    D3Q19 velocity set and weights (Eq. 7-8), equilibrium (Eq. 6),
                 moments (Eq. 10), viscosity (Eq. 9), the forcing scheme
                 (Eq. 12-15) and streaming (Eq. 16) with half-way bounce-back
                 walls (Sec. 3.3).
* ``mapping``    clipped fourth-order polynomial mapping Z (Eq. 18), its cell
                 integral (Eq. 19), interpolation Psi (Eq. 20) and spreading
                 Phi (Eq. 21).
* ``bubble``     interface-force closures (Table 1, Eq. 3) and the explicit
                 Newton update of a bubble (Eq. 1, 2, 4; Algorithm 1 step 5).
* ``binning``    bubble-to-cell and bubble-to-tile assignment (Algorithm 1
                 step 2), by brute force.
* ``step``       the coupled time loop in the order of Algorithm 1.
* ``validation`` theoretical relative and terminal velocities (Eq. 22-25).

Every function cites the passage it follows.  Where the paper is garbled or
silent, the reading taken is stated beside the code.
"""

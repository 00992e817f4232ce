"""FP64 CPU oracle for the octree SBFEM central-difference step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

Everything here is a plain, slow, obviously-correct restatement of the paper
(Zhang et al., "A massively parallel explicit solver for elasto-dynamic
problems exploiting octree meshes", arXiv 2103.09100):

* ``cube``      -- reference octree cell: corner / mid-edge / face-centre node
                   slots, the 48 signed-permutation transforms built from the
                   rotations and mirrors of Eqs. (Rotate)/(Reflect), and the
                   reduction of the 4096 mid-edge masks to 144 unique patterns
                   (Sec. 3.2.2).
* ``sbfem``     -- the scaled boundary finite element of one cubic cell:
                   surface discretisation (Sec. 3.2.1), coefficient matrices
                   E0/E1/E2 (Eq. E0E1E2), eigen-solution and stiffness
                   K = Phi_q1 Phi_u1^-1 (Eqs. SBFE, q_E0E1, u_q_phixic, K),
                   consistent mass M = Phi_u1^-T m Phi_u1^-1 (Sec. 2.2),
                   the direction-wise mass lumping (Sec. 3.3) and the
                   element critical time step (Eq. tcr).
* ``assembly``  -- element matrices of real cells by scaling (Eq. KM_scale)
                   and transforming the master-cell matrices (Sec. 3.2.2),
                   the brute-force global sparse K, the global diagonal mass
                   and the critical time step (Eqs. tcr, tcr_scale).
* ``cdm``       -- the element-by-element explicit solver of Algorithm 1 with
                   Eqs. (D0), (DnMdiag) and the Ricker load (Eq. Ricker),
                   as plain C (``cdm.c``) driven through ctypes, plus a
                   pure-Python sparse-matrix stepper used to pin it.
* ``adjoint``   -- the exact discrete adjoint of the same recurrence and the
                   per-cell modulus gradient.

Functions whose result no test can tie to something other than the oracle
itself say "parity unpinned" in their docstring.
"""

"""Oracle for the batched nonlinear constraint projection -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
arm may import this package.  The CUDA library (``paper_2607_00095_b300``) never imports,
links or calls anything here, and shares no code with it; the only common module is the
seeded input generator ``paper_2607_00095_b300.synthetic``, which holds none of the
method's arithmetic.

Contents
  kkt_dense.c     dense Newton-KKT (Appendix B) with Bunch-Kaufman LDL^T, generic over
                  rows h_r(u) = A_r u + sum_j Q_rj u_j^2 - b_r; dense adjoint (IFT).
  problems.py     the constraint rows of each problem family, written from the paper's
                  definitions (Table I, Appendix A, Appendix C, Appendix D) and the
                  workload definitions; dh/dtheta for the adjoint.
  solve.py        ctypes wrapper: project(), adjoint(), components().
  flux.py         family E (Burgers IC + mass + Godunov flux rows, Appendix A and D): the
                  KKT point by its definition (forward Godunov steps, stationarity solve),
                  the Newton-KKT iteration on the full system for small cases, the adjoint.
  pcfm.py         the sampling loop of Eqs. 1-3 around the oracle projection.
  closed_form.py  exact projections with a plain definition (2-D Leray projection onto
                  divergence-free fields intersected with the energy sphere, via FFT).

Every function cites the passage it follows.  Pins that tie the oracle to something other
than itself live in tests/test_oracle_*.py.
"""

"""CPU oracle for the scenario absorber design NLP (problem (10) of the paper).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm may import or execute anything in this package; the library's
product path (paper_2607_15420_gb300 and its CUDA code) never does, and shares no code
with it.  The only module both sides use is absorber_inputs (seeded data, no method
arithmetic).

Plain, slow, FP64, numpy/scipy:
  ad.py      second-order forward-mode AD (Taylor arithmetic) -- derivatives by definition
  model.py   the MESH equations (1), (3a), (4), (6), (9a-b) and the hydraulic row (10b)
             of the case study, per stage and scenario, written out once
  kkt.py     per-scenario dense Bunch-Kaufman LDL^T (LAPACK via scipy), inertia by
             Sylvester's law, scalar Schur complement on the shared diameter; a
             monolithic dense LDL^T for tiny cases
  ipm.py     filter line-search primal-dual interior point (Wachter & Biegler 2006)
  checks.py  independent checks: complex-step Jacobians, conservation of elements,
             charge and enthalpy, the square MESH system by Newton, the closed-form
             optimal diameter, E_0 from the definitions
  mlp.py     the warm-start network (3 -> 256 -> 256 -> 256 -> 440, GELU, bfloat16
             weights): forward pass, loss, reverse-mode gradient, Adam step

Pins (tests/test_oracle_*.py, -m "not gpu"): the paper's printed problem size at
|Omega| = 5000; AD against closed forms and against complex step; the Hessian against
finite differences of complex-step gradients; Schur solve against the monolithic
LDL^T; inertia against eigenvalue signs; at the returned point E_0 <= 1e-8, d* equal
to max sqrt(4 V R T / (pi u_max P)), one active hydraulic row, C/H/N/O/charge and
enthalpy conserved, the square MESH system's Newton root, identical-scenario symmetry,
a brute-force diameter sweep; for mlp.py, bfloat16 rounding against hand-worked
ties, GELU against Phi(+-1), the gradient against central finite differences, the
zero-weight and single-path networks and the first Adam steps against closed forms.
Parity unpinned: agreement with the paper's own numbers
(its constants and scenario data are not published), and uniqueness of the MESH root.
"""

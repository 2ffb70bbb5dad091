"""Plain, slow FP64 CPU oracle of the DG thermosphere discretisation.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package: only tests/,
__graft_entry__.smoke() and the cpu_baseline / --impl reference legs of bench.py may use it.
It shares no code with the CUDA library; its only common dependency is the seeded input module
paper_2306_01085_gb300.workloads, which holds no arithmetic of the method.

Everything is written from the definitions, element by element, with dense per-element operators
(no sum factorisation, no fusion):
  quadrature.py  Gauss / Gauss-Lobatto-Legendre rules and Lagrange bases (Sec. 3.1, spaces W_h, Q_h)
  mesh.py        box and cubed-sphere meshes, isoparametric geometry, face matching (Sec. 3.1, 3.3)
  physics.py     flux F(u, q) and source s(u, q) of Eq. fluxSWNondimensional, stabilisation of Eq. LDG2
  dg.py          LDG gradient (Eq. DGformulation a), residual (Eq. DGformulation b), complex-step Jv
  solver.py      DIRK / Newton / GMRES and block-Jacobi (Sec. 3.1-3.2)

Parity status of every function is stated in its docstring; pins live in tests/test_oracle_*.py.
"""

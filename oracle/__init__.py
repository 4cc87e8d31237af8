"""Plain FP64 CPU oracle of the HEOM method (arXiv 2306.07522, HierarchicalEOM.jl paper).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import or execute anything in this package. The product library
(``paper_2306_07522_gb300``) never calls it, and this package never imports the product.

What it computes, each piece following the paper's statement (cited per function):

* ``exponents``   bath correlation exponents (Methods: Lorentzian / Drude-Lorentz; Pade and
                  Matsubara decompositions of the Fermi and Bose functions).
* ``hierarchy``   ADO multi-indices (Eq. HEOM multi-index notation, Pauli exclusion) in the
                  canonical order that the GPU path must reproduce bit-exactly.
* ``liouvillian`` the HEOM Liouvillian superoperator M (Eq. HEOM with A, B, C, D, P_s), twice:
                  as an explicit scipy.sparse matrix in Liouville space, and as a per-ADO
                  loop of dense matrix products.
* ``solvers``     RK4 dynamics, dense propagator exp(Mt), stationary state (sparse LU with a
                  trace row), spectra (Methods: Numerical computation of the spectrum), the
                  electronic current (Methods: Electronic current, Eq. last).

Every function is pinned by a ``-m "not gpu"`` test against something other than itself
(closed forms, the paper's Table 3 counts, quadrature of Eqs. C_f / C_b, invariants).
"""

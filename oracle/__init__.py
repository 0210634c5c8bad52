"""Plain, slow, fp64 CPU oracle for the T-matrix multiple-scattering method
(arXiv 2107.09879, App. I, II and IV).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (``paper_2107_09879_b300``) never imports, calls or links
anything here, and nothing here imports the product package: the two share no
code, tables or constants. Only the seeded input generators
(``paper_2107_09879_b300.workloads``), which hold none of the method's
arithmetic, feed both sides.

Every function follows a passage of the paper (cited in its docstring) or the
plain textbook definition that passage relies on. No blocking, fusion or
reordering beyond what the definition states: each step can be checked
against the paper by eye.

Modules
-------
specfun      spherical Bessel/Hankel, normalised Legendre, pi/tau, Wigner-3j
vswf         vector spherical wave functions Phi, RPhi (App. I-A)
mie          sphere T-matrix (closed-form special case of App. I-B) and dT/dr
nullfield    null-field T-matrix of a scatterer bounded by a surface (App. I-B): cylinders
translation  addition-theorem coefficients xi = alpha/beta (App. I-C)
incident     plane-wave and jinc-source expansion coefficients (App. II)
system       Maxwell operator (I - T A), dense assembly, LU, GMRES (App. I-C/D)
field        scattered field and figure of merit (App. I-C, App. IV)
adjoint      adjoint solve and radius gradient (App. IV)
geometry     neighbour lists within a cutoff and sub-region index sets (main text)
"""

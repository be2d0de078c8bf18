"""Plain CPU FP64 oracle for the vertex-patch multigrid method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path (``paper_2405_19004_gb300``) and imports
nothing from it.

Everything here is written from the definitions in Cui, Grosse-Bley,
Kanschat, Strzodka, "An implementation of tensor product patch smoothers on
GPU" (arXiv 2405.19004):

* ``fe``        -- Q_k Lagrange elements on Gauss-Lobatto support points,
                   element matrices by quadrature (Section 2, Eq. 2.4, 2.9).
* ``assembly``  -- global stiffness matrix and load vector by an explicit
                   loop over cells, prolongation by interpolation
                   (Section 2, Eq. 2.2-2.4; Section 2.1).
* ``smoothers`` -- vertex patches, colouring, the sequential and colourised
                   multiplicative smoothers and the additive smoother
                   (Section 2.2, Eq. 2.5-2.7, Algorithm 3).
* ``multigrid`` -- V-cycle (Algorithm 1), full multigrid (Algorithm 2),
                   preconditioned CG, L2 error.
* ``local``     -- the same definitions evaluated for single patches / rows
                   at sizes where the global matrix cannot be assembled.

Precision: FP64 throughout; the paper fixes no precision for the method.
Every function has a pin in ``tests/test_oracle_*.py`` (closed forms,
invariants, textbook special cases, values printed in the paper); none is
"parity unpinned".
"""

from . import fe, assembly, smoothers, multigrid, local  # noqa: F401

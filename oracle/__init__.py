"""Plain, slow FP64 CPU oracle for the HOT method (arXiv 2408.00598).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or runs anything in this package; only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may use it.  It shares no code, tables or
helpers with the GPU path.

Every function follows the paper in its own order and notation:

* ``reduced_model``  -- the reduced L2^2 model eq. (3), its standard form
  eq. (4)-(6), the full-row-rank A and b of eq. (7)-(8), and the AA^T blocks
  of eq. (Mat:OT_AAT), with A built explicitly as a sparse matrix from the
  Kronecker products of eq. (6).
* ``linsolve``       -- the closed-form solution of AA^T y = R, Prop. 3.
* ``hot``            -- Algorithm 2 (HOT), the relative KKT residual of
  eq. (kkt_res), gap and feaserr of Sec. IV-A, and the restart / sigma rule the
  paper leaves open (a stated reading, see ``HotParams``).
* ``recover``        -- Algorithm 1 (transport-plan recovery), literal loops.
* ``exact``          -- exact optimal values: an LP solve of eq. (1) and of
  eq. (3), and a successive-shortest-path min-cost-flow written in plain C
  (``mcf.c``) for the full problem on tiny grids.
* ``closed_forms``   -- textbook closed forms used as pins: 1D quantile
  (north-west-corner) cost, integer translation, product measures.

Parity status: every function above is pinned by a ``-m "not gpu"`` test to
something other than itself (a dense solve, an LP solver, a closed form, brute
force or an invariant the paper proves); none is "parity unpinned".
"""

"""FP64 CPU oracle for the successive-convolution (MOL^T) fast-summation path.

TEST INFRASTRUCTURE ONLY.  Nothing in the library (``paper_2007_03041_gb300``)
may import, call or link anything here; only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  The oracle shares no code with the CUDA path.

It follows Christlieb, Guthrey, Sands, Thavappiragasm, "Parallel Algorithms
for Successive Convolution" (arXiv 2007.03041), step by step and in its
notation, in plain numpy float64 with no blocking, fusion or reordering beyond
what the paper states:

* ``quadrature``  -- local-integral weights c_l(nu), linear weights d_r and
  smoothness indicators (Sec. 2.4, App. C).
* ``sweep``       -- local integrals J_R/J_L, the O(N) recurrences for I_R/I_L,
  boundary constants A/B, L^{-1}, D and the partial sums sum_p D^p
  (Sec. 2.1-2.4).
* ``schemes``     -- the time integrators that consume the partial sums
  (Sec. 2.1, 2.5, Sec. 4.5 / Algorithm 1).
* ``stability``   -- the exact discrete Fourier symbol of the periodic
  operators and the stability bound on beta it implies.
* ``mlp``         -- FP64 forward/backward of the WENO-weight network used by
  the learned weight path (no counterpart in the paper).
* ``dense``       -- the partial sums of one axis as a dense matrix (the image
  of the identity under ``sweep``), applied along the grid's axes by matrix
  products: the linear schemes' steps at full grid sizes.
* ``parallel``    -- ``sweep``'s partial sums on blocks of lines in a process
  pool (lines are independent), and the Hamilton-Jacobi step composed from
  them as ``schemes`` composes it.

Every function cites the passage it follows.  Readings of garbled or silent
passages are stated in the docstring of the function that takes them.
"""

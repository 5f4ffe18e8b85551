"""CPU FP64 oracle for the finite-periodic fast multipole BEM.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import anything from here; the
GPU library never does, and nothing here imports the GPU library.  The two
share no code: the only common inputs come from the ``workloads`` package,
which holds meshes, lattices and random vectors but none of the method's
arithmetic.

Contents (each function cites the part of the paper it follows):

* ``special``  -- spherical Bessel/Hankel functions (scipy as the library
  primitive), associated Legendre functions and the spherical harmonics of
  the multipole expansion, gradients of the regular wave functions, Wigner
  3j symbols by Racah's formula in exact integer arithmetic.
* ``bem``      -- the Burton-Miller collocation operator of Sec. 2.1 for a
  rigid boundary with constant flat-triangle elements: quadrature rules,
  kernels, singular self term, dense matrix, the offset-indexed blocks of the
  multilevel block Toeplitz form of Sec. 2.2, explicit block-Toeplitz
  products, incident plane waves and field points.
* ``fmm``      -- the single-level FMM operators of Sec. 3 and Appendix A:
  P2M and L2P tables shared by all cells, M2L blocks from the Wigner formula,
  the explicit (unconvolved) operator S + U K V of Sec. 3.2, and an
  independent M2L built by projecting the outgoing wave on a sphere.
* ``solve``    -- the dense solve of reference solutions (a library primitive).

Pins of every part live in ``tests/test_oracle_*.py`` (marked not-gpu).
"""

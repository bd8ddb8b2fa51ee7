"""FP64 CPU oracle for the Schwarz neural-operator FDFD solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package; only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is a plain, slow restatement of what the method computes, written from
the paper (arXiv 2509.03622) and sharing no code with the CUDA library:

* ``fdfd``      -- Eq. 1 discretised with the UPML stretching of Methods
                   (Eq. 3-6), sparse assembly, SuperLU direct solve, adjoint
                   solve, adjoint-variable gradient and mode-overlap FoM.
* ``krylov``    -- Algorithm 1 (flexible GMRES) with restarts and Givens.
* ``partition`` -- the "partitioner" of Methods: 80 x 80 windows around
                   64 x 64 cores, restriction, restricted prolongation, the
                   Robin traces of Eq. 2 and the local Robin operator.
* ``nno``       -- the Fourier neural operator forward (Fig. 2).
* ``coarse``    -- pseudo-plane-wave trials, Gram-Schmidt, Robin-to-Robin
                   basis, the coarse normal equations (Eq. 8) and the
                   correction of Algorithm 3.
* ``schwarz``   -- one two-level Schwarz sweep used as the FGMRES
                   preconditioner, and an exact-local-solve variant.

Parity status per function is stated in each module header.
"""

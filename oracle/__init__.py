"""CPU oracle for the HSC-extension selected inversion -- TEST INFRASTRUCTURE ONLY.

Plain, slow, complex128 restatements of what the method computes, written from the paper's
definitions and independent of the CUDA path (no shared code, no shared constants):

* ``dense``    -- Eq. 1 and Eq. 2 written out: A = (E + i eta) I - H - Sigma^r, G^r = A^{-1},
                  G^< = G^r Sigma^< (G^r)^dagger, by dense LAPACK inversion (tiny grids);
* ``rgf``      -- the recursive Green's function sweep of Section 2.1 (Eqs. 3-6) along the
                  transport direction, for block-tridiagonal A (mid sizes, the paper's comparison
                  method);
* ``columns``  -- single columns of G^r by sparse direct solves of A x = e_a, which give G^r_aa and
                  G^<_aa one sampled unknown at a time at any size;
* ``observables`` -- DOS, transmission (Caroli form) and densities from the oracle's outputs;
* ``lead``     -- open-boundary (DENSE) contact self-energies of Section 3.1.2: the surface Green's
                  function of a semi-infinite lead by decimation, Sigma^r = tau g_s tau^T, Gamma;
* ``scba``     -- the self-consistent loop with local elastic dephasing (the scattering part of
                  Sigma^r in Eq. 1) around the dense definition, its single-site closed forms and
                  the terminal currents that its fixed point balances.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this
package. The product path never does.
"""

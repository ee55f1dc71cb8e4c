"""CPU oracle for the periodic FM-BEM transmission problem (test infrastructure).

Plain, slow FP64 code that states what the fast GPU path computes:

* ``greens``   -- free-space Helmholtz kernels and the quasi-periodic Green's
                  function G_qp = sum_m alpha^m Phi(x, y + m h) (Sec. 2, eq. 7),
                  evaluated by an Ewald split, with its spectral (Rayleigh) form
                  and a direct lossy-medium sum as independent checks;
* ``lattice``  -- lattice sums S_j = sum_{|m|>=2} alpha^m H_j(k|m|H) e^{i j theta}
                  that feed the periodic root translation (Sec. 3.3);
* ``bem``      -- flat constant-element collocation of the Kress transmission
                  system (I - A) Psi = B (Sec. 2, eqs. 4-9), dense assembly,
                  dense LU solve, Rayleigh (Bragg) coefficients, ETC and field;
* ``mie``      -- Mie series of one isolated circular fiber (physics check);
* ``nystrom``  -- high-order Nystrom discretisation of the same equations on
                  circles (Kress product quadrature, Maue's identity for T),
                  used only to pin the physics at tight tolerances;
* ``tree``     -- the quadtree's M2L interaction rule and the convergence
                  factors gamma, lambda, tau of Table 1;
* ``mlp``      -- FP64 forward/backward of the warm-start network.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
may import this package.  It shares no code with the CUDA library and never
calls it.
"""

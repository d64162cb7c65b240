"""FP64 CPU oracle for the AIMx operator (Sharma & Triverio, arXiv 2009.02281).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64/complex128
restatement of what the GPU library computes, written from the paper's
equations so that a reader can check it against the paper by eye.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` may import it.  The GPU library never imports, links or
runs anything from here, and nothing here imports the library.

Modules and the passages they follow:

* ``constants``   -- free-space constants.
* ``rwg``         -- RWG basis functions on triangle pairs (Sec. II-A, Eq. EFIEdis).
* ``quadrature``  -- collapsed Gauss-Legendre product rule on triangles.
* ``grid``        -- AIM grid, stencil anchors, moment-matching projection
                     weights P and W = P^T (Sec. II-B, Eq. aimLFR; Sec. IV intro),
                     near-region pair list.
* ``potentials``  -- closed-form static triangle potentials for 1/r, (r'-rho)/r
                     and grad(1/r) (kernel of Eq. hgfs and Eq. ghgfs).
* ``greens``      -- G, G_s, G_d, grad G (Eqs. hgf, hgfs, hgfd, ghgf, ghgfs),
                     grid kernel samples with the self-term rule (Eqs. Hsmm,
                     Hdmm, Hmm, gH00), interpolation error bound (Eqs. Lbounds,
                     Dhgf, Dghgf).
* ``static``      -- frequency-independent near matrices L_s,NR, K_s,NR and the
                     precorrections L_s,P, K_s,P (Eqs. Lmatdecomp2, aimLPs, KAIMx).
* ``operator``    -- the AIMx matvec by direct (non-FFT) grid summation and the
                     dense AIMx matrix (Eqs. LAIMx, EFIEAIMx, KAIMx); EFIE and a
                     two-region (PMCHWT) form.
* ``excitation``  -- plane-wave right-hand sides.
* ``farfield``    -- far field and radar cross section of surface currents.
* ``mie``         -- Mie series for PEC and dielectric spheres (textbook).
* ``mom``         -- dense MoM by direct integration (error reference).
* ``solve``       -- dense LU and plain GMRES.
* ``chargepot``   -- the EFIE scalar potential in charge form, L^Phi = D^T Pt D
                     with the pulse matrix Pt in AIMx form (the discretisation of
                     the augmented EFIE the paper cites for small conductors);
                     oracle of a row with no GPU path yet.

Where the paper is silent each module states the reading it takes.
"""

"""Plain FP64 CPU oracle of the matrix-free macro-element HDG method (arXiv 2402.11361).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or runs
this code; only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with the
CUDA path: every formula here is written out again from the paper, slowly and
plainly, so that a reader can check it against the equations by eye.

Modules
-------
physics   -- nondimensional fluxes, numerical trace flux, boundary operator,
             SUPG coefficient (Sec. 2.1, 2.3; eqs. C4-C6, num. flux, S^inv/S^vis)
space     -- GLL-Lagrange C0 spaces on macro-elements, Gauss quadrature, the
             macro-face trace space and the global trace numbering (Sec. 2.2);
             isoparametric curved macros and the cubed-sphere shell
simplex   -- simplicial macro-elements: P_p on m-refined simplices, their faces
             and trace spaces, and a box mesh of them (Sec. 2.2)
assemble  -- residuals R_Q, R_U, R_Uhat (eq. C31221) and the Newton blocks of
             eq. C312 for one macro-element
solve     -- one-layer (eq. C47) and second-layer (eqs. AP12, ASC2, Csc4)
             static condensation, dense LU, explicit global trace matrix,
             Algorithm 2, GMRES/FGMRES (Sec. 4.2), pseudo-transient Newton with
             SER (eq. C31222), the DIRK stage equations (eq. C242) and the
             Taylor-Green flow integrals (eq. C5321)
fields    -- closed-form fields: manufactured solution, Couette (2D, and 3D with a
             source), Taylor-Green, the sphere's initial state
mlp       -- FP64 forward/backward of the preconditioner-correction MLP

Parity status of each function is listed in its docstring ("pinned by ...").
"""

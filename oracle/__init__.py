"""CPU FP64 oracle for the AMR axion-string step -- TEST INFRASTRUCTURE ONLY.

A plain, slow, readable restatement of what the scheme computes, used to check
the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
library never does, and this package imports nothing from the library.  It
shares no code, tables or constants with the CUDA path: inputs arrive as
arrays from the seeded generators.

Modules and the paper passages they restate:

* ``stencil``  -- finite-difference Laplacian / gradient (App. A).
* ``eom``      -- right-hand side of the first-order system (Sec. 3.1,
                  Eqs. EOM1-EOM2; the ``Rhs`` listing fixes the potential form).
* ``rk4``      -- classic RK4 (integrator type 4, Tab. "integrator") on a
                  uniform periodic lattice.
* ``winding``  -- string-winding plaquette count and cell tags (the problem
                  specific tagging hook of Sec. 4.2; the winding rule itself is
                  not in the paper, see the reading in the module).
* ``interp``   -- ratio-2 prolongation (interpolation types 2 and 4,
                  Tab. "amr") and 2^3 restriction (Sec. 2.1).
* ``energy``   -- energy components and pierced-plaquette string length.
* ``regrid``   -- tags -> buffer -> block coarsening -> Berger-Rigoutsos style
                  clustering -> nesting (Sec. 2.2-2.3).
* ``amr``      -- level hierarchy with ghost fill, time interpolation,
                  recursive subcycling and synchronisation (Sec. 2.1, Fig. 2).

Everything is float64 numpy evaluated element by element in the order the
docstrings state (numpy does not contract a*b+c into an FMA).  Parity status of
each function is stated in its module header.
"""

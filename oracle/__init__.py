"""FP64 CPU oracle for the thermal lattice Boltzmann hot path (test infrastructure).

This package is a plain, slow, obviously-correct restatement of what the paper
(J. W. Shim, "Multidimensional On-lattice Higher-order Models in the Thermal
Lattice Boltzmann Theory", arXiv:1303.4624) defines, written in numpy FP64:

* ``model``        the D2Q33 / D3Q95 velocity sets of Tables 2 and 3, the moment
                   equations of Formulas 3-5 solved for the weights, and the
                   equation counts of Formulas 6-10 / Table 1;
* ``equilibrium``  the fourth-order Hermite equilibrium (Formula 1 with m = N = 4),
                   written as the tensor Hermite series;
* ``lbm``          the BGK stream-and-collide update, macroscopic fields,
                   conservation audit and the discrete adjoint of the update;
* ``riemann``      the exact Riemann solution of the ideal gas the models
                   describe (used as a physics pin).

It is test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product path (the CUDA
library and its Python binding) never does, and shares no code with it.

Parity status per function is stated in each module header.  Every function
here is pinned by a ``-m "not gpu"`` test against something other than itself
(the paper's printed tables, closed-form Gaussian moments, Gauss-Hermite
quadrature, brute force on tiny inputs, finite differences, exact Riemann
plateaus), except where a module header says "parity unpinned".
"""

"""GB300-native lattice-Boltzmann step with velocity-interpolation
bounce-back (arXiv:1903.01111).

Submodules:

* ``geometry`` -- masks, cut-link lists with q, sphere packs (host, no CUDA);
* ``lbm``      -- ctypes binding of the C-ABI library ``liblbm.so`` whose
                  entry points are declared in ``include/lbm.h``;
* ``build``    -- compiles ``liblbm.so`` (nvcc, sm_103a) and ``libgeom.so``.

Importing the package loads nothing; ``lbm`` raises if ``liblbm.so`` has not
been built, and there is no CPU fallback.
"""

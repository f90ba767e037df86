"""FP64 CPU oracle for the dual messenger Wiener filter on the HEALPix sphere.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the product package never does, and this package never imports the product.

Modules
-------
sht      HEALPix ring geometry, normalised Legendre functions and the direct
         O(Npix*Nalm) synthesis Y and plain transpose Y^T (C, via ctypes),
         plus explicit real-basis matrices for small Nside.
dm       The paper's Algorithm 2 (hybrid dual messenger) on the sphere, the
         dense fixed-point and exact Wiener-filter solves (Eq. 2 and the
         symmetric form of App. C), PCG with the harmonic-diagonal
         preconditioner (App. C), residual and chi^2 diagnostics.
"""

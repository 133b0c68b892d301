"""The oracle: plain, slow, obviously correct CPU implementations of what the
sFMM computes.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import anything from here.  The CUDA solver never does, and
this package imports nothing from the solver: the two share no code.

Modules
-------
direct   FP64 direct sum of G and its covariant gradient (Sec. 3.1, Eq. SUM;
         Sec. 2.1, Eqs. GRE_FUN, ALP_PSI), C + OpenMP via ctypes.
healpix  HEALPix nested keys and pixel geometry (Sec. 3.1; Gorski et al. 2005).
tree     CPU rebuild of the adaptive 12-root quad-tree (Sec. 3.1, steps 1-3).
lemmas   Lemmas 1-4 and the L2P formulas of Sec. 3.6, written as printed.
walk     Algorithm 1 (Sec. 3.4) with the MAC of Sec. 3.5, plain recursion.
"""

"""GB300-native two-level additive Schwarz + block ILU(0) Krylov solver: the boundary-conditioned
additive Schwarz preconditioner of Section 4 (near- and far-field lumps, Eq. 4.1) with column-sum
block ILU(0) local solves (Section 2), for GMRES / ORTHOMIN on black-oil Jacobians.

The solver lives in a C-ABI shared library (``libasm2.so``, hand-written CUDA for sm_103a);
:mod:`paper_1401_7227_gb300.asm2` is its thin ctypes binding and :mod:`.synth` makes seeded
inputs.  Submodules are imported lazily so that the input generator can be used without loading
the CUDA library.
"""

__all__ = ["asm2", "synth"]

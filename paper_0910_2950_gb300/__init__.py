"""GB300-native force-gradient Hybrid Monte Carlo for 4D SU(3) lattice gauge theory.

The compute path is the CUDA library ``libfg_lattice.so`` (hand-written
kernels for sm_103a behind the C ABI declared in ``include/fg_lattice.h``);
``paper_0910_2950_gb300.fg`` is the thin ctypes binding to it and
``paper_0910_2950_gb300.inputs`` draws seeded synthetic inputs.  Importing
this package loads nothing; the binding loads the library on first use and
raises if it is missing.
"""

__all__ = ["inputs", "fg"]

"""GB300 (sm_103a) lattice SU(2) heat bath: checkerboard sweeps, plaquette and
Polyakov loop (Cardoso & Bicudo, "Lattice SU(2) on GPU's", LAT2010).

Modules:
  su2       -- ctypes binding of the C ABI in include/su2.h (needs libsu2.so)
  analysis  -- host-side statistics (integrated autocorrelation time)
  workloads -- the seeded synthetic workloads (lattice shapes, beta, seeds)
  _build    -- nvcc build of libsu2.so
"""
__all__ = ["su2", "analysis", "workloads"]

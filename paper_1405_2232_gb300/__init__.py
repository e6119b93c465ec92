"""GB300-native fused thermal pseudopotential D2Q9 lattice Boltzmann step.

Implements the double-distribution thermal pseudopotential LB method of
Li & Luo (arXiv:1405.2232): the density LBE Eq. (1) with the pseudopotential
force Eqs. (2)/(4), and the temperature LBE either as Eq. (7) (forcing-term
effect present) or as the corrected Eq. (24)-(25).

Submodules:
  lb      -- ctypes binding of the C-ABI library (liblbgb.so, CUDA sm_103a)
  inputs  -- seeded synthetic input generators (no method arithmetic)
  build   -- compiles the CUDA library in-tree
"""
__all__ = ["lb", "inputs", "build"]

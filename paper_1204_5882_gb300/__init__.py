"""GB300-native successive-cancellation decoding of long polar codes for QKD
error correction (syndrome form), after Jouguet & Kunz-Jacques, arXiv 1204.5882.

Submodules:
  ``polar``  -- ctypes binding of the C ABI (include/polar.h);
  ``synth``  -- seeded synthetic inputs (random draws only);
  ``build``  -- in-tree build of the sm_103a library.
"""

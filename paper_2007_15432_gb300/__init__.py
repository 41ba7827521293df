"""GB300-native soft step of the P3T planetary N-body integrator with
individual cut-off radii (Ishigaki et al. 2021, PASJ 73, 660).

Sub-modules:
  * ``p3t``   -- thin ctypes binding of the C-ABI library ``libp3t.so``
                 (sm_103a CUDA kernels); importing it loads the library and
                 fails loudly if it is missing;
  * ``disks`` -- seeded synthetic protoplanetary disks (input generators only);
  * ``build`` -- nvcc build of ``libp3t.so``.

Importing the package itself loads nothing.
"""
__all__ = ["p3t", "disks", "build"]

"""GB300-native hot path of the implicit octree GIMP Material Point Method.

The compute runs in the CUDA library `libmpm_gb300.so` (built from csrc/);
`paper_2606_09275_gb300.mpm` is the thin ctypes binding over its C ABI.
"""

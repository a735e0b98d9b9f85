"""B300-native matrix-free NGF + curvature deformable registration.

The compute path is the C-ABI library `libngf_b300.so` (hand-written CUDA for
sm_103a, built in-tree from `csrc/`); `paper_1804_10541_b300.ngf` is its thin
ctypes binding and raises if the library is missing.  `synth` holds the seeded
synthetic input generators (no arithmetic of the method).  Importing this
package loads nothing.
"""
__all__ = ["ngf", "synth"]

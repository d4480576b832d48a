"""GB300-native parametric voxel generation of 3D straight-line segments.

Layers (top to bottom): ``vox`` (Python binding of the C ABI in include/vox.h),
``libvox.so`` (csrc/: count + decoupled look-back scan + voxel-parallel
generation kernels for sm_103a), plus ``workloads`` (seeded synthetic inputs),
``batching`` (batched scenes in one persistent launch captured in a CUDA graph)
and ``serving`` (continuous-batching request loop).
"""

__all__ = ["vox", "workloads", "build"]

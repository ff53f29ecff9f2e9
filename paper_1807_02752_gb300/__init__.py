"""GB300-native stereo lane detection (Fan & Dahnoun, "Real-Time Stereo Vision-Based Lane Detection
System", arXiv 1807.02752): the per-frame dense path from a disparity map and a left image to lanes.

The compute path is the CUDA library built from ``csrc/`` (C-ABI declared in ``include/ld.h``);
``ld`` is its Python binding.  ``scenes`` renders seeded synthetic inputs.
"""
__all__ = ["scenes", "ld"]

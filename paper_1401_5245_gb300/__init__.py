"""GB300-native edge detection of binary images by the method of masks.

The compute path lives in the CUDA library ``libme.so`` (sources under
``csrc/``, C ABI in ``include/me.h``); :mod:`._lib` is its ctypes binding.
"""
__all__ = ["synth"]

"""GB300-native positional population count (arXiv 2412.16370).

The counting runs in hand-written sm_103a CUDA kernels behind the C ABI
declared in ``include/pospopcnt.h`` (``libpospopcnt.so``).  ``binding`` is
the thin ctypes layer over that ABI (argument marshalling only); ``synth``
makes seeded synthetic inputs.  Importing the package loads nothing: the
shared library is opened on first use and every call raises if it is
missing -- there is no CPU fallback.
"""

__all__ = ["binding", "synth", "build"]

"""GB300-native hot path of the Jasche & Wandelt (arXiv:1306.1821) sampler.

The compute lives in the CUDA library `libbps.so` (C ABI, declared in
include/bps.h); `bps` is its thin ctypes binding and `inputs` the seeded
synthetic survey generator.  Importing the package loads nothing; the library is
loaded on first use and a missing library is an error, never a fallback.
"""

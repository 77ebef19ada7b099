"""GB300 (sm_103a) library for the quantized-tensor-train Moulinec-Suquet hot
path of arXiv 2512.07811.

Submodules (imported explicitly, nothing is loaded eagerly):
  qtt     ctypes binding of the C-ABI in include/qtt.h (needs libqtt.so)
  build   nvcc build of libqtt.so
  inputs  seeded synthetic inputs (geometries, random trains)
"""

"""VeST (Very Sparse Tucker factorization) on one GB300 GPU.

Modules:
  vest        ctypes binding of the C ABI in include/vest.h (libvest.so, CUDA for sm_103a)
  build       in-tree build of libvest.so with nvcc
  datagen     seeded synthetic inputs (observed positions, planted models, initial states)
  batch       many independent factorisations as CUDA graphs over a pool of streams
  serve       a continuous-batching request loop (factorisation jobs, completion queries)
  checkpoint  save and load a long auto-search run (model and report)
"""

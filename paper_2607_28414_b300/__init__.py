"""B300 (sm_103a) hot path of the reduced Kelvin-Voigt shear-wave method:
libkv (CUDA, C ABI in include/kv.h), its Python binding `kv`, the seeded
synthetic inputs `inputs` and a workload `runner`."""

"""GPU FCIQMC engine for one NVIDIA GB300 (sm_103a).

`hande` binds the C ABI of libhande.so (include/hande.h); `inputs` holds the
seeded synthetic workloads.  Importing the package does not load the CUDA
library; the first `hande.Hande(...)` does, and raises if it cannot.
"""

"""GB300-native GPLHR eigensolver (arXiv 1506.06829): CUDA hot path behind a C ABI.

Submodules
----------
gplhr     -- ctypes binding to ``libgplhr.so`` (gplhr_create / solve / vectors / ...).
problems  -- seeded synthetic pencils and start blocks (inputs only).
build     -- compiles ``libgplhr.so`` for sm_103a with nvcc.

Nothing is imported eagerly, so ``problems`` can be used without the CUDA library.
"""

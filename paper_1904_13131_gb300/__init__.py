"""GB300-native matrix-free finite-strain hyperelasticity with geometric multigrid (arXiv 1904.13131).

  build    compile libhyperelastic.so (sm_103a) in-tree
  api      ctypes binding of the C ABI in include/hyperelastic.h (Context)
  inputs   seeded synthetic problem data (meshes, inclusions, fields)

Importing the package loads nothing; api.Context loads the library and fails loudly if it is
missing.
"""
__all__ = ["api", "build", "inputs"]

"""GB300 (sm_103a) implementation of one IMEX time step of the spherical
quasi-geostrophic convection model of Gastine (pizza, GJI 2019).

Submodules:
  binding  - ctypes binding of libpizza (the C interface in include/pizza.h)
  inputs   - seeded synthetic initial states (shared by tests and benchmark)
  build    - nvcc build of libpizza.so
Importing the package loads nothing; ``binding.load()`` opens the library.
"""

"""GB300-native ASE-DFF compact gas-kinetic scheme (S2O4 step on Cartesian meshes).

``paper_2508_13705_gb300.cgks`` is the ctypes binding of the CUDA C-ABI library
``libcgks.so``; ``paper_2508_13705_gb300.inputs`` generates seeded synthetic
initial states.  Importing the package does not load the CUDA library.
"""

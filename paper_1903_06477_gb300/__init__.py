"""GB300-native SuperSCS hot path (arXiv 1903.06477).

The solver itself is the C-ABI library ``libsuperscs.so`` built from
``csrc/`` (hand-written CUDA for sm_103a).  ``binding`` marshals arguments to
it; ``workloads`` builds seeded synthetic problems.  Importing this package
loads nothing: the binding loads the library on first use and raises if it is
missing.
"""

"""GB300-native (sm_103a) solver for the second-order convex-splitting scheme of
the periodic 3D phase field crystal equation, with a nonlinear FAS multigrid
time step (arXiv:1611.06288).

The compute path is the CUDA library ``libpfc.so`` behind the C ABI declared in
``include/pfc.h``; :mod:`.binding` marshals arguments to it and
:class:`.solver.PFCSolver` is the user-facing wrapper.  Importing the package
does not load the library; the first call that needs it does, and fails
loudly if it is missing.
"""

"""B300-native executor for vector bytecode (the data-parallel hot path of
cphVB, Kristensen et al., SciPy 2012).

The executor is the C-ABI library ``libvbe.so`` (header ``include/vbe.h``);
``paper_1210_7774_b300.vbe`` is its ctypes binding and
``paper_1210_7774_b300.runner`` marshals bytecode programs onto it. Importing
this package does not load the library; importing ``vbe`` does, and fails
loudly when it is not built.
"""
__all__ = ["vbe", "runner", "build"]

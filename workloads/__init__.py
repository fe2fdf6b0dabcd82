"""Seeded synthetic workloads: bytecode programs and their input arrays.

Shared by the oracle and by the CUDA executor's tests and benchmark. This
package holds no arithmetic of the executed method; it only builds
instruction lists and draws inputs from seeded generators.
"""
from .program import (DTYPES, ITEMSIZE, NP_DTYPE, Base, Const, Instr, Program, ProgramBuilder,
                      View, c_strides)
from .jacobi import jacobi, jacobi_inputs
from .blackscholes import blackscholes, bs_inputs
from .shallow_water import shallow_water, sw_inputs
from .montecarlo import montecarlo_pi, mc_sizes
from .stencil import gray_scott, stencil_inputs
from .knn import knn, knn_inputs

__all__ = ["DTYPES", "ITEMSIZE", "NP_DTYPE", "Base", "Const", "Instr", "Program", "ProgramBuilder",
           "View", "c_strides", "jacobi", "jacobi_inputs", "blackscholes", "bs_inputs",
           "shallow_water", "sw_inputs", "montecarlo_pi", "mc_sizes", "gray_scott", "stencil_inputs",
           "knn", "knn_inputs"]

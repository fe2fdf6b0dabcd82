"""Oracle: a plain, slow, CPU reference for the vector-bytecode executor.

TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
benchmark's CPU-baseline leg may import, call or run anything in this
package. The executor never routes work through it; it shares no code with
the CUDA path (it depends only on the seeded workload generators, which hold
none of the method's arithmetic).

``oracle.run(program)`` executes the program's bytecodes one at a time, in
order, with NumPy-ufunc semantics (see ``oracle.interp``).
``oracle.OwnershipModel`` adds a host copy to bases and follows the
sync / release / discard ownership rules (see ``oracle.ownership``). RANDOM follows the
counter form of splitmix64 (``oracle.splitmix``). Every function is pinned
by tests against values fixed by mathematics or by brute force, not by
itself: IEEE correct rounding via exact rationals, transcendentals via
mpmath, views via explicit index loops, the workloads via closed forms,
invariants and pure-Python loops on tiny inputs.
"""
from .interp import Memory, OracleError, execute, run
from .ownership import OwnershipModel
from .splitmix import GAMMA, mix64, random_u01

__all__ = ["Memory", "OracleError", "execute", "run", "OwnershipModel", "GAMMA", "mix64", "random_u01"]

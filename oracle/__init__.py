"""CPU oracle of the DD-CCLB time step: test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything under this package.  The CUDA path never
calls it, and the two share no code: the only common module is the seeded
input generator ``workloads``, which holds none of the method's arithmetic.

Parity status of each function is stated in its docstring; every function
used by the step is pinned by a test of ``tests/test_oracle_*.py`` against a
fact the paper or the mathematics fixes (moment identities of Eq. B.5,
conservation, reduction consistency, stencil exactness, the flat-interface
profile, the Laplace law, the shear-wave viscosity of Eq. 16 and the
wetting direction of Eq. 2.14), except the Hermite rows above second order,
the lag choices and the outer-wall details, which are "parity unpinned".
"""
from .ddcc_oracle import Oracle  # noqa: F401

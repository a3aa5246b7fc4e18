"""CPU oracle of the DD-CCLB time step: test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything under this package.  The CUDA path never
calls it, and the two share no code: the only common module is the seeded
input generator ``workloads``, which holds none of the method's arithmetic.

Parity status of each function is stated in its docstring; every function
used by the step is pinned by a test of ``tests/test_oracle_*.py`` against a
fact the paper or the mathematics fixes (moment identities of Eq. B.5,
conservation, reduction consistency, stencil exactness, the flat-interface
profile, the Laplace law, the shear-wave viscosity of Eq. 16, the wetting
direction of Eq. 2.14, the Eq. 19 coefficients derived from the collision
matrix as in App. C, the joint velocity / pressure / force solve, Galilean
invariance of a translating density interface and App. B's sum of g^ne).
``ddcc_naive`` is a second transcription of the step written separately
(node by node, full collision matrices, Newton's method for the pressure,
push streaming); the two agree to 1e-13 on random 8 x 8 inputs over 50
steps, which is what pins the Hermite rows above second order, the lagged
fields and the outer-wall details: no closed form reaches those, and the
paper leaves their readings open.
The three-dimensional step (D3Q7 phase, D3Q15 flow; ``ddcc_oracle3d``) is
pinned the same way by ``tests/test_oracle3d.py``, plus the 3D pressure
constants of Eq. 19 derived from its collision matrix and the symmetry of
the step under axis permutations and reflections.
"""
from .ddcc_oracle import Oracle  # noqa: F401
from .ddcc_oracle3d import Oracle3D  # noqa: F401

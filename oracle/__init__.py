"""FP64 CPU oracle for the AMOEBA induced-dipole solve (test infrastructure only).

A plain, slow NumPy/SciPy restatement of what the GPU path computes: the permanent
multipole field (real space + reciprocal + self), the Thole-damped Ewald dipole-field
operator, the diagonally preconditioned conjugate gradient, and the polarization energy
and forces. It follows the definitions behind the paper's citations (smooth PME with
order-5 B-splines, Sec. 1.2.2 "Reciprocal space scheme"; PCG with a diagonal
preconditioner, Sec. 1.3 and Sec. 3 "Performance and Scalability Results").

Only the test suite, the smoke check of the entry module and the CPU-baseline leg of the
benchmark may import it. The CUDA library never calls it, and it shares no code with
the library: both take the same arrays from the seeded input generators.

Modules: radial (screened and damped radial functions), frames (local frames and their
derivatives), pairs (pair enumeration and scale tables), realspace (pair sums, single and
two-dipole-set forces), ewald (exact reciprocal k-sum), spme (smooth PME), model (field,
operator, PCG, Jacobi/DIIS, energy, forces, virial, and AMOEBA's two dipole sets: d/p
fields, lockstep PCG, energy, forces and virial), mlp (the learned-guess network in FP64),
md (the minimal rigid-water integrator: velocity Verlet with SHAKE/RATTLE and a
force-shifted oxygen Lennard-Jones term).
"""
from . import radial, frames, pairs, realspace, ewald, spme, model, mlp, md  # noqa: F401
from .model import Params, Oracle  # noqa: F401

"""Seeded synthetic inputs shared by the tests, the smoke check and bench.py.

This module holds no arithmetic of the DG method: only the workload recipes
(mesh sizes, mapping, degree, geometry storage, coefficient) and seeded
random vectors.  Both the CUDA path and the oracle receive the same arrays.

Workloads (Kronbichler & Kormann, arXiv:1711.03590, stand-ins for the
paper's meshes: Cartesian boxes and a curved mesh; the hypershell of
Sec. 5 is replaced by the sine-deformed cube):
  cartesian_periodic_4x4x4_p2  64 cells, degree 2, periodic, kappa = 1 (1728 dofs)
  deformed_dirichlet_32^3_p<p> 32768 cells, x_i + 0.1 sin(pi x) sin(pi y) sin(pi z),
                               full per-point Jacobians, kappa = 1 + 0.5 sin(2 pi x),
                               Dirichlet, degree p = 1..8 (p = 4: 4,096,000 dofs)
Source vectors are uniform on [-1, 1] from numpy's PCG64 generator.
"""
import numpy as np

VELOCITY = (1.0, 0.5, 0.25)


def src_vector(n, seed=1):
    """Uniform[-1, 1] float64 vector of length n from a fixed seed."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, int(n))


def sample_cells(n_cells, count, seed=11, must=()):
    """Sorted unique cell indices: the listed ones plus a seeded sample."""
    rng = np.random.default_rng(seed)
    pick = set(int(c) for c in must if 0 <= c < n_cells)
    pick.update(int(c) for c in rng.choice(n_cells, size=min(count, n_cells), replace=False))
    return np.array(sorted(pick), dtype=np.int64)


def workload(name):
    """Workload recipe by name: mesh, degree, geometry, operator options."""
    if name == "cartesian_periodic_4x4x4_p2":
        return dict(mesh=dict(n=(4, 4, 4), periodic=True, mapping=0, amplitude=0.0), degree=2,
                    geom="cartesian", coeff=0)
    if name.startswith("deformed_dirichlet_32^3_p"):
        p = int(name.rsplit("_p", 1)[1])
        return dict(mesh=dict(n=(32, 32, 32), periodic=False, mapping=1, amplitude=0.1), degree=p,
                    geom="full", coeff=1)
    raise KeyError(name)


def paper_size_schedule(p):
    """Cells per direction of the paper's larger-than-cache schedule
    (8-57 M dofs): 128^3 for p = 1-2, 64^3 for p = 3-5, 32^3 for p = 6-8."""
    return 128 if p <= 2 else 64 if p <= 5 else 32

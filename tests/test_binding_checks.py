"""The Python binding refuses arrays whose shape, type or placement does not match the handle's
problem before it passes a pointer to the library (the kernels read and write R whole volumes or
trace vectors, so a mismatched array would be read or written out of bounds).  No GPU: a binding
object without a library handle is enough, since every check runs before the library call."""
import numpy as np
import pytest

from paper_1801_08655_gb300 import hz

torch = pytest.importorskip("torch")


@pytest.fixture()
def solver():
    s = object.__new__(hz.Solver)
    s.lib, s.h = None, None          # any library call would fail: the checks must come first
    s.shape, s.K, s.P, s.n_layers, s.precision = (6, 5, 4), 2, 20, 3, "mixed"
    return s


def test_host_solve_checks_shapes_and_output(solver):
    with pytest.raises(ValueError):
        solver.solve_host(np.zeros((2, 6, 5, 5), np.complex128))             # wrong grid
    with pytest.raises(ValueError):
        solver.solve_host(np.zeros((6, 5, 4), np.complex128))                # no column axis
    rhs = np.zeros((2, 6, 5, 4), np.complex128)
    for bad in (np.zeros((2, 6, 5, 4)), np.zeros((3, 6, 5, 4), np.complex128),
                np.zeros((2, 6, 5, 8), np.complex128)[..., ::2]):
        with pytest.raises(ValueError):
            solver.solve_host(rhs, u=bad)                                    # float, wrong R, strided


def test_device_entry_points_check_shapes(solver):
    cpu = torch.zeros((2, 6, 5, 4), dtype=torch.complex128)
    with pytest.raises(ValueError):
        solver.solve(cpu)                                                    # not on the device
    with pytest.raises(ValueError):
        solver.polarized_rhs(cpu)
    with pytest.raises(ValueError):
        solver.apply_mpol(torch.zeros(solver.trace_shape(2), dtype=torch.complex128))
    with pytest.raises(ValueError):
        solver.apply_precond(torch.zeros((2, 2, 2, 2, 5, 5), dtype=torch.complex128))
    with pytest.raises(ValueError):
        solver.reconstruct(cpu, torch.zeros((2, 2, 2, 5, 4), dtype=torch.complex128))
    with pytest.raises(ValueError):
        solver.volume_residual_noalloc(cpu, cpu)

"""Pins of the variable-density operator div(b grad u) + omega^2 m u (b = 1/rho) in the oracle:
it reduces to the constant-density operator for b = 1, stays complex symmetric, converges to the
continuous operator at second order on a manufactured solution, and the method of polarized traces
built on it (local operators with the layers' b, interface weights with b at the interface half
plane) reproduces the global direct solve exactly (Green's representation formula) and through
its GMRES.  No GPU."""
import numpy as np

from oracle import direct, discretization as disc, polarized
from paper_1801_08655_gb300 import workloads as W


def test_unit_density_is_the_laplacian_operator():
    p = W.small_problem(12, 3, 2, seed=51, R=1)
    A0 = disc.global_operator(p.m, p.omega, p.npml, p.C)
    A1 = disc.global_operator(p.m, p.omega, p.npml, p.C, b=np.ones_like(p.m))
    assert abs(A1 - A0).max() == 0.0


def test_variable_density_operator_is_complex_symmetric():
    p = W.small_problem(12, 3, 2, seed=52, R=1)
    b = W.density_smooth_random(12, seed=53)
    A = disc.global_operator(p.m, p.omega, p.npml, p.C, b=b)
    assert abs(A - A.T).max() == 0.0
    assert abs(A - A.conj().T).max() > 1e-3     # not Hermitian (PML, complex stretching)


def test_second_order_convergence_to_the_continuous_operator():
    """No PML, Dirichlet box: (A u_h)(x) - [div(b grad u) + omega^2 m u](x) at nodes away from the
    boundary falls like h^2 for smooth u, b, m."""
    omega = 3.0

    def err(n):
        h = 1.0 / (n + 1)
        x = (np.arange(n) + 1) * h
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        u = np.sin(np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(np.pi * Z)
        b = 1.0 + 0.5 * X + 0.3 * Y * Z
        m = 1.0 + X
        # grad b and the Laplacian of u in closed form
        ux = np.pi * np.cos(np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(np.pi * Z)
        uy = 2 * np.pi * np.sin(np.pi * X) * np.cos(2 * np.pi * Y) * np.sin(np.pi * Z)
        uz = np.pi * np.sin(np.pi * X) * np.sin(2 * np.pi * Y) * np.cos(np.pi * Z)
        lap = -(1 + 4 + 1) * np.pi ** 2 * u
        exact = b * lap + 0.5 * ux + 0.3 * Z * uy + 0.3 * Y * uz + omega ** 2 * m * u
        p = disc.global_profiles(n, 0, 0.0, omega, h)
        A = disc.assemble(m, omega, p, p, p, h, b=b)
        Au = (A @ u.ravel()).reshape(u.shape)
        sl = slice(2, n - 2)
        return np.abs(Au - exact)[sl, sl, sl].max()

    e1, e2 = err(15), err(31)
    assert 3.2 < e1 / e2 < 4.8, (e1, e2)


def test_polarized_traces_exact_with_variable_density():
    p = W.small_problem(18, 3, 3, seed=54, R=1)
    b = W.density_smooth_random(18, seed=55, corr=3.0)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f, b=b)[0]
    M = polarized.PolarizedModel(p.m, p.omega, p.npml, p.C, p.n_layers, b=b)
    ur = M.reconstruct(f[0], M.traces_of(u))
    assert np.linalg.norm(ur - u) / np.linalg.norm(u) < 1e-12
    us, its = M.solve(f[0], tol=1e-11)
    assert np.linalg.norm(us - u) / np.linalg.norm(u) < 1e-9
    # the constant-density model on the same medium gives a different field
    u0 = direct.solve(p.m, p.omega, p.npml, p.C, f)[0]
    assert np.linalg.norm(u0 - u) / np.linalg.norm(u) > 1e-2

"""GPU parity of the variable-density operator div(b grad u) + omega^2 m u (b = 1/rho, created
with hz_create_ex) against the oracle: local solves against SciPy's direct solve of the oracle's
local operator, the FP64 volume residual against the oracle's assembled operator (both entry
points), end-to-end solves against the global direct solve in both precisions, and the 64^3
variable-density workload against stored oracle samples.  Tolerances as in test_gpu_parity."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import direct, discretization as D
from paper_1801_08655_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STAGE_TOL = {"fp64": 1e-10, "mixed": 2e-4}
E2E_TOL = {"fp64": 1e-6, "mixed": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.fixture(scope="module")
def hz():
    from paper_1801_08655_gb300 import build, hz as _hz
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _hz


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_density_layer_solve_and_residual(hz, precision):
    p = W.small_problem(20, 4, 3, seed=61, R=2)
    b = W.density_smooth_random(20, seed=62, corr=3.0)
    s = hz.Solver(p.m, p.omega, p.npml, p.C, p.n_layers, precision=precision, b=b)
    s.factor()
    parts = D.layer_partition(p.n, p.npml, p.n_layers)
    rng = np.random.default_rng(7)
    for ell in range(p.n_layers):
        lo, hi, zlo, zhi = s.layer_info(ell)
        H = D.local_operator(p.m, p.omega, ell, parts, p.npml, p.npml, p.C, b=b).tocsc()
        g = rng.standard_normal((2, H.shape[0])) + 1j * rng.standard_normal((2, H.shape[0]))
        ref = spla.splu(H).solve(g.T).T
        w = s.layer_solve(ell, cuda(g.reshape(2, zhi - zlo + 1, p.n, p.n))).cpu().numpy().reshape(2, -1)
        assert rel(w, ref) < STAGE_TOL[precision], (ell, rel(w, ref))
    # FP64 volume residual against the oracle's operator, through both residual entry points
    A = D.global_operator(p.m, p.omega, p.npml, p.C, b=b)
    Sc = D.row_scaling(p.n, p.npml, p.C, p.omega)
    f = p.rhs()
    u = rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape)
    rel_gpu, r_gpu = s.volume_residual(cuda(f), cuda(u), want_r=True)
    rel_na = s.volume_residual_noalloc(cuda(f), cuda(u))
    for k in range(p.R):
        r_ref = (Sc * f[k]).ravel() - A @ u[k].ravel()
        assert rel(r_gpu[k].cpu().numpy().ravel(), r_ref) < 1e-13
        assert rel_gpu[k] == pytest.approx(np.linalg.norm(r_ref) / np.linalg.norm((Sc * f[k]).ravel()), rel=1e-12)
        assert rel_na[k] == pytest.approx(rel_gpu[k], rel=1e-12)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,npml,L,R", [(20, 4, 4, 3), (22, 4, 2, 2)])
def test_density_end_to_end(hz, precision, n, npml, L, R):
    p = W.small_problem(n, npml, L, seed=63 + n + L, R=R)
    b = W.density_smooth_random(n, seed=64 + n, corr=3.0)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f, b=b)
    s = hz.Solver(p.m, p.omega, p.npml, p.C, p.n_layers, precision=precision, b=b)
    s.factor()
    ug, info, st = s.solve(cuda(f))
    ug = ug.cpu().numpy()
    for r in range(R):
        assert rel(ug[r], u[r]) < E2E_TOL[precision], (r, rel(ug[r], u[r]))
    # a constant-density solve of the same medium is a different field
    u0 = direct.solve(p.m, p.omega, p.npml, p.C, f[:1])[0]
    assert rel(ug[0], u0) > 1e-2
    s.close()


def test_density_rejects_bad_b(hz):
    p = W.small_problem(12, 3, 2, seed=65, R=1)
    b = np.ones_like(p.m)
    b[3, 4, 5] = -1.0
    with pytest.raises(hz.HzError) as e:
        hz.Solver(p.m, p.omega, p.npml, p.C, 2, b=b)
    assert e.value.status == hz.HZ_ERR_ARG
    b[3, 4, 5] = np.nan
    with pytest.raises(hz.HzError) as e:
        hz.Solver(p.m, p.omega, p.npml, p.C, 2, b=b)
    assert e.value.status == hz.HZ_ERR_NONFINITE


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_density_workload_against_stored_oracle_samples(hz, precision):
    """64^3 smooth random medium and density, 8 layers, 16 sources (the second workload)."""
    d = np.load(os.path.join(os.path.dirname(__file__), "golden", "cfg2_64cube_density_samples.npz"))
    p = W.config(2)
    b = W.density_smooth_random(p.n, seed=int(d["density_seed"]))
    s = hz.Solver(p.m, p.omega, p.npml, p.C, p.n_layers, precision=precision, b=b)
    s.factor()
    u, info, st = s.solve(cuda(p.rhs()))
    uu = u.cpu().numpy().reshape(p.R, -1)
    for r in range(p.R):
        assert rel(uu[r, d["idx"]], d["u"][r]) < E2E_TOL[precision], (r, rel(uu[r, d["idx"]], d["u"][r]))
        assert np.linalg.norm(uu[r]) == pytest.approx(d["norms"][r], rel=E2E_TOL[precision])
    s.close()

"""GPU parity of the explicit trace-to-trace Green's blocks (hz_trace_blocks), through the C ABI.

With the blocks built, M_pol and the preconditioner of Eq. 16 are dense block products instead of
local solves.  They are compared element-wise with the same handle's local-solve operators and
with the oracle's model (matrix-free Algorithms 4-9); end-to-end solutions with the global direct
solve and with the stored 64^3 oracle samples.  Tolerances as in the other parity tests: FP64
stages 1e-10, mixed stages 2e-4 (complex64 blocks from complex64 local solves, FP32 sums), end to
end 1e-6 (FP64) and 1e-5 (mixed, after FP64 defect correction).  The grids include one whose
pair length 2 nx ny is not a multiple of the kernel's 64-entry staging step and column counts
that are not multiples of its column groups.
"""
import os

import numpy as np
import pytest

from oracle import direct, polarized
from paper_1801_08655_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STAGE_TOL = {"fp64": 1e-10, "mixed": 2e-4}
E2E_TOL = {"fp64": 1e-6, "mixed": 1e-5}


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def hz():
    from paper_1801_08655_gb300 import build, hz as _hz
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _hz


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_solver(hz, p, precision):
    s = hz.Solver(p.m, p.omega, p.npml, p.C, p.n_layers, precision=precision)
    s.factor()
    return s


def block_bytes(p, precision):
    n2 = 2 * p.n * p.n
    return (4 * p.n_layers - 6) * n2 * n2 * (16 if precision == "fp64" else 8)


@pytest.fixture(scope="module")
def case18():
    p = W.small_problem(18, 3, 4, seed=71, R=3)     # 2 nx ny = 648
    return p, polarized.PolarizedModel(p.m, p.omega, p.npml, p.C, p.n_layers)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("R", [3, 20])
def test_block_operators_match_local_solves_and_oracle(hz, case18, precision, R):
    p, M = case18
    s = make_solver(hz, p, precision)
    rng = np.random.default_rng(17 + R)
    shp = s.trace_shape(R)
    x = cuda(rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    y_ls, z_ls = s.apply_mpol(x).cpu().numpy(), s.apply_precond(x).cpu().numpy()
    nbytes = s.trace_blocks(max_cols=R)
    assert nbytes == block_bytes(p, precision)
    y_tb, z_tb = s.apply_mpol(x).cpu().numpy(), s.apply_precond(x).cpu().numpy()
    assert rel(y_tb, y_ls) < STAGE_TOL[precision], rel(y_tb, y_ls)
    assert rel(z_tb, z_ls) < STAGE_TOL[precision], rel(z_tb, z_ls)
    xh = x.cpu().numpy()
    for r in (0, R - 1):
        yd, yu = M.apply_Mpol(xh[r, 0], xh[r, 1])
        assert rel(y_tb[r, 0], yd) < STAGE_TOL[precision] and rel(y_tb[r, 1], yu) < STAGE_TOL[precision]
        zd, zu = M.apply_P(xh[r, 0], xh[r, 1])
        assert rel(z_tb[r, 0], zd) < STAGE_TOL[precision] and rel(z_tb[r, 1], zu) < STAGE_TOL[precision]
    # detail profiling attributes one block-product launch per M_pol apply reading every block once
    s.profile_begin(detail=True)
    s.apply_mpol(x)
    s.profile_end()
    k2 = s.profile_kernel(2)
    assert k2["launches"] == 1 and k2["ms"] > 0
    assert k2["bytes"] == pytest.approx(nbytes, rel=1e-12)
    assert k2["flops"] == pytest.approx(8.0 * R * nbytes / (16 if precision == "fp64" else 8), rel=1e-12)
    # more columns than max_cols: the local solves again, on the same handle
    if R > 3:
        s.trace_blocks(max_cols=R - 1)
        assert rel(s.apply_mpol(x).cpu().numpy(), y_ls) < STAGE_TOL[precision]
    # released: the local solves
    assert s.trace_blocks(0) == 0
    assert rel(s.apply_precond(x).cpu().numpy(), z_ls) < STAGE_TOL[precision]
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,npml,L,R", [(20, 4, 4, 3), (18, 3, 2, 1), (24, 4, 6, 5)])
def test_block_solve_end_to_end(hz, precision, n, npml, L, R):
    p = W.small_problem(n, npml, L, seed=300 + n + L, R=R)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)
    s = make_solver(hz, p, precision)
    s.trace_blocks(max_cols=32)
    ug, info, st = s.solve(cuda(f))
    ug = ug.cpu().numpy()
    for r in range(R):
        assert rel(ug[r], u[r]) < E2E_TOL[precision], (r, rel(ug[r], u[r]))
    assert max(i.iters for i in info) <= 12
    s.close()


def test_config2_with_trace_blocks_against_stored_oracle_samples(hz):
    """64^3 smooth random medium, 8 layers, 16 sources, mixed precision with the explicit blocks
    (the workload they are built for): the sampled values and norms of the oracle's global direct
    solve (tests/golden/make_golden.py)."""
    d = np.load(os.path.join(os.path.dirname(__file__), "golden", "cfg2_64cube_smooth_samples.npz"))
    p = W.config(2)
    f = p.rhs()
    s = make_solver(hz, p, "mixed")
    assert s.trace_blocks(max_cols=p.R) == block_bytes(p, "mixed")
    u, info, st = s.solve(cuda(f))
    uu = u.cpu().numpy().reshape(p.R, -1)
    for r in range(p.R):
        assert rel(uu[r, d["idx"]], d["u"][r]) < E2E_TOL["mixed"], (r, rel(uu[r, d["idx"]], d["u"][r]))
        assert np.linalg.norm(uu[r]) == pytest.approx(d["norms"][r], rel=E2E_TOL["mixed"])
    s.close()


def test_trace_block_errors_are_statuses(hz):
    p = W.small_problem(16, 3, 3, seed=77, R=1)
    s = hz.Solver(p.m, p.omega, p.npml, p.C, p.n_layers, precision="mixed")
    with pytest.raises(hz.HzError) as e:
        s.trace_blocks(8)
    assert e.value.status == hz.HZ_ERR_STATE
    s.factor()
    with pytest.raises(hz.HzError) as e:
        s.trace_blocks(-1)
    assert e.value.status == hz.HZ_ERR_ARG
    # released and built again: the same solution
    f = cuda(p.rhs())
    s.trace_blocks(4)
    u1 = s.solve(f)[0].cpu().numpy()
    s.trace_blocks(0)
    s.trace_blocks(4)
    u2 = s.solve(f)[0].cpu().numpy()
    assert rel(u2, u1) < 1e-6
    s.close()

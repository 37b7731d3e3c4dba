"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Every comparison is element-wise on the same seeded inputs.  Tolerances:
* FP64 mode: 1e-10 relative (L2) for stages, and the end-to-end solution within 1e-6
  of the global direct solve (expected ~1e-10).
* Mixed mode (complex64 factors and local solves): stages within 2e-4 relative (FP32
  rounding through an unpivoted LDL^T of a PML-padded Helmholtz operator); the end-to-end
  solution after FP64 defect correction within 1e-5 of the global direct solve.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import direct, discretization as D, polarized
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


def make_solver(hz, p, precision, n_layers=None, npml_local=-1):
    s = hz.Solver(p.m, p.omega, p.npml, p.C, n_layers or p.n_layers, precision=precision,
                  npml_local=npml_local)
    s.factor()
    return s


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_layer_solve_matches_local_direct_solve(hz, precision):
    p = W.config(1)
    s = make_solver(hz, p, precision)
    parts = D.layer_partition(p.n, p.npml, p.n_layers)
    rng = np.random.default_rng(5)
    for ell in range(p.n_layers):
        lo, hi, zlo, zhi = s.layer_info(ell)
        assert (zlo, zhi) == D.local_grid(ell, parts, p.n, p.npml)
        assert (lo, hi) == parts[ell]
        H = D.local_operator(p.m, p.omega, ell, parts, p.npml, p.npml, p.C).tocsc()
        nzl = zhi - zlo + 1
        g = rng.standard_normal((3, nzl, p.n, p.n)) + 1j * rng.standard_normal((3, nzl, p.n, p.n))
        ref = spla.spsolve(H, g.reshape(3, -1).T).T.reshape(g.shape)
        w = s.layer_solve(ell, cuda(g)).cpu().numpy()
        assert rel(w, ref) < STAGE_TOL[precision], (ell, rel(w, ref))
    s.close()


@pytest.fixture(scope="module")
def small_case():
    p = W.small_problem(20, 4, 4, seed=31, R=2)
    M = polarized.PolarizedModel(p.m, p.omega, p.npml, p.C, p.n_layers)
    return p, M


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_polarized_stages_match_oracle_model(hz, small_case, precision):
    p, M = small_case
    s = make_solver(hz, p, precision)
    f = p.rhs()
    fpol = s.polarized_rhs(cuda(f)).cpu().numpy()
    rng = np.random.default_rng(9)
    shp = s.trace_shape(p.R)
    x = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    y = s.apply_mpol(cuda(x)).cpu().numpy()
    z = s.apply_precond(cuda(x)).cpu().numpy()
    for r in range(p.R):
        fd, fu = M.polarized_rhs(f[r])
        assert rel(fpol[r, 0], fd) < STAGE_TOL[precision]
        assert rel(fpol[r, 1], fu) < STAGE_TOL[precision]
        yd, yu = M.apply_Mpol(x[r, 0], x[r, 1])
        assert rel(y[r, 0], yd) < STAGE_TOL[precision]
        assert rel(y[r, 1], yu) < STAGE_TOL[precision]
        zd, zu = M.apply_P(x[r, 0], x[r, 1])
        assert rel(z[r, 0], zd) < STAGE_TOL[precision]
        assert rel(z[r, 1], zu) < STAGE_TOL[precision]
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_reconstruction_from_exact_traces(hz, small_case, precision):
    p, M = small_case
    s = make_solver(hz, p, precision)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)
    t = np.stack([M.traces_of(u[r]) for r in range(p.R)])
    ug = s.reconstruct(cuda(f), cuda(t)).cpu().numpy()
    assert rel(ug, u) < STAGE_TOL[precision]
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_end_to_end_config1(hz, precision):
    p = W.config(1)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)
    s = make_solver(hz, p, precision)
    ug, info, st = s.solve(cuda(f))
    ug = ug.cpu().numpy()
    err = rel(ug, u)
    assert err < E2E_TOL[precision], err
    assert 1 <= info[0].iters <= 10
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,npml,L,R", [(20, 4, 4, 3), (24, 4, 6, 5), (16, 3, 1, 2), (18, 3, 2, 1)])
def test_end_to_end_small(hz, precision, n, npml, L, R):
    p = W.small_problem(n, npml, L, seed=100 + n + L, R=R)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)
    s = make_solver(hz, p, precision)
    ug, info, st = s.solve(cuda(f))
    ug = ug.cpu().numpy()
    for r in range(R):
        assert rel(ug[r], u[r]) < E2E_TOL[precision], (r, rel(ug[r], u[r]))
    s.close()


def test_batch_equals_alone(hz):
    """A right-hand side gives the same answer alone and batched with others."""
    p = W.small_problem(20, 4, 4, seed=77, R=4)
    f = p.rhs()
    s = make_solver(hz, p, "mixed")
    ub, _, _ = s.solve(cuda(f))
    u1, _, _ = s.solve(cuda(f[2:3]))
    assert rel(u1.cpu().numpy()[0], ub.cpu().numpy()[2]) < 1e-6
    s.close()


def test_volume_residual_matches_oracle_operator(hz):
    p = W.small_problem(14, 3, 2, seed=3, R=2)
    s = make_solver(hz, p, "fp64")
    rng = np.random.default_rng(1)
    u = rng.standard_normal((2, 14, 14, 14)) + 1j * rng.standard_normal((2, 14, 14, 14))
    f = p.rhs()
    rel_gpu, r = s.volume_residual(cuda(f), cuda(u), want_r=True)
    A = D.global_operator(p.m, p.omega, p.npml, p.C)
    S = D.row_scaling(14, p.npml, p.C, p.omega)
    for q in range(2):
        ref = (S * f[q]).ravel() - A @ u[q].ravel()
        assert rel(r[q].cpu().numpy().ravel(), ref) < 1e-13
        assert rel_gpu[q] == pytest.approx(np.linalg.norm(ref) / np.linalg.norm((S * f[q]).ravel()), rel=1e-10)
    s.close()


def test_errors_are_statuses(hz):
    p = W.small_problem(12, 3, 2, seed=3, R=1)
    s = hz.Solver(p.m, p.omega, p.npml, p.C, 2, precision="fp64")
    with pytest.raises(hz.HzError) as e:
        s.solve(cuda(p.rhs()))
    assert e.value.status == hz.HZ_ERR_STATE
    s.close()
    with pytest.raises(hz.HzError) as e:
        hz.Solver(p.m, -1.0, p.npml, p.C, 2)
    assert e.value.status == hz.HZ_ERR_ARG
    bad = p.m.copy()
    bad[3, 3, 3] = np.nan
    with pytest.raises(hz.HzError) as e:
        hz.Solver(bad, p.omega, p.npml, p.C, 2)
    assert e.value.status == hz.HZ_ERR_NONFINITE


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config2_against_stored_oracle_samples(hz, precision):
    """64^3 smooth random medium, 8 layers, 16 sources: sampled values of the oracle's
    global direct solve (tests/golden/make_golden.py) vs the GPU solution."""
    import os
    d = np.load(os.path.join(os.path.dirname(__file__), "golden", "cfg2_64cube_smooth_samples.npz"))
    p = W.config(2)
    f = p.rhs()
    s = make_solver(hz, p, precision)
    u, info, st = s.solve(cuda(f))
    uu = u.cpu().numpy().reshape(p.R, -1)
    for r in range(p.R):
        assert rel(uu[r, d["idx"]], d["u"][r]) < E2E_TOL[precision], (r, rel(uu[r, d["idx"]], d["u"][r]))
        assert np.linalg.norm(uu[r]) == pytest.approx(d["norms"][r], rel=E2E_TOL[precision])
    assert max(i.iters for i in info) <= 10
    s.close()


def test_solve_on_a_nonblocking_stream(hz):
    """Work queued on a non-blocking stream (as torch creates them) is complete before the
    library reads results back: residual norms and the solution are right."""
    p = W.small_problem(20, 4, 4, seed=55, R=2)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)
    st = torch.cuda.Stream()
    s = hz.Solver(p.m, p.omega, p.npml, p.C, p.n_layers, precision="mixed", stream=st)
    s.factor()
    with torch.cuda.stream(st):
        fd = cuda(f)
    st.synchronize()
    ug, info, _ = s.solve(fd)
    st.synchronize()
    assert rel(ug.cpu().numpy(), u) < E2E_TOL["mixed"]
    assert all(0.0 < i.volume_relres < 1e-8 for i in info)
    s.close()


@pytest.mark.parametrize("cfg", ["0", "1"])
@pytest.mark.parametrize("ncols", [64, 128, 130])
def test_tensor_core_layer_solve(hz, ncols, cfg, monkeypatch):
    """With the tensor-core path enabled, mixed-precision layer solves with >= 64 columns run on
    the tcgen05 kernel (split TF32); they must match the local direct solve within the stage
    tolerance."""
    monkeypatch.setenv("HZ_SUBST_TC", "1")
    monkeypatch.setenv("HZ_TC_MIN_TILES", "3")   # small fronts too: partial quads, masked rows
    monkeypatch.setenv("HZ_TC_CFG", cfg)           # one block per work item (0) or persistent (1) ...
    monkeypatch.setenv("HZ_AUTOTUNE", "0")         # ... as set, not as the autotuner would choose
    p = W.config(1)
    s = make_solver(hz, p, "mixed")
    parts = D.layer_partition(p.n, p.npml, p.n_layers)
    rng = np.random.default_rng(ncols)
    ell = 1
    lo, hi, zlo, zhi = s.layer_info(ell)
    H = D.local_operator(p.m, p.omega, ell, parts, p.npml, p.npml, p.C).tocsc()
    g = rng.standard_normal((ncols, zhi - zlo + 1, p.n, p.n)) + 1j * rng.standard_normal((ncols, zhi - zlo + 1, p.n, p.n))
    ref = spla.spsolve(H, g.reshape(ncols, -1).T).T.reshape(g.shape)
    w = s.layer_solve(ell, cuda(g)).cpu().numpy()
    for c in (0, ncols // 2, ncols - 1):
        assert rel(w[c], ref[c]) < STAGE_TOL["mixed"], (c, rel(w[c], ref[c]))
    s.close()


def test_tensor_core_polarized_stages(hz, small_case, monkeypatch):
    """M_pol on 4R = 128 stacked columns takes the tensor-core path when it is enabled."""
    monkeypatch.setenv("HZ_SUBST_TC", "1")
    monkeypatch.setenv("HZ_TC_MIN_TILES", "3")
    p, M = small_case
    s = make_solver(hz, p, "mixed")
    rng = np.random.default_rng(21)
    R = 32
    shp = s.trace_shape(R)
    x = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    y = s.apply_mpol(cuda(x)).cpu().numpy()
    for r in (0, 17, 31):
        yd, yu = M.apply_Mpol(x[r, 0], x[r, 1])
        assert rel(y[r, 0], yd) < STAGE_TOL["mixed"]
        assert rel(y[r, 1], yu) < STAGE_TOL["mixed"]
    s.close()


def test_tensor_core_and_cuda_core_paths_agree(hz, monkeypatch):
    """Forced tensor-core substitution, forced CUDA-core substitution and the autotuned choice
    between them (the default) give the same refined solution."""
    p = W.config(2)
    f = p.rhs()
    outs = []
    for flag in ("1", "0", "2"):
        monkeypatch.setenv("HZ_SUBST_TC", flag)
        s = make_solver(hz, p, "mixed")
        u, info, _ = s.solve(cuda(f))
        outs.append(u.cpu().numpy())
        if flag == "2":
            # the tuner timed tensor-core candidates for the batches wide enough for them
            assert "(TC, KS" in s.tuning_report()
        s.close()
    assert rel(outs[0], outs[1]) < 1e-8
    assert rel(outs[2], outs[1]) < 1e-8


@pytest.mark.parametrize("split", ["3", "1"])
def test_tensor_core_preconditioner_precision(hz, small_case, split, monkeypatch):
    """P on 64 trace columns with the tensor-core path: with three-term TF32 products it matches
    the oracle's P within the mixed stage tolerance; with single-term TF32 products (the option
    HZ_PRECOND_SPLIT=1) within 5e-3, while M_pol keeps the three-term accuracy."""
    monkeypatch.setenv("HZ_SUBST_TC", "1")
    monkeypatch.setenv("HZ_TC_MIN_TILES", "2")
    monkeypatch.setenv("HZ_PRECOND_SPLIT", split)
    p, M = small_case
    s = make_solver(hz, p, "mixed")
    R = 64
    rng = np.random.default_rng(77)
    shp = s.trace_shape(R)
    x = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    z = s.apply_precond(cuda(x)).cpu().numpy()
    y = s.apply_mpol(cuda(x)).cpu().numpy()
    tol = STAGE_TOL["mixed"] if split == "3" else 5e-3
    for r in (0, 33, 63):
        zd, zu = M.apply_P(x[r, 0], x[r, 1])
        assert rel(z[r, 0], zd) < tol and rel(z[r, 1], zu) < tol, (r, rel(z[r, 0], zd), rel(z[r, 1], zu))
        yd, yu = M.apply_Mpol(x[r, 0], x[r, 1])
        assert rel(y[r, 0], yd) < STAGE_TOL["mixed"] and rel(y[r, 1], yu) < STAGE_TOL["mixed"]
    s.close()


def test_fast_preconditioner_solution_unchanged(hz, monkeypatch):
    """The solution does not depend on the precision of the preconditioner's tensor-core
    products (they only steer GMRES): single- and three-term runs agree after the FP64 residual
    check, and both meet the oracle's solution."""
    monkeypatch.setenv("HZ_SUBST_TC", "1")
    monkeypatch.setenv("HZ_TC_MIN_TILES", "2")
    p = W.small_problem(24, 4, 4, seed=41, R=64)
    f = p.rhs()
    outs, iters = [], []
    for split in ("3", "1"):
        monkeypatch.setenv("HZ_PRECOND_SPLIT", split)
        s = make_solver(hz, p, "mixed")
        u, info, _ = s.solve(cuda(f))
        outs.append(u.cpu().numpy())
        iters.append(info[0].iters)
        assert all(i.volume_relres < 1e-8 for i in info)
        s.close()
    assert rel(outs[0], outs[1]) < 1e-7
    ref = direct.solve(p.m, p.omega, p.npml, p.C, f[:2])
    assert rel(outs[1][:2], ref) < E2E_TOL["mixed"]
    assert iters[1] <= iters[0] + 2, iters


def test_persistent_tensor_core_kernel_matches(hz, monkeypatch):
    """The persistent tensor-core kernel (blocks walking several work items each, alternating
    accumulator buffers, split reductions) gives the same M_pol and P as one block per work item
    and as the CUDA-core kernels, on a 64^3 problem with 256 stacked columns."""
    p = W.config(2)
    rng = np.random.default_rng(123)
    outs = {}
    x = None
    for name, env in (("simt", {"HZ_SUBST_TC": "0"}), ("tc0", {"HZ_SUBST_TC": "1", "HZ_TC_CFG": "0"}),
                      ("tcp", {"HZ_SUBST_TC": "1", "HZ_TC_CFG": "1"})):
        monkeypatch.setenv("HZ_AUTOTUNE", "0")
        monkeypatch.setenv("HZ_TC_MIN_TILES", "2")
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        s = make_solver(hz, p, "mixed")
        if x is None:
            shp = s.trace_shape(64)
            x = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
        y = s.apply_mpol(cuda(x)).cpu().numpy()
        z = s.apply_precond(cuda(x)).cpu().numpy()
        outs[name] = (y, z)
        s.close()
    for name in ("tc0", "tcp"):
        assert rel(outs[name][0], outs["simt"][0]) < 1e-4, name
        assert rel(outs[name][1], outs["simt"][1]) < 1e-4, name
    assert rel(outs["tcp"][0], outs["tc0"][0]) < 1e-5
    assert rel(outs["tcp"][1], outs["tc0"][1]) < 1e-5


def test_profile_detail_attributes_launches_by_kernel_kind(hz, small_case, monkeypatch):
    """Detail profiling times every substitution launch and attributes it to the CUDA-core or
    the tensor-core kernel; the algorithmic flops of the two kinds add up to those of the
    substitution calls."""
    monkeypatch.setenv("HZ_SUBST_TC", "1")
    monkeypatch.setenv("HZ_TC_MIN_TILES", "3")
    p, M = small_case
    s = make_solver(hz, p, "mixed")
    R = 32
    x = cuda(np.random.default_rng(5).standard_normal(s.trace_shape(R)) + 0j)
    s.apply_mpol(x)
    s.profile_begin(detail=True)
    s.apply_mpol(x)
    tot = s.profile_end()
    k0, k1 = s.profile_kernel(0), s.profile_kernel(1)
    assert tot["calls"] > 0 and k0["launches"] > 0 and k1["launches"] > 0
    assert k0["ms"] > 0 and k1["ms"] > 0
    assert abs(k0["flops"] + k1["flops"] - tot["flops"]) <= 0.05 * tot["flops"]
    assert s.profile_kernel(2)["launches"] == 0   # no explicit trace blocks on this handle
    with pytest.raises(RuntimeError):
        s.profile_kernel(3)
    s.close()


def test_graph_replay_matches_direct_launches(hz, monkeypatch):
    """The GMRES matrix-vector product replayed as a captured CUDA graph gives the same
    solution as issuing its launches directly."""
    p = W.small_problem(20, 4, 4, seed=91, R=3)
    f = p.rhs()
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("HZ_GRAPHS", flag)
        s = make_solver(hz, p, "fp64")
        u, info, _ = s.solve(cuda(f))
        outs.append(u.cpu().numpy())
        u2, _, _ = s.solve(cuda(f))  # second solve replays the cached plan / graph
        assert rel(u2.cpu().numpy(), outs[-1]) < 1e-13
        s.close()
    assert rel(outs[0], outs[1]) < 1e-12


def test_group_solve_matches_individual_solves(hz):
    """hz_solve_group on problems of different sizes, layer counts and R (each on its own
    stream) gives each member the same answer as solving it alone, and matches the oracle."""
    specs = [(16, 3, 2, 1), (20, 4, 4, 3), (24, 4, 3, 5)]
    solvers, rhs, refs = [], [], []
    for k, (n, npml, L, R) in enumerate(specs):
        p = W.small_problem(n, npml, L, seed=300 + k, R=R)
        st = torch.cuda.Stream()
        s = hz.Solver(p.m, p.omega, p.npml, p.C, L, precision="mixed", stream=st)
        s.factor()
        solvers.append(s)
        f = p.rhs()
        rhs.append(cuda(f))
        refs.append(direct.solve(p.m, p.omega, p.npml, p.C, f))
    torch.cuda.synchronize()
    us, infos, sts = hz.solve_group(solvers, rhs)
    torch.cuda.synchronize()
    for k, s in enumerate(solvers):
        alone, _, _ = s.solve(rhs[k])
        torch.cuda.synchronize()
        assert rel(us[k].cpu().numpy(), alone.cpu().numpy()) < 1e-6
        assert rel(us[k].cpu().numpy(), refs[k]) < E2E_TOL["mixed"]
        assert sts[k] == 0
        s.close()


@pytest.mark.parametrize("min_upd", ["32", "0"])
def test_tensor_core_factorization_layer_solve(hz, min_upd, monkeypatch):
    """Local solves of a layer factored with the tensor-core L21 and Schur products on every front
    with >= 32 update unknowns (min_upd 32: ragged front sizes, partial 128-row tiles, fronts of
    one own tile) and with the panel steps alone (0), against SciPy's local direct solve."""
    monkeypatch.setenv("HZ_FACTOR_TC_MIN", min_upd)
    p = W.small_problem(28, 4, 2, seed=41, R=1)
    s = make_solver(hz, p, "mixed")
    parts = D.layer_partition(p.n, p.npml, p.n_layers)
    rng = np.random.default_rng(9)
    for ell in range(p.n_layers):
        lo, hi, zlo, zhi = s.layer_info(ell)
        H = D.local_operator(p.m, p.omega, ell, parts, p.npml, p.npml, p.C).tocsc()
        g = rng.standard_normal((3, H.shape[0])) + 1j * rng.standard_normal((3, H.shape[0]))
        w_ref = spla.splu(H).solve(g.T).T
        w = s.layer_solve(ell, cuda(g.reshape(3, zhi - zlo + 1, p.n, p.n))).cpu().numpy().reshape(3, -1)
        assert rel(w, w_ref) < STAGE_TOL["mixed"], (ell, rel(w, w_ref))
    s.close()


def test_tensor_core_factorization_end_to_end(hz, monkeypatch):
    """A mixed-precision solve whose factors come from the tensor-core products on every eligible
    front matches the global direct solve to the end-to-end tolerance."""
    monkeypatch.setenv("HZ_FACTOR_TC_MIN", "32")
    p = W.small_problem(24, 4, 3, seed=42, R=3)
    f = p.rhs()
    u_ref = direct.solve(p.m, p.omega, p.npml, p.C, f)
    s = make_solver(hz, p, "mixed")
    u, info, _ = s.solve(cuda(f))
    for r in range(p.R):
        assert rel(u[r].cpu().numpy(), u_ref[r]) < E2E_TOL["mixed"]
    s.close()


@pytest.mark.parametrize("precision,R", [("fp64", 3), ("mixed", 3), ("fp64", 64), ("mixed", 64)])
def test_sparse_substitution_matches_full(hz, precision, R, monkeypatch):
    """Skipping the products of subtrees away from the interface planes (HZ_SPARSE=3, forward
    and backward) changes neither M_pol, nor the preconditioner, nor the polarized right-hand
    side, nor the end-to-end solution beyond rounding (the skipped products are exactly zero or
    unread); checked on 6 layers of a smooth medium with thick local pads.  At R = 64 M_pol's four
    stacked source blocks are 64-column jobs of their own, each skipping the products its own
    source and read-out planes do not need."""
    p = W.small_problem(22, 4, 6, seed=43, R=R)
    rng = np.random.default_rng(11)
    out = {}
    for flag in ("0", "3"):
        monkeypatch.setenv("HZ_SPARSE", flag)
        s = make_solver(hz, p, precision)
        f = cuda(p.rhs())
        x = torch.from_numpy(rng.standard_normal(s.trace_shape(p.R)) + 1j * rng.standard_normal(s.trace_shape(p.R))).cuda()
        out[flag] = dict(fpol=s.polarized_rhs(f).cpu().numpy(), mpol=s.apply_mpol(x).cpu().numpy(),
                         prec=s.apply_precond(x).cpu().numpy(), u=s.solve(f)[0].cpu().numpy())
        rng = np.random.default_rng(11)
        s.close()
    tol = 1e-12 if precision == "fp64" else 1e-5
    for k in ("fpol", "mpol", "prec", "u"):
        assert rel(out["3"][k], out["0"][k]) < tol, (k, rel(out["3"][k], out["0"][k]))


def test_tensor_core_wait_timeout_is_a_status(hz, monkeypatch):
    """A tensor-core pipeline wait that gives up ends the solve with HZ_ERR_TIMEOUT, not a fault or
    a hang: with a poll limit of 1 (HZ_TC_WAIT_POLLS) the first waits of every block give up before
    its MMAs are issued; each block still drains its own copies and committed MMAs and frees its
    tensor memory.  The same holds for the factorization's tensor-core products (hz_factor).  A
    fresh handle afterwards solves the same problem correctly."""
    p = W.config(1)
    rng = np.random.default_rng(1801 + 64)
    lo, hi = p.npml, p.n - p.npml
    src = np.stack([rng.integers(lo, hi, 64) for _ in range(3)], axis=1)
    wide = W.Problem("timeout_24cube_R64", p.n, p.npml, p.n_layers, p.omega, p.C, p.m, src)
    f = cuda(wide.rhs())
    monkeypatch.setenv("HZ_SUBST_TC", "1")
    monkeypatch.setenv("HZ_TC_MIN_TILES", "2")
    monkeypatch.setenv("HZ_TC_WAIT_POLLS", "1")
    # the factorization's tensor-core products give up too
    monkeypatch.setenv("HZ_FACTOR_TC_MIN", "32")
    s = hz.Solver(wide.m, wide.omega, wide.npml, wide.C, wide.n_layers, precision="mixed")
    with pytest.raises(hz.HzError) as e:
        s.factor()
    assert e.value.status == hz.HZ_ERR_TIMEOUT, e.value
    s.close()
    # factored without them, the solve's tensor-core substitutions give up
    monkeypatch.setenv("HZ_FACTOR_TC_MIN", "0")
    s = make_solver(hz, wide, "mixed")
    o = hz.default_opts("mixed")
    o.max_iter, o.max_refine = 2, 0
    with pytest.raises(hz.HzError) as e:
        s.solve(f, o)
    assert e.value.status == hz.HZ_ERR_TIMEOUT, e.value
    s.close()
    torch.cuda.synchronize()   # the context is still usable
    monkeypatch.delenv("HZ_TC_WAIT_POLLS")
    monkeypatch.delenv("HZ_FACTOR_TC_MIN")
    u_ref = direct.solve(wide.m, wide.omega, wide.npml, wide.C, wide.rhs())
    s = make_solver(hz, wide, "mixed")
    u, info, _ = s.solve(f)
    s.close()
    for r in range(wide.R):
        assert rel(u[r].cpu().numpy(), u_ref[r]) < E2E_TOL["mixed"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,npml,L,R", [(20, 4, 4, 3), (24, 4, 6, 5), (18, 3, 2, 1)])
def test_bicgstab_end_to_end(hz, precision, n, npml, L, R):
    """Bi-CGSTAB on the trace system (krylov = 1) reaches the global direct solve to the
    end-to-end tolerances, like GMRES."""
    p = W.small_problem(n, npml, L, seed=100 + n + L, R=R)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)
    s = make_solver(hz, p, precision)
    o = hz.default_opts(precision)
    o.krylov = 1
    ug, info, st = s.solve(cuda(f), o)
    ug = ug.cpu().numpy()
    for r in range(R):
        assert rel(ug[r], u[r]) < E2E_TOL[precision], (r, rel(ug[r], u[r]))
    assert all(i.trace_relres <= o.gmres_tol for i in info) or precision == "mixed"
    s.close()


@pytest.mark.parametrize("restart", [1, 2])
def test_low_restart_gmres_end_to_end(hz, restart):
    """GMRES restarted every 1 or 2 iterations (the memory-lean setting) still reaches the global
    direct solve (FP64 and mixed)."""
    p = W.small_problem(24, 4, 6, seed=130, R=3)
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f)
    for precision in ("fp64", "mixed"):
        s = make_solver(hz, p, precision)
        o = hz.default_opts(precision)
        o.restart = restart
        ug, info, st = s.solve(cuda(f), o)
        ug = ug.cpu().numpy()
        for r in range(p.R):
            assert rel(ug[r], u[r]) < E2E_TOL[precision], (precision, r, rel(ug[r], u[r]))
        s.close()


def test_bicgstab_config2_against_stored_oracle_samples(hz):
    """64^3 smooth random medium, 8 layers, 16 sources, mixed precision with Bi-CGSTAB inside the
    defect correction: stored oracle samples."""
    import os
    d = np.load(os.path.join(os.path.dirname(__file__), "golden", "cfg2_64cube_smooth_samples.npz"))
    p = W.config(2)
    s = make_solver(hz, p, "mixed")
    o = hz.default_opts("mixed")
    o.krylov = 1
    u, info, st = s.solve(cuda(p.rhs()), o)
    uu = u.cpu().numpy().reshape(p.R, -1)
    for r in range(p.R):
        assert rel(uu[r, d["idx"]], d["u"][r]) < E2E_TOL["mixed"], (r, rel(uu[r, d["idx"]], d["u"][r]))
    s.close()


def test_create_takes_the_medium_from_device_memory(hz):
    """hz_create / hz_create_ex accept m (and b) in device memory as well as host memory, with the
    same factors and solution."""
    import ctypes as ct
    p = W.small_problem(16, 3, 2, seed=44, R=2)
    f = cuda(p.rhs())
    ref = make_solver(hz, p, "fp64")
    u_ref = ref.solve(f)[0]
    ref.close()
    lib = hz.load()
    m_dev = torch.from_numpy(np.ascontiguousarray(p.m)).cuda()
    b_dev = torch.ones_like(m_dev)
    g = hz.Grid(p.n, p.n, p.n, 1.0)
    pm = hz.Pml(p.npml, p.C, -1)
    for use_b in (False, True):
        hnd = ct.c_void_p()
        st = lib.hz_create_ex(ct.byref(g), m_dev.data_ptr(), b_dev.data_ptr() if use_b else None, p.omega,
                              ct.byref(pm), p.n_layers, hz.PREC["fp64"], None, ct.byref(hnd))
        assert st == hz.HZ_OK, lib.hz_last_error(None)
        assert lib.hz_factor(hnd) == hz.HZ_OK
        u = torch.empty_like(f)
        assert lib.hz_solve(hnd, f.data_ptr(), p.R, u.data_ptr(), None, None) == hz.HZ_OK
        torch.cuda.synchronize()
        assert float(torch.linalg.vector_norm(u - u_ref) / torch.linalg.vector_norm(u_ref)) < 1e-12
        lib.hz_destroy(hnd)


def test_host_buffer_solve_matches_device_solve(hz):
    """hz_solve_host (host rhs and u; the handle keeps the device copies between calls) gives the
    device path's solution, also on a repeated call and on a later call with more right-hand
    sides (the copies are then replaced), and its solution meets the oracle's, also when it is the
    first call of a fresh handle."""
    p = W.small_problem(16, 3, 2, seed=45, R=3)
    f = p.rhs()
    s = make_solver(hz, p, "mixed")
    u_dev = s.solve(cuda(f))[0].cpu().numpy()
    for R in (2, 2, 3):
        rhs = np.ascontiguousarray(f[:R])
        u = np.zeros_like(rhs)
        out, info, st = s.solve_host(rhs, u=u)
        assert out is u and st == hz.HZ_OK and len(info) == R
        # the same refined solution up to the refinement tolerance (float atomics in the
        # substitution make the rounding order differ from call to call)
        assert rel(u, u_dev[:R]) < 1e-7, (R, rel(u, u_dev[:R]))
    s.close()
    ref = direct.solve(p.m, p.omega, p.npml, p.C, f)
    assert rel(u_dev, ref) < E2E_TOL["mixed"]
    # a host-buffer solve as the first call of a fresh handle: the handle's residual buffers are
    # created inside that call, after its device copies of rhs and u, and must leave them intact
    s = make_solver(hz, p, "mixed")
    u_host, info, st = s.solve_host(f)
    assert st == hz.HZ_OK and rel(u_host, ref) < E2E_TOL["mixed"], rel(u_host, ref)
    u_again, _, st = s.solve_host(f)
    assert st == hz.HZ_OK and rel(u_again, u_host) < 1e-7
    s.close()

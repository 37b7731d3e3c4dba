"""Pins of the oracle's explicit trace-to-trace Green's blocks: the local Green's functions between
the interface plane pairs, i.e. the blocks that Algorithms 4-9 apply matrix-free, written out.

A block E_rs of layer ell maps a trace pair on the layer's interface s (top 't' / bottom 'b')
through that interface's source to the read-out pair at r.  It is pinned by:
* reciprocity: the local operator is complex symmetric, so its Green's function between two
  plane pairs is the transpose of the one the other way; with J_s the source's weights on its two
  planes, E_rs J_s^{-1} = (E_sr J_r^{-1})^T (symmetric for r = s).  A swapped read-out pair, a
  transposed block or a sign slip in the source weights breaks it;
* the matrix-free operators of Algorithms 4-9 (pinned against the global direct solve): the block
  forms of M_pol and of the preconditioner of Eq. 16 give the same vectors;
* GMRES on the trace system with block products meets the global direct solve.
No GPU.
"""
import numpy as np
import pytest

from oracle import direct, polarized
from paper_1801_08655_gb300 import workloads as W


def _J(M, P, sign):
    """Weights of an interface source on its two planes as a (2P x 2P) matrix acting on the pair
    (t(P), t(Q)) flattened as (plane, y, x): plane P receives sign*c t(Q), plane Q receives
    -sign*c t(P) (S_top: sign +1; S_bot: sign -1), c the coupling across the interface."""
    c = M.coupling(P).ravel()
    q = c.size
    J = np.zeros((2 * q, 2 * q), dtype=np.complex128)
    J[np.arange(q), q + np.arange(q)] = sign * c
    J[q + np.arange(q), np.arange(q)] = -sign * c
    return J


@pytest.fixture(scope="module", params=["constant_density", "variable_density"])
def model(request):
    p = W.small_problem(10, 2, 4, seed=61, R=1)
    b = W.density_smooth_random(10, seed=62) if request.param == "variable_density" else None
    M = polarized.PolarizedModel(p.m, p.omega, p.npml, p.C, p.n_layers, b=b)
    return p, b, M, M.trace_blocks()


def test_blocks_present_per_layer(model):
    p, b, M, E = model
    L = M.L
    for ell in range(L):
        want = set()
        for rd in "tb":
            for src in "tb":
                if (rd == "t" or src == "t") and ell == 0:
                    continue
                if (rd == "b" or src == "b") and ell == L - 1:
                    continue
                want.add(rd + src)
        assert set(E[ell]) == want
        for B in E[ell].values():
            assert B.shape == (2 * M.n ** 2, 2 * M.n ** 2)


def test_blocks_are_reciprocal(model):
    p, b, M, E = model
    for ell in range(M.L):
        Jinv = {}
        if ell >= 1:
            Jinv["t"] = np.linalg.inv(_J(M, M.parts[ell - 1][1], +1.0))
        if ell <= M.L - 2:
            Jinv["b"] = np.linalg.inv(_J(M, M.parts[ell][1], -1.0))
        for key, B in E[ell].items():
            r, s = key
            G_rs = B @ Jinv[s]
            G_sr = E[ell][s + r] @ Jinv[r]
            scale = np.abs(G_rs).max()
            assert scale > 0
            assert np.abs(G_rs - G_sr.T).max() <= 1e-10 * scale, (ell, key)


def test_block_operators_match_matrix_free(model):
    p, b, M, E = model
    rng = np.random.default_rng(5)
    shape = M.zeros_trace().shape
    vec = lambda: rng.standard_normal(shape) + 1j * rng.standard_normal(shape)   # noqa: E731
    xd, xu = vec(), vec()
    for got, ref in zip(M.apply_Mpol_blocks(E, xd, xu), M.apply_Mpol(xd, xu)):
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    for got, ref in zip(M.apply_P_blocks(E, xd, xu), M.apply_P(xd, xu)):
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_block_gmres_matches_direct(model):
    p, b, M, E = model
    f = p.rhs()
    u = direct.solve(p.m, p.omega, p.npml, p.C, f, b=b)[0]
    us, its = M.solve(f[0], tol=1e-11, blocks=E)
    assert np.linalg.norm(us - u) / np.linalg.norm(u) < 1e-9
    assert 2 <= its <= 10

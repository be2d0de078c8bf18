"""Pins of the oracle's V-cycle, full multigrid, PCG and L2 error (Algorithms 1-2, Section 4.2)."""

import itertools
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assembly, fe, multigrid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fmg_iterations_paper.txt")


def _paper_counts():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        tok = line.split()
        d, L = int(tok[0]), int(tok[1])
        for k, v in enumerate(tok[2:], start=1):
            if v != "-":
                out[(d, L, k)] = int(v)
    return out


def _vcycle_matrix(H):
    N = H.levels[H.L].N
    B = np.zeros((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        B[:, i] = H.vcycle(H.L, e)
    return B


@pytest.mark.parametrize("d,k,L", [(2, 1, 3), (2, 2, 3), (3, 2, 2)])
def test_symmetric_vcycle_is_spd_and_contracting(d, k, L):
    """Reverse-order post-smoothing makes B symmetric positive definite with eig(BA) in (0, 1]."""
    H = multigrid.Hierarchy(d, k, L, symmetric=True)
    B = _vcycle_matrix(H)
    A = H.A[L].toarray()
    assert np.abs(B - B.T).max() <= 1e-13 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    ev = np.linalg.eigvals(B @ A).real
    assert ev.min() > 0.5 and ev.max() < 1 + 1e-10


def test_forward_forward_vcycle_is_not_symmetric():
    H = multigrid.Hierarchy(2, 2, 3, symmetric=False)
    B = _vcycle_matrix(H)
    assert np.abs(B - B.T).max() > 1e-6 * np.abs(B).max()


@pytest.mark.parametrize("d,k", [(2, 1), (2, 2), (2, 3), (2, 4), (2, 5), (2, 6), (2, 7)])
def test_fmg_iteration_counts_against_paper_2d(d, k):
    """Algorithm 2 with f = 1 at L = 4 in 2D: never more V-cycles than Table 1
    prints, and at most 3 for k >= 3 (Section 2.2).  One-sided: Algorithm 2
    as printed converges in fewer cycles than Table 1 in 2D (no reading of the
    algorithm tried reproduces Table 1 and Table 2 together)."""
    paper = _paper_counts()[(d, 4, k)]
    it = multigrid.fmg_iterations(d, k, 4, lambda X: np.ones(len(X)))
    assert 1 <= it <= paper
    if k >= 3:
        assert it <= 3


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_fmg_iteration_counts_against_paper_3d(k):
    """Algorithm 2 with f = 1 at L = 4 in 3D: within one V-cycle of Table 2
    (6, 5, 3, 3 for k = 1..4), both ways."""
    paper = _paper_counts()[(3, 4, k)]
    it = multigrid.fmg_iterations(3, k, 4, lambda X: np.ones(len(X)))
    assert abs(it - paper) <= 1


def _patch_sets(d, k, l):
    """Compact interior DoF sets of the vertex patches, written from their
    definition (the nodes strictly inside the 2^d cells around an interior
    vertex v, v_t in 1..2^l - 1), grouped by the colour of Section 2.2
    (vertex parity per direction)."""
    ni = k * 2 ** l - 1
    sets = {c: [] for c in range(2 ** d)}
    for v in itertools.product(range(1, 2 ** l), repeat=d):
        axes = [np.arange(k * (vt - 1) + 1, k * (vt + 1)) for vt in v]
        grids = np.meshgrid(*axes, indexing="ij")
        idx = sum((grids[t] - 1) * ni ** t for t in range(d)).ravel()
        colour = sum(((v[t] - 1) % 2) << t for t in range(d))
        sets[colour].append(idx)
    return sets


def _smoothing_propagator(A, sets, order):
    """Error propagation of one multiplicative step: the colours in `order`,
    each I - sum_j R_j^T A_j^-1 R_j A (patches of one colour do not couple)."""
    N = A.shape[0]
    S = np.eye(N)
    for c in order:
        M = np.eye(N)
        for I in sets[c]:
            Aj = A[np.ix_(I, I)]
            M[I, :] -= np.linalg.solve(Aj, A[I, :])
        S = M @ S
    return S


@pytest.mark.parametrize("d,k,L,sym", [(2, 2, 3, True), (2, 2, 3, False), (2, 1, 4, True),
                                       (3, 1, 3, True), (3, 2, 2, False)])
def test_vcycle_equals_product_of_error_propagators(d, k, L, sym):
    """Algorithm 1 as an operator: E_l = S_post (I - P_l B_{l-1} P_l^T A_l) S_pre,
    B_1 = A_1^-1, B_l = (I - E_l) A_l^-1, with S the one-step multiplicative
    smoother (colours forward before, reverse or forward after) built from
    dense patch matrices; the oracle's V-cycle applied to unit vectors gives
    the columns of B_L.  Catches a cycle that smooths more or less than one
    step before and after, in another colour order, or corrects wrongly."""
    H = multigrid.Hierarchy(d, k, L, symmetric=sym)
    nc = 2 ** d
    B = None
    for l in range(1, L + 1):
        A = H.A[l].toarray()
        if l == 1:
            B = np.linalg.inv(A)
            continue
        sets = _patch_sets(d, k, l)
        Spre = _smoothing_propagator(A, sets, range(nc))
        Spost = _smoothing_propagator(A, sets, range(nc - 1, -1, -1) if sym else range(nc))
        P = H.P[l].toarray()
        E = Spost @ (np.eye(len(A)) - P @ B @ P.T @ A) @ Spre
        B = (np.eye(len(A)) - E) @ np.linalg.inv(A)
    Bo = _vcycle_matrix(H)
    assert np.abs(Bo - B).max() <= 1e-11 * np.abs(B).max()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_fmg_iterations_independent_of_level(k):
    """Section 2.2: the count is independent of the mesh level (2D, L = 3..6), up to
    one step for the lowest order, which the paper says saturates more slowly."""
    its = [multigrid.fmg_iterations(2, k, L, lambda X: np.ones(len(X))) for L in (3, 4, 5, 6)]
    assert max(its) - min(its) <= 1
    if k >= 2:
        assert its[-1] <= its[0]


@pytest.mark.parametrize("d,k,L,sm,om", [(2, 2, 4, "multiplicative", 1.0), (2, 3, 3, "additive", 0.35),
                                         (3, 2, 3, "multiplicative", 1.0), (3, 1, 3, "additive", 0.175)])
def test_pcg_converges_to_direct_solution(d, k, L, sm, om):
    H = multigrid.Hierarchy(d, k, L, smoother=sm, omega=om)
    b = np.random.default_rng(5).uniform(-1, 1, H.levels[L].N)
    x, it, rel = multigrid.pcg(H.A[L], b, H.precondition, rtol=1e-10, max_it=60)
    assert rel <= 1e-10 and it < 30
    xd = spla.spsolve(H.A[L].tocsc(), b)
    assert np.abs(x - xd).max() <= 1e-8 * np.abs(xd).max()


def test_pcg_breaks_down_or_stalls_with_literal_additive_damping_in_3d():
    """omega = 0.7 with lambda_max(sum P_j) = 8 makes the 3D additive V-cycle indefinite."""
    H = multigrid.Hierarchy(3, 2, 3, smoother="additive", omega=0.7)
    b = np.random.default_rng(6).uniform(-1, 1, H.levels[3].N)
    try:
        _, it, rel = multigrid.pcg(H.A[3], b, H.precondition, rtol=1e-10, max_it=40)
    except FloatingPointError:
        return
    assert rel > 1e-10


@pytest.mark.parametrize("d,k,L", [(2, 2, 3), (3, 2, 2)])
def test_pcg_recovers_polynomial_solution_in_Vh(d, k, L):
    H = multigrid.Hierarchy(d, k, L)
    lv = H.levels[L]
    u = lambda X: np.prod(X * (1 - X), axis=1)

    def f(X):
        s = np.zeros(len(X))
        for t in range(d):
            s += 2 * np.prod(np.delete(X * (1 - X), t, axis=1), axis=1)
        return s
    x, it, rel = multigrid.pcg(H.A[L], assembly.load_vector(lv, f), H.precondition, rtol=1e-12)
    np.testing.assert_allclose(x, assembly.interpolate(lv, u), atol=1e-11)
    assert multigrid.l2_error(lv, x, u) < 1e-12


@pytest.mark.parametrize("d,k,levels", [(2, 1, (3, 4, 5)), (2, 2, (2, 3, 4)), (2, 3, (2, 3)), (3, 1, (2, 3))])
def test_l2_error_converges_with_order_k_plus_1(d, k, levels):
    """u = prod sin(pi x_t), f = d pi^2 u: ||u_h - u|| = O(h^(k+1)) (Section 4.2 test problem)."""
    u = lambda X: np.prod(np.sin(np.pi * X), axis=1)
    f = lambda X: d * np.pi ** 2 * u(X)
    errs = []
    for L in levels:
        lv = fe.Level(d, k, L)
        A = assembly.stiffness(lv)
        x = spla.spsolve(A.tocsc(), assembly.load_vector(lv, f))
        errs.append(multigrid.l2_error(lv, x, u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - (k + 1)) < 0.25), rates


def test_l2_error_of_exact_interpolant_of_constant_zero():
    lv = fe.Level(2, 2, 2)
    assert multigrid.l2_error(lv, np.zeros(lv.N), lambda X: np.zeros(len(X))) == 0.0
    # ||1||_{L2} over the unit square, with u_h = 0: exactly 1
    assert abs(multigrid.l2_error(lv, np.zeros(lv.N), lambda X: np.ones(len(X))) - 1.0) < 1e-14


def _krylov_min_residual(A, b, B, k):
    """min ||b - A Z y|| over span{B r0, B A B r0, ...} (k vectors), brute force."""
    Z = []
    v = b.copy()
    for _ in range(k):
        z = B @ v
        Z.append(z)
        v = A @ z
    Z = np.array(Z).T
    Q, _ = np.linalg.qr(A @ Z)
    return np.linalg.norm(b - Q @ (Q.T @ b))


@pytest.mark.parametrize("pre", ["none", "jacobi", "vcycle"])
def test_fgmres_is_the_minimal_residual_method(pre):
    """With a fixed linear preconditioner B, FGMRES after k steps attains the
    minimal residual over b + A span{B r0, (B A) B r0, ...}: the Krylov space of
    A B, mapped by B (brute-force least squares on a small problem)."""
    H = multigrid.Hierarchy(2, 2, 3, symmetric=False)
    A = H.A[3].toarray()
    n = A.shape[0]
    b = np.random.default_rng(21).normal(size=n)
    if pre == "none":
        B = np.eye(n)
    elif pre == "jacobi":
        B = np.diag(1.0 / np.diag(A))
    else:  # the V-cycle as a matrix (it is linear in its right-hand side)
        B = np.column_stack([H.vcycle(3, e) for e in np.eye(n)])
    _, it, rel, hist = multigrid.fgmres(A, b, lambda v: B @ v, rtol=1e-14, restart=200, max_it=8)
    nb = np.linalg.norm(b)
    checked = 0
    for k in range(1, len(hist) + 1):
        ref = _krylov_min_residual(A, b, B, k) / nb
        if ref < 1e-10:  # both at round-off (the monomial basis is ill-conditioned)
            break
        assert abs(hist[k - 1] - ref) <= 1e-8 * ref, (k, hist[k - 1], ref)
        checked += 1
    assert checked >= 3


def test_fgmres_finite_termination_and_restart():
    """Without restarts GMRES solves an n x n system in at most n steps; with
    restarts the least-squares estimate agrees with the true residual."""
    rng = np.random.default_rng(22)
    n = 12
    M = rng.normal(size=(n, n)) + n * np.eye(n)
    b = rng.normal(size=n)
    x, it, rel, _ = multigrid.fgmres(M, b, lambda v: v, rtol=1e-13, restart=n, max_it=n)
    assert it <= n and np.linalg.norm(b - M @ x) <= 1e-11 * np.linalg.norm(b)
    x, it, rel, hist = multigrid.fgmres(M, b, lambda v: v, rtol=1e-10, restart=3, max_it=200)
    assert rel <= 1e-10 and np.isclose(rel, np.linalg.norm(b - M @ x) / np.linalg.norm(b))
    assert np.all(np.diff(hist[:3]) <= 1e-15)  # monotone within a cycle


def test_fgmres_with_vcycle_solves_the_poisson_problem():
    H = multigrid.Hierarchy(3, 2, 3, symmetric=False)
    b = np.random.default_rng(23).uniform(-1, 1, H.levels[3].N)
    x, it, rel, _ = multigrid.fgmres(H.A[3], b, H.precondition, rtol=1e-9)
    assert rel <= 1e-9 and it <= 12
    import scipy.sparse.linalg as spla
    xd = spla.spsolve(H.A[3].tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)

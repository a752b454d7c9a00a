"""Pins for the oracle's CGLS and LSQR inner solvers and IRN outer loop (CPU only).

The inner problem is the augmented least-squares system of Sec. 2.3
[A; alpha W1 D; lambda W2 D] x ~ [b; 0; lambda W2 D x_p], solved by CGLS or
by LSQR (mathematically equivalent, Sec. 2.3).  These tests build the
same system densely from independently pinned pieces (A column by column, D
from Kronecker products) and compare with numpy/scipy solvers; the IRN loop is
pinned by the majorisation-minimisation decrease of the smoothed objective.
"""
import numpy as np
import pytest
from scipy.sparse.linalg import lsqr

import oracle as O
import phantoms as P


def _D1_padded(n):
    D1 = np.zeros((n, n))
    for i in range(n - 1):
        D1[i, i], D1[i, i + 1] = 1.0, -1.0
    return D1


def _kron_D(nx, ny, nz):
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    return np.vstack([np.kron(np.kron(_D1_padded(nx), Iy), Iz),
                      np.kron(np.kron(Ix, _D1_padded(ny)), Iz),
                      np.kron(np.kron(Ix, Iy), _D1_padded(nz))])


def _dense_A(g):
    cols = []
    for j in range(g.M):
        e = np.zeros(g.M)
        e[j] = 1.0
        cols.append(O.forward(g, e.reshape(g.vol_shape())).reshape(-1))
    return np.stack(cols, 1)


@pytest.fixture(scope="module")
def small():
    g = P.tiny_geometry(n=(6, 6, 5), det=(10, 8), n_views=12, dso=40.0, dsd=60.0)
    A = _dense_A(g)
    D = _kron_D(g.nx, g.ny, g.nz)
    rng = np.random.default_rng(7)
    x_true = np.zeros(g.vol_shape())
    x_true[1:5, 2:5, 1:4] = 1.0
    x_true += 0.05 * rng.normal(size=g.vol_shape())
    b = A @ x_true.reshape(-1) + 0.01 * rng.normal(size=g.N)
    xp = x_true.copy()
    xp[2:4, 2:4, 2:3] += 0.4  # prior differs locally
    w1 = rng.uniform(0.5, 2.0, size=g.M)
    w2 = rng.uniform(0.5, 2.0, size=g.M)
    return dict(g=g, A=A, D=D, b=b, xp=xp.reshape(-1), x_true=x_true, w1=w1, w2=w2)


def _dense_aug(s, variant, alpha, lam):
    A, D, b, xp, w1, w2 = s["A"], s["D"], s["b"], s["xp"], s["w1"], s["w2"]
    M = A.shape[1]
    W1 = np.diag(np.tile(w1, 3))
    W2 = np.diag(np.tile(w2, 3))
    if variant == O.CGLS:
        return A, b
    rows = [A, alpha * W1 @ D]
    rhs = [b, np.zeros(3 * M)]
    if variant == O.PICCS:
        rows.append(lam * W2 @ D)
        rhs.append(lam * W2 @ D @ xp)
    elif variant == O.PIPLE:
        rows.append(lam * np.eye(M))
        rhs.append(lam * xp)
    return np.vstack(rows), np.concatenate(rhs)


@pytest.mark.parametrize("variant", [O.PICCS, O.PIPLE, O.TV])
def test_converged_cgls_solves_normal_equations(small, variant):
    g = small["g"]
    At, bt = _dense_aug(small, variant, 0.7, 0.4)
    x_ref = np.linalg.solve(At.T @ At, At.T @ bt)
    x, res = O.cgls_fixed(g, small["b"], small["xp"], small["w1"], small["w2"], 0.7, 0.4,
                          variant, np.zeros(g.M), 400)
    np.testing.assert_allclose(x.reshape(-1), x_ref, rtol=0, atol=1e-8 * np.abs(x_ref).max())


def test_unregularised_cgls_is_least_squares(small):
    g = small["g"]
    A, b = small["A"], small["b"]
    x_ref = np.linalg.lstsq(A, b, rcond=None)[0]
    x, _ = O.cgls_fixed(g, b, small["xp"], small["w1"], small["w2"], 0.0, 0.0, O.CGLS,
                        np.zeros(g.M), 3000)
    np.testing.assert_allclose(x.reshape(-1), x_ref, rtol=0, atol=1e-6 * np.abs(x_ref).max())


def _krylov_minimiser(At, bt, x0, k):
    """x_0 + argmin over K_k(At^T At, At^T r_0) of ||At x - bt||, from an
    orthonormal basis of the Krylov space and a dense least-squares solve."""
    r0 = bt - At @ x0
    AtA = At.T @ At
    v = At.T @ r0
    basis = []
    for _ in range(k):
        for q in basis:  # Gram-Schmidt twice
            v = v - (q @ v) * q
        for q in basis:
            v = v - (q @ v) * q
        v = v / np.linalg.norm(v)
        basis.append(v)
        v = AtA @ v
    K = np.stack(basis, 1)
    z = np.linalg.lstsq(At @ K, r0, rcond=None)[0]
    return x0 + K @ z


@pytest.mark.parametrize("variant", [O.PICCS, O.PIPLE])
@pytest.mark.parametrize("k", [1, 2, 5, 8])
def test_iterate_k_is_krylov_subspace_minimiser(small, variant, k):
    """x_k = x_0 + argmin over K_k(At^T At, At^T r_0) of ||At x - bt||."""
    g = small["g"]
    At, bt = _dense_aug(small, variant, 0.5, 0.6)
    x0 = small["xp"].copy()
    x_ref = _krylov_minimiser(At, bt, x0, k)
    x, _ = O.cgls_fixed(g, small["b"], small["xp"], small["w1"], small["w2"], 0.5, 0.6,
                        variant, x0, k)
    np.testing.assert_allclose(x.reshape(-1), x_ref, rtol=0, atol=1e-9 * np.abs(x_ref).max())


@pytest.mark.parametrize("reorth", [False, True])
@pytest.mark.parametrize("variant", [O.PICCS, O.PIPLE, O.TV, O.CGLS])
@pytest.mark.parametrize("k", [1, 3, 10])
def test_oracle_lsqr_matches_scipy_lsqr(small, variant, k, reorth):
    """The oracle's LSQR against scipy's (Paige-Saunders) on the dense system."""
    g = small["g"]
    At, bt = _dense_aug(small, variant, 0.6, 0.45)
    x0 = small["xp"].copy()
    x_ref = lsqr(At, bt, x0=x0, iter_lim=k, atol=0, btol=0, conlim=0)[0]
    x, res = O.lsqr_fixed(g, small["b"], small["xp"], small["w1"], small["w2"], 0.6, 0.45,
                          variant, x0, k, reorth=reorth)
    assert len(res) == k + 1
    np.testing.assert_allclose(x.reshape(-1), x_ref, rtol=0, atol=1e-9 * np.abs(x_ref).max())
    np.testing.assert_allclose(res, [np.sum((bt - At @ x0) ** 2)] + list(res[1:]))
    assert abs(res[-1] - np.sum((bt - At @ x_ref) ** 2)) <= 1e-9 * res[0]


@pytest.mark.parametrize("variant", [O.PICCS, O.PIPLE])
@pytest.mark.parametrize("k", [2, 5, 8])
def test_lsqr_iterate_is_krylov_subspace_minimiser(small, variant, k):
    g = small["g"]
    At, bt = _dense_aug(small, variant, 0.5, 0.6)
    x0 = np.zeros(g.M)
    x_ref = _krylov_minimiser(At, bt, x0, k)
    for reorth in (False, True):
        x, _ = O.lsqr_fixed(g, small["b"], small["xp"], small["w1"], small["w2"], 0.5, 0.6,
                            variant, x0, k, reorth=reorth)
        np.testing.assert_allclose(x.reshape(-1), x_ref, rtol=0,
                                   atol=1e-9 * np.abs(x_ref).max())


def test_converged_lsqr_with_reorthogonalisation_solves_normal_equations(small):
    """With full re-orthogonalisation the bidiagonalisation terminates in at
    most M steps in exact arithmetic; the stop rule must then end the loop
    early, at the least-squares solution."""
    g = small["g"]
    At, bt = _dense_aug(small, O.PICCS, 0.7, 0.4)
    x_ref = np.linalg.solve(At.T @ At, At.T @ bt)
    x, res = O.lsqr_fixed(g, small["b"], small["xp"], small["w1"], small["w2"], 0.7, 0.4,
                          O.PICCS, np.zeros(g.M), 4 * g.M, reorth=True)
    assert len(res) - 1 < 4 * g.M
    np.testing.assert_allclose(x.reshape(-1), x_ref, rtol=0, atol=1e-8 * np.abs(x_ref).max())
    assert np.all(np.diff(res) <= 1e-12 * res[0])


@pytest.mark.parametrize("solver", [O.SOLVER_LSQR, O.SOLVER_LSQR_REORTH])
def test_irn_with_lsqr_equals_irn_with_cgls(small, solver):
    g = small["g"]
    a, ra, _ = O.irn(g, small["b"], small["xp"], small["xp"], 0.5, 0.5, 0.05, 3, 5)
    b, rb, _ = O.irn(g, small["b"], small["xp"], small["xp"], 0.5, 0.5, 0.05, 3, 5,
                     solver=solver)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-9 * np.abs(a).max())
    np.testing.assert_allclose(rb, ra, rtol=1e-8)


@pytest.mark.parametrize("k", [3, 10])
def test_cgls_matches_lsqr(small, k):
    """CGLS and LSQR produce the same iterates in exact arithmetic (Sec. 2.3)."""
    g = small["g"]
    At, bt = _dense_aug(small, O.PICCS, 0.5, 0.5)
    x0 = small["xp"].copy()
    x_lsqr = lsqr(At, bt, x0=x0, iter_lim=k, atol=0, btol=0, conlim=0)[0]
    x, _ = O.cgls_fixed(g, small["b"], small["xp"], small["w1"], small["w2"], 0.5, 0.5,
                        O.PICCS, x0, k)
    np.testing.assert_allclose(x.reshape(-1), x_lsqr, rtol=0, atol=1e-8 * np.abs(x_lsqr).max())


def test_residual_decreases_within_each_cycle(small):
    g = small["g"]
    _, res, _ = O.irn(g, small["b"], small["xp"], small["xp"], 0.5, 0.5, 0.05, 4, 6)
    assert np.all(np.isfinite(res))
    assert np.all(np.diff(res, axis=1) <= 1e-12 * res[:, :1])


def _phi_r1(t, tau):
    return t - tau ** 2 * np.log1p(t / tau ** 2)


def _phi_r2(t, tau):
    return np.sqrt(t ** 2 + tau ** 2)


def _J(s, x, alpha, lam, tau, phi, variant):
    """Smoothed objective whose tangent majorant the IRN term is: data misfit
    plus 2 alpha^2 sum phi(|(Dx)_i|) plus the prior term."""
    A, D, b, xp = s["A"], s["D"], s["b"], s["xp"]
    M = A.shape[1]
    x = x.reshape(-1)
    gx = (D @ x).reshape(3, M)
    J = np.sum((A @ x - b) ** 2) + 2 * alpha ** 2 * phi(np.sqrt((gx ** 2).sum(0)), tau).sum()
    if variant == O.PICCS:
        gd = (D @ (x - xp)).reshape(3, M)
        J += 2 * lam ** 2 * phi(np.sqrt((gd ** 2).sum(0)), tau).sum()
    elif variant == O.PIPLE:
        J += lam ** 2 * np.sum((x - xp) ** 2)
    return J


@pytest.mark.parametrize("rule,phi", [(O.RULE_R1, _phi_r1), (O.RULE_R2, _phi_r2)])
@pytest.mark.parametrize("variant", [O.PICCS, O.PIPLE, O.TV])
def test_irn_decreases_smoothed_objective(small, rule, phi, variant):
    g = small["g"]
    alpha, lam, tau = 0.4, 0.6, 0.05
    Js = [_J(small, small["xp"], alpha, lam, tau, phi, variant)]
    for n_outer in range(1, 6):
        x, _, _ = O.irn(g, small["b"], small["xp"], small["xp"], alpha, lam, tau, n_outer, 4,
                        variant=variant, rule=rule)
        Js.append(_J(small, x, alpha, lam, tau, phi, variant))
    Js = np.array(Js)
    assert np.all(np.diff(Js) <= 1e-12 * Js[0]), Js
    assert Js[-1] < 0.999 * Js[0]


def test_irn_weights_follow_previous_iterate(small):
    """The returned last-cycle weights are W(D x_{K-1}) and W(D x_{K-1} - D x_p)."""
    g = small["g"]
    x_prev, _, _ = O.irn(g, small["b"], small["xp"], small["xp"], 0.5, 0.5, 0.05, 2, 3)
    _, _, (w1, w2) = O.irn(g, small["b"], small["xp"], small["xp"], 0.5, 0.5, 0.05, 3, 3)
    D = small["D"]
    M = g.M
    n1 = np.sqrt(((D @ x_prev.reshape(-1)).reshape(3, M) ** 2).sum(0))
    n2 = np.sqrt(((D @ (x_prev.reshape(-1) - small["xp"])).reshape(3, M) ** 2).sum(0))
    np.testing.assert_allclose(w1.reshape(-1) ** -2 - 0.05 ** 2, n1, atol=1e-10)
    np.testing.assert_allclose(w2.reshape(-1) ** -2 - 0.05 ** 2, n2, atol=1e-10)


def test_piccs_with_zero_lambda_is_tv(small):
    g = small["g"]
    a, _, _ = O.irn(g, small["b"], small["xp"], small["xp"], 0.5, 0.0, 0.05, 3, 4,
                    variant=O.PICCS)
    b, _, _ = O.irn(g, small["b"], small["xp"], small["xp"], 0.5, 0.0, 0.05, 3, 4,
                    variant=O.TV)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_cgls_variant_ignores_regularisation(small):
    g = small["g"]
    a, _, _ = O.irn(g, small["b"], small["xp"], np.zeros(g.M), 0.9, 0.9, 0.05, 1, 6,
                    variant=O.CGLS)
    b, _ = O.cgls_fixed(g, small["b"], small["xp"], small["w1"], small["w2"], 0.0, 0.0,
                        O.CGLS, np.zeros(g.M), 6)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_lsqr_reorthogonalisation_keeps_the_basis_orthonormal():
    """Golub-Kahan in floating point loses the orthogonality of V within a few
    tens of steps on this system; re-orthogonalised, V stays orthonormal to
    rounding, and the bidiagonal relation A~^T u_{k+1} = alpha_{k+1} v_{k+1}
    + beta_{k+1} v_k keeps consecutive v's tied to the operator."""
    g = P.tiny_geometry(n=(6, 6, 5), det=(10, 8), n_views=12, dso=40.0, dsd=60.0)
    rng = np.random.default_rng(7)
    b = rng.normal(size=g.N)
    xp = rng.normal(size=g.M)
    w1 = rng.uniform(0.5, 2.0, g.M)
    w2 = rng.uniform(0.5, 2.0, g.M)
    k = 30
    _, _, V = O.lsqr_fixed(g, b, xp, w1, w2, 0.3, 0.2, O.PICCS, np.zeros(g.M), k,
                           reorth=True, return_basis=True)
    assert V.shape == (k + 1, g.M)
    assert np.abs(V @ V.T - np.eye(k + 1)).max() < 1e-12
    _, _, V0 = O.lsqr_fixed(g, b, xp, w1, w2, 0.3, 0.2, O.PICCS, np.zeros(g.M), k,
                            reorth=False, return_basis=True)
    assert np.abs(V0 @ V0.T - np.eye(k + 1)).max() > 1e-3
    # the first vectors agree while the plain recurrence is still orthogonal
    np.testing.assert_allclose(V0[:6], V[:6], rtol=0, atol=1e-9)

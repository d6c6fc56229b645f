"""The host-side tridiagonal eigensolver of the eigenpair call (implicit
symmetric QR with Wilkinson shifts), through the C ABI. Host code only: no GPU.

Pins: the closed form of the tridiagonal Toeplitz matrix (eigenvalues
a + 2 b cos(q pi / (k + 1)), eigenvectors sin(j q pi / (k + 1))), a diagonal
matrix, scipy's LAPACK tridiagonal solver, T Z = Z Theta and Z^T Z = I on
random and on Lanczos matrices of a spectrum with a 50-fold eigenvalue."""
import numpy as np
import pytest

from paper_2305_16086_gb300 import binding


def _T(a, e):
    return np.diag(a) + np.diag(e, 1) + np.diag(e, -1)


@pytest.mark.parametrize("k", [1, 2, 5, 64, 301])
def test_toeplitz_closed_form(k):
    a, b = 0.25, -0.5
    theta, Z = binding.tridiag_eig(np.full(k, a), np.full(k - 1, b))
    q = np.arange(1, k + 1)
    want = np.sort(a + 2 * b * np.cos(q * np.pi / (k + 1)))
    assert np.max(np.abs(theta - want)) < 1e-14 * max(k, 8)
    j = np.arange(1, k + 1)
    for col in range(k):
        # the eigenvector of a + 2 b cos(qq pi / (k + 1)) is sin(j qq pi / (k + 1)), up to sign
        qq = np.argmin(np.abs(a + 2 * b * np.cos(q * np.pi / (k + 1)) - theta[col])) + 1
        v = np.sin(j * qq * np.pi / (k + 1))
        v /= np.linalg.norm(v)
        assert abs(abs(v @ Z[:, col]) - 1.0) < 1e-12


def test_diagonal_matrix_is_sorted_with_unit_vectors():
    a = np.array([3.0, -1.0, 2.0, 0.5])
    theta, Z = binding.tridiag_eig(a, np.zeros(3))
    assert np.array_equal(theta, np.sort(a))
    assert np.array_equal(np.abs(Z), np.eye(4)[:, np.argsort(a)])


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("k", [3, 40, 200])
def test_random_against_lapack(seed, k):
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(seed)
    a, e = rng.standard_normal(k), rng.standard_normal(k - 1)
    theta, Z = binding.tridiag_eig(a, e)
    ref = sl.eigh_tridiagonal(a, e, eigvals_only=True)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(theta - ref)) < 1e-14 * k * scale
    assert np.max(np.abs(_T(a, e) @ Z - Z * theta)) < 1e-14 * k * scale
    assert np.max(np.abs(Z.T @ Z - np.eye(k))) < 1e-13 * k


def test_lanczos_matrix_of_a_repeated_eigenvalue():
    """Lanczos (full reorthogonalisation) on a spectrum with 0.3 fifty times,
    run until the Krylov space is exhausted (351 distinct eigenvalues): T holds
    every distinct eigenvalue once, 0.3 included."""
    rng = np.random.default_rng(3)
    n, steps = 400, 351
    ev = np.concatenate([np.full(50, 0.3), np.linspace(-0.6, 0.95, n - 50)])
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * ev) @ Q.T
    V = [rng.standard_normal(n)]
    V[0] /= np.linalg.norm(V[0])
    alpha, beta = [], []
    for j in range(steps):
        w = A @ V[-1]
        M = np.array(V)
        for _ in range(2):
            w -= M.T @ (M @ w)
        alpha.append(V[-1] @ A @ V[-1])
        b = np.linalg.norm(w)
        if j + 1 < steps:
            beta.append(b)
            V.append(w / b)
    a, e = np.array(alpha), np.array(beta)
    theta, Z = binding.tridiag_eig(a, e)
    assert np.max(np.abs(_T(a, e) @ Z - Z * theta)) < 1e-13
    assert np.max(np.abs(Z.T @ Z - np.eye(steps))) < 1e-12
    assert np.sum(np.abs(theta - 0.3) < 1e-10) == 1  # one vector of the 50-dimensional eigenspace
    distinct = np.unique(ev)
    assert np.max(np.abs(theta - distinct)) < 1e-10

"""Pins of the oracle's F-space projection of the SNH element Hessian
(H = V B^T proj(d2psi/dF2) B: §5.2's eigenvalue clamp taken on the 9x9
material Hessian).

Fixed by: the PSD property of the result; H_F - H being PSD (the clamp only
adds the negative part back); equality with the plain Hessian at rest (the
material Hessian is PSD there); rotation invariance; and the spectrum of
d2psi/dF2 against its closed form in the frame of the signed SVD of F
(numpy's SVD and eigh as library routines): three pairs of twist/flip
eigenvalues a -+ b sigma_k and the eigenvalues of a 3x3 stretch block.
"""
import numpy as np
import pytest

from oracle import oracle as orc

MU, LAM = 3.0e4, 8.0e4   # mu', lambda'


def _tet(seed, jitter=0.2):
    rng = np.random.default_rng(seed)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    X += rng.uniform(-jitter, jitter, X.shape)
    if np.linalg.det((X[1:] - X[0]).T) < 0:
        X = X[[0, 2, 1, 3]]
    return X


def _elem(X):
    Dminv, V, bad = orc.tet_rest(X, np.array([[0, 1, 2, 3]], np.int32))
    assert bad == 0
    return Dminv[0], V[0]


def _deformed(X, seed, amp):
    return X + np.random.default_rng(100 + seed).uniform(-amp, amp, X.shape)


def _psd_tol(A):
    return -1e-12 * np.abs(np.linalg.eigvalsh(A)).max()


@pytest.mark.parametrize("seed", range(6))
def test_fproj_is_psd_and_dominates_the_plain_hessian(seed):
    X = _tet(seed)
    x = _deformed(X, seed, 0.3)
    Dminv, V = _elem(X)
    E0, g0, H0 = orc.snh_element(x.ravel(), Dminv, V, MU, LAM)
    E1, g1, H1 = orc.snh_element_fproj(x.ravel(), Dminv, V, MU, LAM)
    assert E1 == E0 and np.array_equal(g1, g0)
    assert np.allclose(H1, H1.T, rtol=0, atol=1e-12 * np.abs(H1).max())
    assert np.linalg.eigvalsh(H1).min() >= _psd_tol(H1)
    assert np.linalg.eigvalsh(H1 - H0).min() >= _psd_tol(H1)


def test_fproj_equals_plain_hessian_at_rest():
    X = _tet(3)
    Dminv, V = _elem(X)
    A = orc.snh_dPdF(X.ravel(), Dminv, MU, LAM)
    assert np.linalg.eigvalsh(A).min() >= -1e-9 * np.abs(A).max()
    _, _, H0 = orc.snh_element(X.ravel(), Dminv, V, MU, LAM)
    _, _, H1 = orc.snh_element_fproj(X.ravel(), Dminv, V, MU, LAM)
    assert np.abs(H1 - H0).max() <= 1e-9 * np.abs(H0).max()


@pytest.mark.parametrize("seed", range(3))
def test_fproj_rotation_invariance(seed):
    X = _tet(seed)
    x = _deformed(X, seed, 0.3)
    Dminv, V = _elem(X)
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    R = np.kron(np.eye(4), q)
    _, _, H = orc.snh_element_fproj(x.ravel(), Dminv, V, MU, LAM)
    _, _, Hr = orc.snh_element_fproj((x @ q.T).ravel(), Dminv, V, MU, LAM)
    assert np.abs(Hr - R @ H @ R.T).max() <= 1e-9 * np.abs(H).max()


@pytest.mark.parametrize("seed,amp", [(0, 0.1), (1, 0.3), (2, 0.5), (3, 0.7), (4, 0.9)])
def test_material_hessian_spectrum_closed_form(seed, amp):
    X = _tet(seed)
    x = _deformed(X, seed, amp)
    Dminv, V = _elem(X)
    A = orc.snh_dPdF(x.ravel(), Dminv, MU, LAM)
    F = (x[1:] - x[0]).T @ np.linalg.inv((X[1:] - X[0]).T)
    U, s, Vh = np.linalg.svd(F)
    s = s.copy()
    if np.linalg.det(U) < 0:
        U[:, 2] *= -1
        s[2] *= -1
    if np.linalg.det(Vh) < 0:
        s[2] *= -1
    Ic = (F * F).sum()
    J = np.linalg.det(F)
    alpha = 1.0 + 0.75 * MU / LAM
    a = MU * (1.0 - 1.0 / (Ic + 1.0))
    gam = 2.0 * MU / (Ic + 1.0) ** 2
    b = LAM * (J - alpha)
    pairs = []
    for k in range(3):
        pairs += [a - b * s[k], a + b * s[k]]
    pi = np.array([s[1] * s[2], s[0] * s[2], s[0] * s[1]])
    K = np.array([[0, s[2], s[1]], [s[2], 0, s[0]], [s[1], s[0], 0]])
    A3 = a * np.eye(3) + gam * np.outer(s, s) + LAM * np.outer(pi, pi) + b * K
    closed = np.sort(np.concatenate([pairs, np.linalg.eigvalsh(A3)]))
    assert np.abs(np.sort(np.linalg.eigvalsh(A)) - closed).max() <= 1e-10 * np.abs(closed).max()

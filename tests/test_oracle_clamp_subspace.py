"""The accuracy argument the GPU projection rests on (§5.2 "Projection to
positive semi-definiteness"; the clamp-accuracy reading), checked with numpy
and the oracle's cyclic-Jacobi clamp, independently of the CUDA path.

In the orthonormal Hadamard basis of the four nodes an element Hessian H
becomes diag(0_3, M). If V (9 x k, orthonormal) spans the subspace of M's
eigenvalues below some level and the rest of M has no eigenvalue below -s,
then the clamp of M is M - V B_- V^T with B = V^T M V and B_- its part below
zero, up to s; and for a V that spans it only approximately, the result is
within 2 sqrt(2) ||M V - V B||_F of the clamp (clamping is 1-Lipschitz in the
Frobenius norm). The CUDA refinement (k <= 3 lowest modes) and deflation
(the clearly negative modes of a stencil with a null space) rely on both.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes

HD = 0.5 * np.array([[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]], float)
P = np.kron(HD, np.eye(3))


def _m9(H):
    return (P.T @ H @ P)[3:, 3:]


def _h12(M):
    Z = np.zeros((12, 12))
    Z[3:, 3:] = M
    return P @ Z @ P.T


def _neg_part(B):
    w, G = np.linalg.eigh(B)
    return (G * np.minimum(w, 0.0)) @ G.T


@pytest.fixture(scope="module")
def snh_hessians():
    m = scenes.kuhn_box(8, 7, 6, h=0.25, seed=3)
    T = m["tets"].shape[0]
    E, nu = scenes.material_random(T, seed=3)
    x = scenes.jitter_state(m["X"], 0.02 * 0.25, seed=4)
    snh, _, bad = orc.snh_scene_inputs(m["X"], m["tets"], E, nu, 1000.0)
    assert bad == 0
    _, _, H = orc.snh_batch(x, snh["tets"], snh["Dminv"], snh["V"], snh["mu"], snh["lam"],
                            2, False)
    return H


@pytest.fixture(scope="module")
def barrier_hessians():
    sh = scenes.shell_sheet(10, length=0.01, noise=0.05, seed=5)
    nv = sh["x"].shape[0]
    bp = scenes.barrier_pairs(sh["x"], sh["tris"], 300, 1e-4, 1e-3, seed=5,
                              tri_node_offset=0, point_node_offset=nv)
    x = np.vstack([sh["x"], bp["points"]])
    _, _, H, act, bad = orc.barrier_batch(x, bp["pairs"], 1e-3, 1e4, 2, False)
    assert bad == 0
    return H[act == 1]


def test_low_mode_subspace_gives_the_clamp(snh_hessians):
    """SNH tets: with V the eigenvectors of the eigenvalues below 1e-5
    ||M||_F (k <= 3: the refinement's stencils), M - V B_- V^T is the
    oracle's clamp."""
    n = 0
    for H in snh_hessians:
        M = _m9(H)
        fro = np.linalg.norm(M)
        w, U = np.linalg.eigh(M)
        if w[0] >= -1e-13 * fro:
            continue
        k = int((w < 1e-5 * fro).sum())
        if k > 3:
            continue
        V = U[:, :k]
        Mc = M - V @ _neg_part(V.T @ M @ V) @ V.T
        ref, _ = orc.clamp_psd(H)
        assert np.linalg.norm(_h12(Mc) - ref) <= 1e-12 * np.linalg.norm(H)
        n += 1
    assert n > 100


def test_perturbed_subspace_within_the_residual_bound(snh_hessians):
    """A V rotated away from the exact subspace by up to 1e-6 rad: the
    result differs from the clamp by at most 2 sqrt(2) ||M V - V B||_F."""
    rng = np.random.default_rng(7)
    n = 0
    for H in snh_hessians[:400]:
        M = _m9(H)
        fro = np.linalg.norm(M)
        w, U = np.linalg.eigh(M)
        if w[0] >= -1e-13 * fro:
            continue
        k = int((w < 1e-5 * fro).sum())
        S = rng.standard_normal((9, 9)) * 1e-6
        Q, _ = np.linalg.qr(np.eye(9) + (S - S.T) / 2)
        V = (U @ Q)[:, :k]
        B = V.T @ M @ V
        R = M @ V - V @ B
        Mc = M - V @ _neg_part(B) @ V.T
        w2, U2 = np.linalg.eigh(M)
        exact = (U2 * np.maximum(w2, 0.0)) @ U2.T
        err = np.linalg.norm(Mc - exact)
        assert err <= 2 * np.sqrt(2) * np.linalg.norm(R) + 1e-13 * fro, (err, np.linalg.norm(R))
        n += 1
    assert n > 50


def test_deflation_certifies_the_barrier_null_space(barrier_hessians):
    """Barrier stencils: k = 6 with two clearly negative modes and four
    exact zeros. With V the two negative modes, M - V B V^T + tau I is
    positive definite (the certificate), and M - V B_- V^T is the clamp."""
    n = 0
    for H in barrier_hessians:
        M = _m9(H)
        fro = np.linalg.norm(M)
        w, U = np.linalg.eigh(M)
        if w[0] >= -1e-13 * fro:
            continue
        kneg = int((w < -1e-5 * fro).sum())
        assert kneg == 2 and int((w < 1e-5 * fro).sum()) == 6
        V = U[:, :kneg]
        B = V.T @ M @ V
        np.linalg.cholesky(M - V @ B @ V.T + 1e-13 * fro * np.eye(9))
        Mc = M - V @ _neg_part(B) @ V.T
        ref, _ = orc.clamp_psd(H)
        assert np.linalg.norm(_h12(Mc) - ref) <= 1e-12 * np.linalg.norm(H)
        n += 1
    assert n > 100


def test_certificate_rejects_a_missed_negative_mode(barrier_hessians):
    """Deflating only one of the two negative modes leaves one below -tau
    in the rest: the LDL^T certificate must fail (Cholesky raises)."""
    H = barrier_hessians[0]
    M = _m9(H)
    fro = np.linalg.norm(M)
    w, U = np.linalg.eigh(M)
    V = U[:, :1]
    B = V.T @ M @ V
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky(M - V @ B @ V.T + 1e-13 * fro * np.eye(9))

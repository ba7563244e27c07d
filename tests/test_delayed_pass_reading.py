"""The reading behind the FP32 Lanczos steps: CGS2 with the second pass delayed.

The CUDA path's FP32 steps orthogonalise each new Lanczos vector by the two classical
Gram-Schmidt passes of the oracle's Lanczos (§6, R3), but take the second pass one step
late: the vector v_j that enters step j has had only its first pass; one pass over the
basis B takes a = B^T v_j and g = B^T L v_j, from which q_j = (v_j - B a) / rho (its second
pass), column j of S = Q^T L Q and the first pass of the next vector follow.  This file
restates that recurrence in plain numpy on the oracle's Laplacian (the oracle's own
Lanczos keeps both passes in the step) and checks, in FP64 where the algebra is exact up to rounding, that it yields an
orthonormal basis, S = Q^T L Q, and the same Ritz values as two passes per step.  The
recurrence's formulas are the ones the kernels implement (step D2's closing arithmetic and
step D3's two updates).
"""
import numpy as np

from meshgen import box_graph_deleted
from oracle.amg import laplacian_csr


def _graph():
    g = box_graph_deleted(11, 9, 7, 0.08, 4, "vertex")
    return laplacian_csr(g).toarray().astype(np.float64)


def _start(n, seed=3):
    u0 = np.ones(n) / np.sqrt(n)
    x = np.random.default_rng(seed).standard_normal(n)
    return x - u0 * (u0 @ x), u0


def delayed_cycle(L, x, m, leak=0.0, drop_sa=False, seed=5):
    """One Lanczos cycle of m steps with the second pass delayed by one step.

    leak > 0 adds leak * (a random combination of the basis) to every first-pass result,
    standing in for a first pass that leaves components behind (which the FP32 first pass
    does at rounding level); drop_sa plants a mistake: S_kj without its - (S a)_k term.
    """
    n = L.shape[0]
    u0 = np.ones(n) / np.sqrt(n)
    rng = np.random.default_rng(seed)
    Q = np.zeros((m, n))
    S = np.zeros((m, m))
    src, nu = x.copy(), np.linalg.norm(x)
    for j in range(m):
        v = src / nu
        z = L @ v                                        # step D1
        B = np.vstack([u0[None, :], Q[:j]])
        a, g = B @ v, B @ z                              # step D2: one pass, two dots
        rho = np.sqrt(v @ v - a @ a)
        qz = (v @ z - a @ g) / rho
        aq = a[1:]
        sk = (g[1:] - (0.0 if drop_sa else S[:j, :j] @ aq)) / rho   # S_kj, k < j
        S[:j, j] = S[j, :j] = sk
        S[j, j] = (qz - sk @ aq) / rho
        q = (v - a @ B) / rho                            # step D3: q_j and w_{j+1}
        w = (z - g @ B - qz * q) / rho
        Q[j] = q
        if leak:
            Bn = np.vstack([u0[None, :], Q[: j + 1]])
            w = w + leak * np.linalg.norm(w) * (rng.standard_normal(j + 2) @ Bn)
        src, nu = w, np.linalg.norm(w)
    return Q, S


def two_pass_cycle(L, x, m):
    """The same cycle with both passes in the step (R3)."""
    n = L.shape[0]
    u0 = np.ones(n) / np.sqrt(n)
    Q = np.zeros((m, n))
    S = np.zeros((m, m))
    w = x.copy()
    for j in range(m):
        Q[j] = w / np.linalg.norm(w)
        w = L @ Q[j]
        B = np.vstack([u0[None, :], Q[: j + 1]])
        c1 = B @ w
        w = w - c1 @ B
        c2 = B @ w
        w = w - c2 @ B
        S[: j + 1, j] = S[j, : j + 1] = (c1 + c2)[1:]
    return Q, S


def test_delayed_pass_gives_an_orthonormal_basis_and_its_projection():
    L = _graph()
    x, u0 = _start(L.shape[0])
    Q, S = delayed_cycle(L, x, 40)
    assert np.abs(Q @ Q.T - np.eye(40)).max() < 1e-12
    assert np.abs(Q @ u0).max() < 1e-12
    assert np.abs(Q @ L @ Q.T - S).max() < 1e-11 * np.abs(L).max()


def test_delayed_pass_has_the_ritz_values_of_two_passes():
    L = _graph()
    x, _ = _start(L.shape[0])
    th_d = np.linalg.eigvalsh(delayed_cycle(L, x, 40)[1])
    th_2 = np.linalg.eigvalsh(two_pass_cycle(L, x, 40)[1])
    assert np.allclose(th_d, th_2, rtol=0, atol=1e-10 * np.abs(L).max())
    # and the smallest one approaches lambda_2 of the graph from above
    lam = np.linalg.eigvalsh(L)
    assert lam[1] - 1e-12 <= th_d[0] < lam[1] + 1e-3 * lam[-1]


def test_second_pass_removes_what_the_first_pass_leaves():
    # a first pass that leaves 1e-3 of every basis direction behind: the delayed second
    # pass still gives an orthonormal basis and S = Q^T L Q (the - (S a)_k term at work)
    L = _graph()
    x, _ = _start(L.shape[0])
    Q, S = delayed_cycle(L, x, 30, leak=1e-3)
    assert np.abs(Q @ Q.T - np.eye(30)).max() < 1e-12
    assert np.abs(Q @ L @ Q.T - S).max() < 1e-11 * np.abs(L).max()


def test_a_dropped_correction_term_breaks_the_projection():
    # planted mistake: without the - (S a)_k term S is off by about |S| |a|
    L = _graph()
    x, _ = _start(L.shape[0])
    Q, S = delayed_cycle(L, x, 30, leak=1e-3, drop_sa=True)
    assert np.abs(Q @ L @ Q.T - S).max() > 1e-6 * np.abs(L).max()

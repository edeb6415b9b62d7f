"""Pins of the BTP comparison preconditioner (Sec. 4) oracle: the
block-triangular structure (with exact inner inverses FGMRES converges in
two steps, the minimal-polynomial bound for a block-triangular
preconditioner with the exact Schur complement), the SA V-cycle as a
contracting stationary iteration, the exact block-diagonal mass inverse
for P1disc, and convergence with the V-cycle inverses."""
import numpy as np
import pytest

from oracle import btp as obtp, krylov
from problems import btp as pbtp, configs


@pytest.fixture(scope="module")
def c1():
    return configs.c1()


@pytest.fixture(scope="module")
def c1_btp(c1):
    return pbtp.build_btp(c1)


def _exact_parts(c1_btp):
    bt = c1_btp
    A = bt.A[0].toarray()
    B = bt.B.toarray()
    Ainv = np.linalg.inv(A)
    S = B @ Ainv @ B.T
    Sp = np.linalg.pinv(S, rcond=1e-10)  # enclosed flow: constant pressure null space
    return A, B, Ainv, Sp


def test_btp_with_exact_inverses_is_unipotent_and_converges_in_two_steps(c1, c1_btp):
    """With Q_A = A and Q_B = S = B A^-1 B^T the preconditioned operator is
    [[I, A^-1 B^T], [0, I]]: (P^-1 K - I)^2 = 0, so FGMRES takes two steps;
    the opposite sign of the pressure update gives eigenvalues +1 and -1
    instead (the square is then not zero)."""
    A, B, Ainv, Sp = _exact_parts(c1_btp)
    nu = A.shape[0]
    K = c1.K[0]

    def pre(r, sign=1.0):
        du = Ainv @ r[:nu]
        return np.concatenate([du, sign * (Sp @ (B @ du - r[nu:]))])

    rng = np.random.default_rng(5)
    v = rng.standard_normal(K.shape[0])
    v[nu:] -= v[nu:].mean()  # pressure part away from the constant null vector
    for sign, nilpotent in ((1.0, True), (-1.0, False)):
        Mv = pre(K @ v, sign) - v
        M2v = pre(K @ Mv, sign) - Mv
        ratio = np.linalg.norm(M2v) / np.linalg.norm(v)
        assert (ratio < 1e-8) == nilpotent, (sign, ratio)
    x, its, rel = krylov.fgmres(K, c1.b, pre, rtol=1e-8, restart=30, maxit=10)
    assert rel <= 1e-8 and its <= 3


def test_sa_vcycle_contracts_on_the_vector_laplacian(c1_btp):
    bt = c1_btp
    V = obtp.SAVCycle(bt.A, bt.PA)
    A = bt.A[0]
    rng = np.random.default_rng(3)
    e = rng.standard_normal(A.shape[0])
    for _ in range(3):
        e_new = e - V.apply(A @ e)
        assert np.sqrt(e_new @ (A @ e_new)) < 0.5 * np.sqrt(e @ (A @ e))
        e = e_new


def test_sv_mass_inverse_is_exact():
    pr = configs.c3(8)
    bt = pbtp.build_btp(pr)
    Q = pr.Mp / pr.nu
    I = (bt.Minv @ Q).toarray()
    assert np.abs(I - np.eye(Q.shape[0])).max() < 1e-10
    # P1disc: 3 x 3 blocks per cell
    assert bt.Minv.nnz == 9 * (Q.shape[0] // 3)


@pytest.mark.parametrize("which", ["th", "sv"])
def test_fgmres_with_btp_converges(which, c1):
    pr = c1 if which == "th" else configs.c3(8)
    bt = pbtp.build_btp(pr)
    o = obtp.BTPOracle(bt)
    x, its, rel = krylov.fgmres(pr.K[0], pr.b, o.apply, rtol=1e-8, restart=30, maxit=300)
    assert rel <= 1e-8

"""Pins of the oracle's projection variants (Dykstra, Douglas-Rachford, ADMM;
Sec. III names them as alternatives to POCS).

Each pin is independent of the oracle's recurrences: a quadratic program
solved by a general-purpose solver on the dense cos/sin constraint matrix,
closed forms derived by hand, and the theorem that ADMM on one ordering of
the two sets is Douglas-Rachford on the other ordering, run here with dense
projections (no FFT).
"""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W
from tests.test_oracle_pins import dense_basis

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _stress(shape, seed, frac):
    e0 = W.bimodal_error(shape, seed)
    return e0, 1.0, frac * O.f_violation(O.dft(e0))


def _dense_projections(shape, E, D, eta=O.ETA_DEFAULT):
    """P_S' and P_F' on flat vectors through the dense cos/sin basis."""
    B, nrm = dense_basis(shape)
    Es, Ds = E * (1 - eta), D * (1 - eta)

    def PS(x):
        return np.clip(x, -Es, Es)

    def PF(x):
        c = B @ x
        return x + ((np.clip(c, -Ds, Ds) - c) / nrm) @ B

    return PS, PF, B, Es, Ds


# ------------------------------------------ Dykstra = Euclidean projection
@pytest.mark.parametrize("shape,seed,frac", [((4, 4), 3, 0.5), ((4, 6), 4, 0.5), ((6, 6), 6, 0.4)])
def test_dykstra_converges_to_the_projection_onto_the_intersection(shape, seed, frac):
    e0, E, D = _stress(shape, seed, frac)
    _, _, B, Es, Ds = _dense_projections(shape, E, D)
    n = e0.size
    x0 = e0.reshape(-1)
    A = np.vstack([B, np.eye(n)])
    ub = np.concatenate([Ds * np.ones(len(B)), Es * np.ones(n)])
    qp = minimize(lambda x: 0.5 * np.sum((x - x0) ** 2), np.zeros(n), jac=lambda x: x - x0,
                  method="SLSQP",
                  constraints=[dict(type="ineq", fun=lambda x: ub - A @ x, jac=lambda x: -A),
                               dict(type="ineq", fun=lambda x: A @ x + ub, jac=lambda x: A)],
                  options=dict(ftol=1e-16, maxiter=1000))
    assert np.all(np.abs(A @ qp.x) <= ub * (1 + 1e-12))
    dk = O.correct_dykstra(e0, E, D, min_iters=3000, max_iters=3000)
    np.testing.assert_allclose(dk.e.reshape(-1), qp.x, rtol=0, atol=1e-9)
    # the pin discriminates: POCS stops at another point of the intersection
    pocs = O.correct(e0, E, D)
    assert np.max(np.abs(pocs.e.reshape(-1) - qp.x)) > 1e-3
    # early-stopped Dykstra is feasible and no farther from e0 than POCS here
    d = O.correct_dykstra(e0, E, D)
    assert d.status == O.OK and O.certify(d.e, E, D)[0]
    assert np.linalg.norm(d.e - e0) <= np.linalg.norm(pocs.e - e0)


# ---------------------------------------------------------- closed forms
@pytest.mark.parametrize("shape,k0", [((16,), (3,)), ((8, 8), (1, 2)), ((4, 8, 8), (1, 0, 3))])
def test_single_mode_closed_forms(shape, k0):
    """e0 = A cos(2 pi k0.n), A <= E', Delta' < A N/2 (a bin pair of height A N/2):
    Dykstra and ADMM stop after one iteration at (2 Delta'/N) cos (as Alg. 1);
    Douglas-Rachford reflects: x = P_S'(2y - z) = (4 Delta'/N - A) cos, which
    is feasible (one iteration) when A N/2 <= 3 Delta'."""
    N = int(np.prod(shape))
    grid = np.indices(shape).reshape(len(shape), -1).T
    ph = 2 * np.pi * (grid * (np.array(k0) / np.array(shape))).sum(1)
    c = np.cos(ph).reshape(shape)
    E, eta = 1.0, O.ETA_DEFAULT
    A = 0.5
    D = 0.4 * A * N / 2            # A N/2 = 2.5 D  (between D' and 3 D')
    Ds = D * (1 - eta)
    for fn in (O.correct_dykstra, O.correct_admm):
        r = fn(A * c, E, D)
        assert r.status == O.OK and r.iters == 1, fn.__name__
        np.testing.assert_allclose(r.e, (2 * Ds / N) * c, rtol=0, atol=1e-13)
    r = O.correct_douglas_rachford(A * c, E, D)
    assert r.status == O.OK and r.iters == 1
    np.testing.assert_allclose(r.e, (4 * Ds / N - A) * c, rtol=0, atol=1e-13)
    # A N/2 > 3 Delta': the reflected point is infeasible, DR needs more steps
    r = O.correct_douglas_rachford(A * c, E, 0.2 * A * N / 2)
    assert r.iters > 1 and r.status == O.OK


def test_spike_closed_forms():
    """e0 = E' 1_{n=0} with Delta < E: every bin equals E', so P_F' gives
    Delta' 1_{n=0} (Dykstra, ADMM: one iteration, that point); DR reflects to
    (2 Delta' - E') 1_{n=0}, feasible when E' <= 3 Delta'."""
    shape = (4, 4, 4)
    E, eta = 1.0, O.ETA_DEFAULT
    Es = E * (1 - eta)
    D = 0.6
    Ds = D * (1 - eta)
    e0 = np.zeros(shape)
    e0[0, 0, 0] = Es
    spike = np.zeros(shape)
    spike[0, 0, 0] = 1.0
    for fn in (O.correct_dykstra, O.correct_admm):
        r = fn(e0, E, D)
        assert r.iters == 1 and r.status == O.OK
        np.testing.assert_allclose(r.e, Ds * spike, rtol=0, atol=1e-14)
    r = O.correct_douglas_rachford(e0, E, D)
    assert r.iters == 1 and r.status == O.OK
    np.testing.assert_allclose(r.e, (2 * Ds - Es) * spike, rtol=0, atol=1e-14)


# ------------------------------- ADMM on one order = DR on the other order
def _admm_dense(e0, PS, PF, a_first, b_second, K):
    """Scaled ADMM a <- P1(b - u), b <- P2(a + u), u <- u + a - b (b_0 = e0)."""
    b = e0.copy()
    u = np.zeros_like(b)
    out = []
    for _ in range(K):
        a = a_first(b - u)
        b = b_second(a + u)
        u = u + a - b
        out.append(a)
    return out


@pytest.mark.parametrize("shape,seed,frac", [((4, 6), 4, 0.5), ((6, 6), 6, 0.4), ((16,), 5, 0.3)])
def test_admm_and_douglas_rachford_are_the_same_splitting(shape, seed, frac):
    """ADMM on (F', S') from b_0 = e0 visits a_{k+2} = x_k of DR on (S', F')
    from w_0 = a_1; ADMM on (S', F') from b_0 = e0 visits a_{k+2} = x_{k+1} of
    DR on (F', S') from z_0 = a_1 = P_S'(e0) = e0.  Both DR runs and the
    second ADMM are written here with dense projections."""
    e0, E, D = _stress(shape, seed, frac)
    e0 = np.clip(e0, -E * (1 - O.ETA_DEFAULT), E * (1 - O.ETA_DEFAULT))   # P_S'(e0) = e0
    PS, PF, _, _, _ = _dense_projections(shape, E, D)
    x0 = e0.reshape(-1)
    K = 6
    # oracle ADMM (F' first): trajectory [a_1, a_2, ...]
    ad = O.correct_admm(e0, E, D, min_iters=K, max_iters=K, record=True)
    a = [v.reshape(-1) for v in ad.trajectory]
    w = a[0].copy()
    for k in range(K - 1):                 # DR on (S', F')
        y = PS(w)
        x = PF(2 * y - w)
        w = w + x - y
        np.testing.assert_allclose(a[k + 1], x, rtol=0, atol=1e-12)
    # oracle DR (F' first) against ADMM on (S', F')
    dr = O.correct_douglas_rachford(e0, E, D, min_iters=K, max_iters=K, record=True)
    a2 = _admm_dense(x0, PS, PF, PS, PF, K + 1)
    for k in range(K):
        np.testing.assert_allclose(dr.trajectory[k].reshape(-1), a2[k + 1], rtol=0, atol=1e-12)


# ----------------------------------------------------- loop control rules
@pytest.mark.parametrize("method", ["dykstra", "dr", "admm"])
def test_variant_loop_rules(method):
    e0, E, D = _stress((8, 8), 11, 0.4)
    r = O.correct_method(e0, E, D, method)
    assert r.status == O.OK and r.iters >= 1
    ok, s, v = O.certify(r.e, E, D)
    assert ok
    # zero iterations on feasible input, e returned as given
    z = O.correct_method(0.5 * e0, E, 10 * O.f_violation(O.dft(e0)), method)
    assert z.iters == 0 and np.array_equal(z.e, 0.5 * e0)
    # forced iterations and the cap
    f = O.correct_method(e0, E, D, method, min_iters=r.iters + 3, max_iters=r.iters + 3)
    assert f.iters == r.iters + 3
    c = O.correct_method(e0, E, D, method, max_iters=r.iters - 1)
    assert c.status == O.NOT_CONVERGED and c.iters == r.iters - 1
    # negation: both sets are symmetric, every variant is odd
    n = O.correct_method(-e0, E, D, method)
    assert n.iters == r.iters
    np.testing.assert_allclose(n.e, -r.e, rtol=0, atol=1e-13)


def test_variant_pins_catch_planted_mistakes(monkeypatch):
    """Plant mistakes in the oracle's variant path (on the CPU) and check that
    a pin above fails: a disc projection instead of the Re/Im box misses the
    QP solution; a sign slip in the frequency projection misses the closed
    forms."""
    shape, seed, frac = (4, 4), 3, 0.5
    e0, E, D = _stress(shape, seed, frac)
    good = O.correct_dykstra(e0, E, D, min_iters=3000, max_iters=3000).e

    def disc(z, Ds):
        d = O.dft(z)
        m = np.abs(d)
        return O.idft(np.where(m > Ds, d * (Ds / np.maximum(m, 1e-300)), d))
    monkeypatch.setattr(O, "project_f_spatial", disc)
    bad = O.correct_dykstra(e0, E, D, min_iters=3000, max_iters=3000).e
    assert np.max(np.abs(bad - good)) > 1e-3
    monkeypatch.undo()

    c = np.cos(2 * np.pi * 3 * np.arange(16) / 16)
    want = O.correct_douglas_rachford(0.5 * c, 1.0, 0.4 * 0.5 * 8).e
    monkeypatch.setattr(O, "project_f_spatial", lambda z, Ds: -O.idft(O.project_f(O.dft(-z), Ds)) * 0.5 + 0.5 * z)
    bad = O.correct_douglas_rachford(0.5 * c, 1.0, 0.4 * 0.5 * 8, max_iters=1).e
    assert np.max(np.abs(bad - want)) > 1e-3

"""CPU checks of the forms the scattering kernels evaluate (Eq. 6, S = eps B + (1 - eps) J).

The device builds the rows of Lambda (J = Lambda S for a piecewise-linear source) as second
divided differences of G(t) = E3(|t - tau_j|)/2 + |t - tau_j|/2, whose second derivative is the
kernel E1(|t - tau_j|)/2 of J; it writes dJ/dtau (S fixed) in the same terms, and inverts
M = I - diag(1 - eps) Lambda by Gauss-Jordan elimination with the pivot row and column folded
into one update a_rk - f_r g_k.  These tests restate those three forms in FP64 numpy and compare
them with the oracle's Lambda and dJ/dtau, which the oracle builds from segment weights, and
with numpy's inverse.  A dropped term, a sign or an index slip in a restated form fails here.
They do not call the CUDA path.
"""
import numpy as np
import pytest

special = pytest.importorskip("scipy.special")


def _E(n, x):
    return special.expn(n, np.abs(x))


def _tau_grid(nd, lo, hi, seed):
    rng = np.random.default_rng(seed)
    x = np.sort(np.concatenate([[lo, hi], rng.uniform(lo, hi, nd - 2)]))
    return 10.0 ** x


def lambda_divided_differences(tau):
    """Lambda from qt_k = (E3(|tau_{k+1} - tau_j|) - E3(|tau_k - tau_j|)) / (2 D_k) (qt_{-1} over
    [0, tau_0]): Lambda_jk = qt_k - qt_{k-1} + [k = j] below the bottom layer, G'(tau_{N-1}^-) -
    qt_{N-2} at it, and the top segment's weight of S(0), qt_{-1} - E2(tau_j)/2, carried to
    layers 0 and 1 by S(0) = S_0 (1 + tau_0/D_0) - S_1 tau_0/D_0."""
    N = tau.size
    L = np.zeros((N, N))
    nodes = np.concatenate([[0.0], tau])          # node -1 is t = 0
    h = 0.5 / np.diff(nodes)                      # 1/(2 D) of segments -1 .. N-2
    r = tau[0] / (tau[1] - tau[0])
    for j in range(N):
        e3 = _E(3, nodes - tau[j])                # E3 at t = 0 and at every layer
        qt = (e3[1:] - e3[:-1]) * h               # qt_{-1} .. qt_{N-2}
        for k in range(N - 1):
            L[j, k] = qt[k + 1] - qt[k] + (1.0 if k == j else 0.0)
        gp = -0.5 * _E(2, tau[N - 1] - tau[j]) if j < N - 1 else 0.5
        L[j, N - 1] = gp - qt[N - 1]
        wz = qt[0] - 0.5 * _E(2, tau[j])
        L[j, 0] += wz * (1.0 + r)
        L[j, 1] -= wz * r
    return L


def seg_weights(D, e2n, e3n, e2f, e3f):
    P = e2n - e2f
    Q = 2 * (e3n - e3f - D * e2f) / D - P
    return 0.25 * (P - Q), 0.25 * (P + Q)


def dj_dtau_compact(tau, S):
    """dJ_j/dtau_k at fixed S: inner layers k != j from -sgn(k - j) E2/2 (s_k - s_{k-1}) +
    s_{k-1} qt_{k-1} - s_k qt_k; the end layers from one segment's weight; the top segment's
    extrapolation terms at k <= 1, the slab end at k = N - 1; the diagonal from the row sum
    S(0) E1(tau_j)/2."""
    N = tau.size
    D1 = tau[1] - tau[0]
    t0 = tau[0]
    s0 = (S[1] - S[0]) / D1
    sl = np.diff(S) / np.diff(tau)
    out = np.zeros((N, N))
    for j in range(N):
        e2 = _E(2, tau - tau[j])
        e3 = _E(3, tau - tau[j])
        qt = 0.5 * np.diff(e3) / np.diff(tau)     # qt_0 .. qt_{N-2}
        whi, wlo = seg_weights(t0, e2[0], e3[0], _E(2, tau[j]), _E(3, tau[j]))
        for k in range(N):
            if k == j:
                continue
            if k == 0 or k == N - 1:
                kk = 0 if k == 0 else N - 2
                D = tau[kk + 1] - tau[kk]
                if kk >= j:
                    wa, wb = seg_weights(D, e2[kk], e3[kk], e2[kk + 1], e3[kk + 1])
                else:
                    wb, wa = seg_weights(D, e2[kk + 1], e3[kk + 1], e2[kk], e3[kk])
                v = -sl[kk] * (wa if k == kk else wb)
                if k == N - 1:
                    v += 0.5 * S[N - 1] * special.exp1(tau[N - 1] - tau[j])
            else:
                sg = 1.0 if k > j else -1.0
                v = -0.5 * sg * e2[k] * (sl[k] - sl[k - 1]) + sl[k - 1] * qt[k - 1] - sl[k] * qt[k]
            if k == 0:
                v += -(s0 / D1) * t0 * wlo - s0 * (wlo + whi)
            elif k == 1:
                v += (s0 / D1) * t0 * wlo
            out[j, k] = v
        out[j, j] = 0.5 * (S[0] - s0 * t0) * special.exp1(tau[j]) - out[j].sum()
    return out


def gauss_jordan_fused(M):
    """In-place Gauss-Jordan inverse without pivoting, every element updated as a_rk - f_r g_k
    with f_r = (a_rp - [r = p]) / a_pp and g_k = a_pk + [k = p]."""
    A = np.array(M, dtype=np.float64)
    n = A.shape[0]
    for p in range(n):
        col, row = A[:, p].copy(), A[p, :].copy()
        inv = 1.0 / row[p]
        f = (col - (np.arange(n) == p)) * inv
        g = row + (np.arange(n) == p)
        A -= np.outer(f, g)
    return A


@pytest.mark.parametrize("nd,lo,hi,seed", [(2, -2.0, 0.5, 1), (3, -3.0, 1.0, 2), (12, -4.0, 1.5, 3),
                                          (40, -6.0, 2.0, 4), (72, -7.0, 2.3, 5)])
def test_divided_difference_lambda_matches_the_oracle(oracle, nd, lo, hi, seed):
    """The kernel's Lambda against the oracle's segment-weight Lambda.  Both carry the
    cancellation floor of difference quotients over the finest steps, about 1e-16/D_min
    absolute (the ulp of E3 near 1/2 divided by the step); the bar is ten times that, and
    never below 1e-13."""
    tau = _tau_grid(nd, lo, hi, seed)
    L = lambda_divided_differences(tau)
    ref = oracle.lambda_matrix(tau)
    floor = max(1e-13, 10 * 1.1e-16 / np.min(np.diff(np.concatenate([[0.0], tau]))))
    assert np.max(np.abs(L - ref)) <= floor, (np.max(np.abs(L - ref)), floor)
    # rows sum to the mean intensity of S = 1: 1 - E2(tau_j)/2 - E2(T - tau_j)/2
    J1 = L.sum(axis=1)
    ref1 = 1 - 0.5 * _E(2, tau) - 0.5 * _E(2, tau[-1] - tau)
    assert np.max(np.abs(J1 - ref1)) <= 10 * floor


@pytest.mark.parametrize("nd,seed", [(2, 6), (3, 7), (10, 8), (30, 9)])
def test_compact_dj_dtau_matches_the_oracle(oracle, nd, seed):
    """Row by row against the oracle, relative to the row's largest element.  The top
    segment's extrapolation multiplies its weights (FP64 rounding ~ulp/tau_0) by
    (S_1 - S_0) tau_0 / D_1^2, up to ~3e5 on these grids' finest top steps, so two FP64
    evaluations of the same quantity differ by a few 1e-9 of the row there; the bar is 2e-8,
    far below the O(1) error of a dropped term or a wrong sign."""
    tau = _tau_grid(nd, -3.0, 1.5, seed)
    S = np.random.default_rng(seed).uniform(0.5, 2.0, nd)
    got = dj_dtau_compact(tau, S)
    ref = oracle.lambda_dtau(tau, S)
    rel = np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert np.max(rel) <= 2e-8, (np.max(rel), int(np.argmax(rel)))


@pytest.mark.parametrize("eps_lo", [0.5, 1e-2, 1e-4])
def test_fused_gauss_jordan_is_the_inverse(oracle, eps_lo):
    """On M = I - diag(1 - eps) Lambda (diagonally dominant) the fused update gives the
    inverse without pivoting; the bar follows the condition number (~1/eps)."""
    tau = _tau_grid(30, -4.0, 2.0, 11)
    eps = np.random.default_rng(12).uniform(eps_lo, 1.0, tau.size)
    M = np.eye(tau.size) - (1 - eps)[:, None] * oracle.lambda_matrix(tau)
    inv = gauss_jordan_fused(M)
    cond = np.linalg.cond(M)
    assert np.max(np.abs(inv @ M - np.eye(tau.size))) <= 1e-14 * cond, cond
    np.testing.assert_allclose(inv, np.linalg.inv(M), rtol=0, atol=1e-13 * cond * np.max(np.abs(inv)))

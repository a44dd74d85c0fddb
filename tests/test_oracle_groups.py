"""Pins of the oracle's linked correction groups (Sec. 6, Eq. 10 with q(l)): the greedy
strength-ordered grouping on a worked example and by its defining properties on random
clustered lists, and the group gradients against central differences of the forward."""
import numpy as np
import pytest

from group_util import DE_EV, DLAM_NM, clustered_lines
from tiny import tiny_problem


def test_worked_example(oracle):
    """Seven lines worked by hand: 0 and 6 tie for the strongest (index order: 0 seeds);
    1 is inside both tolerances of 0; 2 is 0.040 nm from 0 and seeds the next group, which
    takes 5 (0.030 nm, 1e-4 eV away); 4 is 0.001 eV from 0 and from 2, so it stands alone;
    3 is another species."""
    lam = np.array([1600.000, 1600.030, 1600.040, 1600.010, 1600.005, 1600.070, 1600.000])
    E = np.array([1.0000, 1.0002, 1.0000, 1.0000, 1.0010, 1.0001, 1.0000], np.float32)
    sp = np.array([3, 3, 3, 4, 3, 3, 3], np.int32)
    st = np.array([5.0, 2.0, 4.0, 1.0, 3.0, 0.5, 5.0], np.float32)
    q, G = oracle.build_line_groups(lam, E, sp, st, DE_EV, DLAM_NM)
    assert G == 4
    assert q.tolist() == [0, 0, 1, 3, 2, 1, 0]


def _close(lam, E, sp, a, b):
    return (sp[a] == sp[b] and abs(float(E[a]) - float(E[b])) <= DE_EV and abs(lam[a] - lam[b]) <= DLAM_NM)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_greedy_grouping_properties(oracle, seed):
    """Brute-force check of the defining properties: every line is in one group; a
    group's seed is its strongest member (lowest index among equals) and every member is
    within both tolerances of it with its species; seeds open groups in descending
    strength; and no line was left out of an earlier group whose seed it was close to."""
    lam, E, sp, st = clustered_lines(120, seed)
    n = lam.size
    q, G = oracle.build_line_groups(lam, E, sp, st, DE_EV, DLAM_NM)
    assert q.min() == 0 and q.max() == G - 1 and np.unique(q).size == G
    seeds = []
    for g in range(G):
        mem = np.nonzero(q == g)[0]
        s = min(mem, key=lambda k: (-float(st[k]), k))
        seeds.append(s)
        assert all(_close(lam, E, sp, s, m) for m in mem)
    keys = [(-float(st[s]), s) for s in seeds]
    assert keys == sorted(keys)
    for m in range(n):
        for g in range(q[m]):                 # groups opened before m's own
            assert not _close(lam, E, sp, seeds[g], m), (m, g)
    assert G < n                              # the clustering formed real groups


def test_group_gradient_matches_central_differences(oracle):
    """dL/ddelta_q (group sum of member gradients) against central differences of the
    forward with the group's correction copied to its members, for all four families."""
    prob = tiny_problem(n_lambda=160, n_depth=10, n_lines=7, W=60, seed=21, instrument=False, E_max=1.0)
    prob.lines.log_gf[:] -= 4.0
    q = np.array([0, 0, 1, -1, 1, 2, 2])
    G = 3
    rng = np.random.default_rng(4)
    keys = ("dlog_gf", "dlog_gamma_rad", "dlog_gamma4", "dlog_gamma6")
    x = rng.normal(0, 0.1, (4, G))

    def corr_of(xg):
        e = oracle.expand_groups(xg, q)
        return {k: e[j] for j, k in enumerate(keys)}

    f0 = oracle.forward(prob, corr_of(x))["f"]
    y = f0 + rng.normal(0, 0.01, f0.size)
    w = np.full(f0.size, 4e4)
    r = oracle.gradient4(prob, y, w, corr_of(x))
    g_line = np.stack([r["gf"], r["gamma_rad"], r["gamma4"], r["gamma6"]])
    g_grp = oracle.group_sum(g_line, q, G)
    assert np.all(oracle.expand_groups(x, q)[:, 3] == 0.0)       # ungrouped line: no correction
    h = 1e-4
    for j in range(4):
        for g in range(G):
            def L_at(t):
                xx = x.copy()
                xx[j, g] += t
                return oracle.chi2(y, w, oracle.forward(prob, corr_of(xx))["f"])[0]
            d1 = (L_at(h) - L_at(-h)) / (2 * h)
            d2 = (L_at(2 * h) - L_at(-2 * h)) / (4 * h)
            fd = (4 * d1 - d2) / 3
            scale = max(abs(fd), 1e-3 * np.max(np.abs(g_grp[j])))
            assert abs(g_grp[j, g] - fd) <= 1e-6 * scale + 1e-9, (keys[j], g, g_grp[j, g], fd)

"""The library's greedy line grouping (host code behind the C ABI) against the oracle's:
identical group ids (integer work, bit-exact) on the worked example, clustered random
lists, exact ties and duplicates, and its argument checks."""
import numpy as np
import pytest

from group_util import DE_EV, DLAM_NM, clustered_lines


@pytest.fixture(scope="module")
def pz():
    import paper_2607_24141_gb300 as pz
    try:
        pz.load(build_if_missing=False)
    except Exception as e:          # the library is built by __graft_entry__.build()
        pytest.skip("libpz.so not built: %s" % e)
    return pz


def _both(pz, oracle, lam, E, sp, st, dE=DE_EV, dlam=DLAM_NM):
    q1, G1 = pz.pz_build_line_groups(lam, E, sp, st, dE, dlam)
    q0, G0 = oracle.build_line_groups(lam, E, sp, st, dE, dlam)
    assert G1 == G0
    np.testing.assert_array_equal(q1, q0)
    return q1, G1


def test_worked_example(pz, oracle):
    lam = np.array([1600.000, 1600.030, 1600.040, 1600.010, 1600.005, 1600.070, 1600.000])
    E = np.array([1.0000, 1.0002, 1.0000, 1.0000, 1.0010, 1.0001, 1.0000], np.float32)
    sp = np.array([3, 3, 3, 4, 3, 3, 3], np.int32)
    st = np.array([5.0, 2.0, 4.0, 1.0, 3.0, 0.5, 5.0], np.float32)
    q, G = _both(pz, oracle, lam, E, sp, st)
    assert q.tolist() == [0, 0, 1, 3, 2, 1, 0] and G == 4


@pytest.mark.parametrize("seed", range(5))
def test_clustered_lists(pz, oracle, seed):
    lam, E, sp, st = clustered_lines(400, seed)
    q, G = _both(pz, oracle, lam, E, sp, st)
    assert G < lam.size


def test_boundaries_ties_and_duplicates(pz, oracle):
    """Lines exactly at the tolerances (both sides decide in FP64 from the same inputs),
    duplicated lines, equal strengths, zero tolerances and the empty list."""
    rng = np.random.default_rng(3)
    base = 1600.0 + np.round(rng.uniform(0, 0.5, 60), 3)
    lam = np.concatenate([base, base + DLAM_NM, base - DLAM_NM, base])
    E = np.concatenate([np.full(60, 1.0), np.full(60, 1.0), np.full(60, 1.0 + DE_EV), np.full(60, 1.0)]).astype(np.float32)
    sp = np.tile(rng.integers(0, 2, 60), 4).astype(np.int32)
    st = np.round(rng.normal(size=240), 1).astype(np.float32)
    _both(pz, oracle, lam, E, sp, st)
    _both(pz, oracle, lam, E, sp, st, 0.0, 0.0)
    q, G = pz.pz_build_line_groups(np.zeros(0), np.zeros(0, np.float32), np.zeros(0, np.int32),
                                   np.zeros(0, np.float32), DE_EV, DLAM_NM)
    assert q.size == 0 and G == 0


def test_argument_checks(pz):
    lam, E, sp, st = clustered_lines(5, 0)
    with pytest.raises(pz.PzError) as e:
        pz.pz_build_line_groups(lam, E, sp, st, -1.0, DLAM_NM)
    assert e.value.status == pz.PZ_EINVAL
    st[0] = np.nan
    with pytest.raises(pz.PzError) as e:
        pz.pz_build_line_groups(lam, E, sp, st, DE_EV, DLAM_NM)
    assert e.value.status == pz.PZ_EINVAL

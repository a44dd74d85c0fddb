"""The seeded generators: sizes, determinism and ranges of the synthetic workloads."""
import numpy as np

from paper_2607_24141_gb300 import inputs as I


def test_grid_sizes_eq2():
    assert I.n_lambda_for(1500.0, 1700.0) == 37550
    assert I.n_lambda_for(300.0, 1000.0) == 361193


def test_config0_shapes_and_determinism():
    a, b = I.config0(), I.config0()
    assert a.grid.n_lambda == 4000 and a.lines.n_lines == 2000 and a.atmos.n_depth == 72
    assert a.atmos.n_species == 12 and a.lines.half_window == 1000
    assert np.array_equal(a.lines.lambda_nm, b.lines.lambda_nm)
    assert np.array_equal(a.atmos.pop, b.atmos.pop)
    assert a.kappa_c.shape == (72, 4000) and np.all(a.kappa_c > 0)
    assert np.all(np.diff(a.atmos.m) > 0)
    assert 2.3e8 < a.n_evals < 2.7e8


def test_config1_recipe():
    p = I.config1()
    assert p.grid.n_lambda == 37550 and p.lines.n_lines == 200_000
    assert p.instrument.pix_lambda_nm.size == 8575
    assert 1510.0 < p.instrument.pix_lambda_nm[0] < p.instrument.pix_lambda_nm[-1] < 1700.0
    band = np.isin(p.lines.species, [36, 37, 38, 39])
    assert band.sum() == 66_500
    assert np.all(p.lines.species < 40) and p.n_elem == 20
    assert 3.8e10 < p.n_evals < 4.6e10


def test_config3_truth_draws():
    p, truth = I.config3()
    assert p.lines.n_lines == 120_000
    assert abs(np.std(truth["dlog_gf"]) - 0.1) < 0.005
    assert abs(np.std(truth["dlog_gamma6"]) - 0.2) < 0.005
    assert truth["noise"].size == 8575


def test_atmosphere_physical_ranges():
    at = I.make_atmosphere(4500.0, 2.0, 40, 1)
    assert np.all(at.T > 2000) and np.all(at.T < 20000)
    assert np.all(at.n_pert > at.n_e)
    assert np.all(at.pop > 0)


def test_config4_batch_recipe():
    b = I.config4()
    assert b.n_stars == 64 and b.lines.n_lines == 300_000
    teff, logg, mh, nk = I.config4_stars(4, 64)
    sizes = np.array([len(s) for s in b.subsets])
    assert np.array_equal(sizes, np.minimum(nk, 300_000))
    assert sizes.min() >= 20_000 and sizes.max() <= 300_000
    for s in b.subsets[:5]:
        assert np.all(np.diff(s) > 0) and s.min() >= 0 and s.max() < 300_000
    # each star keeps its strongest lines by the proxy
    p = I.strength_proxy(b.atmos[0], b.lines)
    kept = np.zeros(300_000, bool)
    kept[b.subsets[0]] = True
    assert p[kept].min() >= p[~kept].max()
    assert [a.teff for a in b.atmos] == list(teff)
    # one chemistry for every star: same masses and partition pattern, scaled by [M/H]
    assert np.array_equal(b.atmos[0].mass_amu, b.atmos[7].mass_amu)
    c = I.config4()
    assert all(np.array_equal(x, y) for x, y in zip(b.subsets, c.subsets))


def test_config4_joint_and_small_batch():
    jb, truth = I.config4_joint()
    assert jb.n_stars == 2 and len(jb.subsets[0]) == 100_000
    assert np.array_equal(jb.subsets[0], jb.subsets[1])
    assert (jb.atmos[0].teff, jb.atmos[1].teff) == (5777.0, 4286.0)
    assert truth["noise"].shape == (2, 8575)
    sb = I.small_batch(n_stars=3)
    assert [len(s) for s in sb.subsets][0] == sb.lines.n_lines
    st = sb.star(1)
    assert st.lines.n_lines == len(sb.subsets[1])
    assert np.array_equal(st.lines.lambda_nm, sb.lines.lambda_nm[sb.subsets[1]])


def test_recipes_give_realistic_line_depths(oracle):
    """The population scale of each workload gives a spectrum with continuum windows and
    saturated cores, not a saturated line forest (checked on small slices with the oracle)."""
    for prob in (I.config0(n_lambda=1500, n_lines=750),
                 I.small_config1(n_lambda_span_nm=3.0, seed=13, with_instrument=False)):
        f = oracle.forward(prob)["f"]
        p5, p50 = np.percentile(f, [5, 50])
        assert 0.8 < p50 < 0.995 and p5 < 0.8, (prob.name, p5, p50)


def test_wavelength_slice_keeps_exactly_the_lines_that_reach_it():
    import math
    p = I.config0()
    q = I.wavelength_slice(p, 502.0, 700)
    lnr = math.log1p(1.0 / p.grid.R_grid)
    i0 = round(math.log(q.grid.lambda0_nm / p.grid.lambda0_nm) / lnr)
    assert q.grid.lambda0_nm >= 502.0 and q.grid.lambda0_nm < 502.0 * (1 + 1.0 / p.grid.R_grid)
    assert q.grid.n_lambda == 700 and q.grid.R_grid == p.grid.R_grid
    assert np.array_equal(q.kappa_c, p.kappa_c[:, i0:i0 + 700])
    il = I.center_index(p.grid, p.lines.lambda_nm)
    W = p.lines.half_window
    reach = (il + W >= i0) & (il - W <= i0 + 699)
    assert q.lines.n_lines == int(reach.sum())
    assert np.array_equal(np.sort(q.lines.lambda_nm), np.sort(p.lines.lambda_nm[reach]))
    # the slice's own evaluation count equals the full problem's evaluations inside the slice
    lo = np.maximum(il - W, i0)
    hi = np.minimum(il + W, i0 + 699)
    assert q.n_evals == int(np.maximum(hi - lo + 1, 0).sum()) * p.atmos.n_depth

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

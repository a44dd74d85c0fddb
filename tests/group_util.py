"""Seeded line lists with component complexes for the grouping tests (no arithmetic of
the method: positions, energies, species and strengths drawn around seeds)."""
import numpy as np

HC_EV_CM = 1.239841984e-4          # h c in eV cm (CODATA 2018): 1 cm^-1 of lower-level energy in eV
DE_EV = 2.0 * HC_EV_CM             # the paper's 2.0 cm^-1
DLAM_NM = 0.035


def clustered_lines(n_seed, seed):
    """Component complexes: seeds spread over 2 nm and a few species, each with 0-3
    companions inside or just outside the tolerances (so that both branches occur)."""
    rng = np.random.default_rng(seed)
    lam, E, sp, st = [], [], [], []
    for _ in range(n_seed):
        l0, e0, s0 = rng.uniform(1600, 1602), rng.uniform(0, 5), int(rng.integers(0, 4))
        for k in range(1 + int(rng.integers(0, 4))):
            lam.append(l0 + (rng.uniform(-0.05, 0.05) if k else 0.0))
            E.append(e0 + (rng.uniform(-1.5, 1.5) * DE_EV if k else 0.0))
            sp.append(s0 if rng.uniform() < 0.9 else s0 + 1)
            st.append(rng.choice([rng.normal(), 1.0]))           # some exact ties
    return (np.array(lam), np.array(E, np.float32), np.array(sp, np.int32), np.array(st, np.float32))

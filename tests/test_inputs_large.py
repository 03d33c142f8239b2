"""The large workload's input recipe (the 1,024-site jittered FCC cluster on a 192^3 grid):
the geometry and parameters the recipe states, checked on the CPU.  No propagation runs
here; the generator holds inputs only."""
import numpy as np
from scipy.spatial.distance import pdist

from paper_2410_09189_gb300 import inputs


def test_fcc_sites_are_the_nearest_lattice_sites():
    sites = inputs.fcc_sites(1024)
    assert sites.shape == (1024, 3)
    assert len(np.unique(np.round(sites, 9), axis=0)) == 1024
    assert np.allclose(sites[0], 0.0)   # a site at the centre
    # nearest-neighbour distance 5.4 bohr (cube edge 5.4 sqrt 2)
    assert abs(pdist(sites).min() - 5.4) < 1e-9
    # no unselected lattice site is nearer the centre than a selected one
    more = inputs.fcc_sites(1400)
    r_sel = np.linalg.norm(sites, axis=1).max()
    r_rest = np.linalg.norm(more[1024:], axis=1).min()
    assert r_sel <= r_rest + 1e-9
    # deterministic selection
    assert np.array_equal(sites, inputs.fcc_sites(1024))


def test_fcc_large_parameters_and_fit_in_the_box():
    s = inputs.fcc_large()
    assert s.n == (192, 192, 192) and abs(s.h - 0.4) < 1e-15
    assert s.pos.shape == (1024, 3) and s.N == 2048 and s.nocc == 1024
    assert np.all(s.Z == 2.0) and 2 * s.nocc == int(s.Z.sum())   # neutral, doubly occupied
    assert s.nproj == 4096
    assert np.array_equal(np.bincount(s.proj_atom), np.full(1024, 4))
    assert np.array_equal(s.proj_l[:4], [0, 1, 1, 1]) and np.array_equal(s.proj_m[:4], [0, 0, 1, 2])
    assert np.all((s.E_kb >= 0.5) & (s.E_kb <= 2.0)) and np.all(s.proj_rc == 1.2)
    jit = s.pos - inputs.fcc_sites(1024)
    assert 0.08 < jit.std() < 0.12 and np.abs(jit).max() < 0.6
    assert pdist(s.pos).min() > 5.4 - 1.2
    # every projector's support (5 r_c) inside the grid
    half = 0.5 * (s.n[0] - 1) * s.h
    assert np.abs(s.pos).max() + 5 * 1.2 < half
    # seeded: the same draws every time
    s2 = inputs.fcc_large()
    assert np.array_equal(s.pos, s2.pos) and np.array_equal(s.E_kb, s2.E_kb)

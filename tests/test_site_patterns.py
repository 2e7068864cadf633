"""The atom-resolved input patterns (synth/sites.py) against a brute-force pair search: every pair of
sites closer than (r_a + r_b)/2 under the minimum image, and no other, with each site its own neighbour,
N(J) ascending and the relation symmetric; water geometry (O-H 0.96 Angstrom, H-O-H 104.5 degrees) and
the function counts of the paper's basis (H 2, O 4, ion 4)."""
import numpy as np

from synth import SiteSpec, make_site_pattern


def test_pattern_matches_brute_force():
    sp = make_site_pattern(SiteSpec(3, 3, 3, ion_fraction=0.2, seed=77))
    n = sp.n_sites
    radius = np.where(sp.species == 2, sp.spec.rc_ion, sp.spec.rc)
    got = {(int(sp.nb_idx[p]), J) for J in range(n) for p in range(sp.nb_ptr[J], sp.nb_ptr[J + 1])}
    want = set()
    for a in range(n):
        for b in range(n):
            d = sp.pos[b] - sp.pos[a]
            d = d - sp.cell * np.rint(d / sp.cell)
            if float(d @ d) < (0.5 * (radius[a] + radius[b])) ** 2:
                want.add((a, b))
    assert got == want
    for J in range(n):
        rows = list(sp.nb_idx[sp.nb_ptr[J]:sp.nb_ptr[J + 1]])
        assert J in rows and rows == sorted(rows)
    assert all((b, a) in got for a, b in got)


def test_water_geometry_and_function_counts():
    sp = make_site_pattern(SiteSpec(3, 3, 3, ion_fraction=0.2, seed=78))
    assert set(np.unique(sp.nbf[sp.species == 1])) == {2}
    assert set(np.unique(sp.nbf[sp.species == 0])) == {4}
    assert set(np.unique(sp.nbf[sp.species == 2])) <= {4}
    o = np.nonzero(sp.species == 0)[0]
    for i in o:                                   # each O is followed by its two H
        assert list(sp.species[i + 1:i + 3]) == [1, 1]
        v = [sp.pos[i + k] - sp.pos[i] for k in (1, 2)]
        v = [x - sp.cell * np.rint(x / sp.cell) for x in v]
        assert np.allclose([np.linalg.norm(x) for x in v], 0.96)
        ang = np.degrees(np.arccos(v[0] @ v[1] / (np.linalg.norm(v[0]) * np.linalg.norm(v[1]))))
        assert abs(ang - 104.5) < 1e-9

"""The seeded input generators shared by the oracle and the CUDA path (no
method arithmetic in them): sphere packs keep the recipe they state
(determinism, porosity, clear reservoirs, every pore reachable from the
inlet), and the simple masks keep their layout."""
import numpy as np
from scipy import ndimage

from lbm_inputs import duct_mask, random_mask, sphere_pack, uniform_field


def test_sphere_pack_recipe():
    n, res = 48, 4
    m, info = sphere_pack(n, 4.0, 8.0, 0.35, seed=5, reservoir=res, cache=False)
    assert m.shape == (n, n, n) and m.dtype == np.uint8 and set(np.unique(m)) <= {0, 1}
    # seeded: the same arguments give the same pack, cached or not
    m2, info2 = sphere_pack(n, 4.0, 8.0, 0.35, seed=5, reservoir=res, cache=False)
    np.testing.assert_array_equal(m, m2)
    assert info == info2
    m3, _ = sphere_pack(n, 4.0, 8.0, 0.35, seed=6, reservoir=res, cache=False)
    assert (m3 != m).any()
    # reservoirs are pure pore; the body porosity is the target less the filled
    # isolated pores (a few per cent at most)
    assert not m[:res].any() and not m[n - res:].any()
    body = m[res:n - res]
    assert abs(info["porosity"] - (1.0 - body.mean())) < 1e-12
    assert 0.30 < info["porosity"] <= 0.35 + 1e-3
    assert info["n_spheres"] > 10
    # every pore is 6-connected to the inlet plane
    lab, _ = ndimage.label(m == 0, structure=ndimage.generate_binary_structure(3, 1))
    inlet_labels = set(np.unique(lab[0][lab[0] > 0]))
    assert set(np.unique(lab[lab > 0])) <= inlet_labels


def test_sphere_pack_cache_round_trip(tmp_path, monkeypatch):
    import tempfile

    monkeypatch.setattr(tempfile, "tempdir", str(tmp_path))
    a, ia = sphere_pack((20, 18, 24), 3.0, 5.0, 0.4, seed=9, reservoir=2)
    b, ib = sphere_pack((20, 18, 24), 3.0, 5.0, 0.4, seed=9, reservoir=2)  # from the cache file
    c, ic = sphere_pack((20, 18, 24), 3.0, 5.0, 0.4, seed=9, reservoir=2, cache=False)
    assert a.shape == (24, 18, 20)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    assert ia == ib == ic


def test_simple_masks():
    d = duct_mask(6, 5, 7)
    assert d.shape == (7, 5, 6)
    assert d[:, 0, :].all() and d[:, -1, :].all() and d[:, :, 0].all() and d[:, :, -1].all()
    assert not d[:, 1:-1, 1:-1].any()
    r = random_mask(3, 3, 4, 1.0, seed=1)  # all solid but one pore on each end plane
    assert (r[0] == 0).sum() == 1 and (r[-1] == 0).sum() == 1
    np.testing.assert_array_equal(random_mask(5, 4, 6, 0.3, 2), random_mask(5, 4, 6, 0.3, 2))
    u = uniform_field((4, 5), 3, -2.0, 2.0)
    assert u.shape == (4, 5) and (u >= -2.0).all() and (u < 2.0).all()
    np.testing.assert_array_equal(u, uniform_field((4, 5), 3, -2.0, 2.0))

"""Host logic of the seeded input generators (no GPU): the parameter presets
keep the relations they state, the generators are reproducible, and the
ansatz fields have the structure their docstrings give."""
import math

import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I


def test_table1_regime_splits_alpha4_and_keeps_gamma():
    """Table I in lattice units: the isotropic viscosity a4 is shared as
    2 rho c_s^2 (tau - 1/2) (lattice Boltzmann, c_s^2 = 1/3) + a4' (FD force),
    and gamma1 = a3 - a2, gamma2 = a3 + a2 (Sec. II.A)."""
    a4 = 0.9318
    for split in (0.15, 0.5):
        p, n0 = I.table1_regime(split=split)
        lb = 2.0 * (p["tau"] - 0.5) / 3.0
        assert abs(lb + p["alpha4p"] - a4) < 1e-15
        assert abs(p["alpha4p"] - split * a4) < 1e-15
    p, _ = I.table1_regime(split=0.15, lb_share=0.5)
    assert abs(2.0 * (p["tau"] - 0.5) / 3.0 - 0.5 * a4) < 1e-15
    assert abs(p["gamma1"] - (p["alpha3"] - p["alpha2"])) < 1e-15
    assert abs(p["gamma2"] - (p["alpha3"] + p["alpha2"])) < 1e-15
    # Parodi: alpha6 - alpha5 = gamma2, to the printed digits of Table I
    assert abs((p["alpha6"] - p["alpha5"]) - p["gamma2"]) < 5e-4
    # the Table I nematic is flow aligning: |gamma2 / gamma1| > 1
    assert abs(p["gamma2"] / p["gamma1"]) > 1.0
    assert p["nx"] * p["ny"] * p["nz"] == n0.shape[1]


def test_warmstart_samples_are_metastable_tubes():
    """kappa = pi^2 K q0^2 / (4 W0) < 1 (uniform ground state), pitch in [20, 40],
    radius in [0.3, 0.5] pitch, reproducible from the seed."""
    a = I.warmstart_samples(40, seed=3)
    b = I.warmstart_samples(40, seed=3)
    c = I.warmstart_samples(40, seed=4)
    for (pa, na), (pb, nb) in zip(a, b):
        assert pa == pb and np.array_equal(na, nb)
    assert any(pa["q0"] != pc["q0"] for (pa, _), (pc, _) in zip(a, c))
    for p, n0 in a:
        pitch = 2 * math.pi / p["q0"]
        kappa = math.pi ** 2 * p["K"] * p["q0"] ** 2 / (4 * p["W0"])
        assert 20.0 <= pitch <= 40.0
        assert kappa < 1.0
        assert p["anchoring"] == "none" and p["g"] == (0.0, 0.0, 0.0)
        assert np.allclose(np.linalg.norm(n0, axis=0), 1.0)


def test_place_tubes_keeps_periodic_distance():
    for seed in range(5):
        cs = I.place_tubes(256, 256, 8, 20.0, seed=seed)
        assert len(cs) == 8
        for i in range(8):
            for j in range(i):
                dx = (cs[i][0] - cs[j][0] + 128) % 256 - 128
                dy = (cs[i][1] - cs[j][1] + 128) % 256 - 128
                assert dx * dx + dy * dy >= 40.0 ** 2
    assert I.place_tubes(256, 256, 8, 20.0, seed=1) == I.place_tubes(256, 256, 8, 20.0, seed=1)
    with pytest.raises(RuntimeError):
        I.place_tubes(32, 32, 4, 12.0, seed=0, max_tries=2000)


def test_skyrmion_ansatz_core_and_background():
    """Unit director, -z_hat on the tube axis, z_hat beyond the radius, the same in every layer."""
    nx, ny, nz, R = 32, 32, 4, 8.0
    n = I.skyrmion_tubes(nx, ny, nz, [(16.0, 16.0)], R)
    assert np.allclose(np.linalg.norm(n, axis=0), 1.0)
    site = lambda x, y, z: x + nx * (y + ny * z)
    for z in range(nz):
        assert np.allclose(n[:, site(16, 16, z)], [0.0, 0.0, -1.0])
        assert np.allclose(n[:, site(0, 0, z)], [0.0, 0.0, 1.0])
        assert np.array_equal(n[:, site(5, 9, z)], n[:, site(5, 9, 0)])


def test_multi_tube_channel_and_batched_sweep_shapes():
    p, n0, cs = I.multi_tube_channel(nx=64, ny=64, nz=8, tubes=2, radius=8.0)
    assert n0.shape == (3, 64 * 64 * 8) and len(cs) == 2 and p["dt_fd"] == 16
    chans = I.batched_sweep(count=12, seed=2)
    assert len(chans) == 12
    for p, n0, (cx, cy) in chans:
        assert p["nx"] == p["ny"] in (32, 48, 64, 96) and p["nz"] in (16, 24, 32)
        assert 1e-7 <= p["g"][0] <= 1e-5
        assert p["nz"] <= 2 * math.pi / p["q0"] <= 2 * p["nz"]
        assert (cx, cy) == (p["nx"] / 2, p["ny"] / 2)
        assert n0.shape == (3, p["nx"] * p["ny"] * p["nz"])


def test_generators_are_seeded():
    assert np.array_equal(I.tilted_director(8, 6, 4, seed=7), I.tilted_director(8, 6, 4, seed=7))
    assert not np.array_equal(I.tilted_director(8, 6, 4, seed=7), I.tilted_director(8, 6, 4, seed=8))
    assert np.array_equal(I.random_velocity(8, 6, 4, 1e-3, seed=1), I.random_velocity(8, 6, 4, 1e-3, seed=1))
    assert np.max(np.abs(I.random_velocity(8, 6, 4, 1e-3, seed=1))) <= 1e-3
    w = I.unet_init_params(seed=0)
    assert np.array_equal(w, I.unet_init_params(seed=0))
    n_params = sum(27 * ci * co + co for _, ci, co in I.UNET_CONV_LAYERS) + 16 * 3 + 3
    assert w.size == n_params == 394419


def test_table1_regime_uses_the_printed_table():
    """The preset's material constants are Table I's (tests/golden/table1_mbba.txt):
    the Leslie alpha's (alpha4 split between the LB fluid and alpha4'), the
    one-constant K as the mean of K11, K22, K33, the pitch P and the thickness Lz.
    The lateral size follows the text of Sec. III.A (64), not Table I (56)."""
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table1_mbba.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    p, _ = I.table1_regime(split=0.15)
    for k in ("alpha1", "alpha2", "alpha3", "alpha5", "alpha6"):
        assert p[k] == vals[k], k
    assert abs(p["alpha4p"] + 2.0 * (p["tau"] - 0.5) / 3.0 - vals["alpha4"]) < 1e-15
    assert abs(p["K"] - (vals["K11"] + vals["K22"] + vals["K33"]) / 3.0) < 1e-22
    assert abs(2 * math.pi / p["q0"] - vals["P"]) < 1e-12
    assert p["nz"] == int(vals["Lz"]) and (p["nx"], p["ny"]) == (64, 64)

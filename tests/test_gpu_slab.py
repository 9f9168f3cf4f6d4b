"""A channel split into slabs along y on one GPU (nh_slab_*) against the
single-channel run: the interior rows must be identical bit for bit (the same
kernels on the same operands), for two and three uneven slabs, both stores,
and one slab that is its own neighbour; the single channel itself is checked
against the oracle."""
import math

import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_06610_gb300 import nh as m
    m.load_library()
    return m


def _params(nx, ny, nz, **kw):
    d = dict(I.LESLIE_ALIGN_09, nx=nx, ny=ny, nz=nz, walls_z=True, anchoring="none", shifted=True, tau=0.8,
             g=(1e-5, -3e-6, 0.0), K=0.03, q0=2 * math.pi / 10, W0=0.01, dt_fd=3, alpha1=0.1, alpha4p=0.2)
    d.update(kw)
    return d


@pytest.mark.parametrize("split", [[12], [5, 7], [4, 3, 5]])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_slabs_equal_single_channel_bitwise(nh, oracle_mod, split, prec):
    nx, ny, nz = 18, 12, 7
    params = dict(_params(nx, ny, nz), precision=prec)
    n0 = I.skyrmion_tubes(nx, ny, nz, [(9.0, 6.0)], 4.5)
    steps = 3 * 5 + 1
    one = nh.Channel(params)
    one.set_fd_variant(0)
    one.set_fields(n0)
    one.step(steps)
    n1, u1, _ = one.get_fields()
    f1, F1 = one.get_populations(), one.get_force()
    grp = nh.SlabGroup(params, split)
    grp.set_fields(n0)
    grp.step(7)
    grp.step(steps - 7)
    n2, u2, _ = grp.get_fields()
    assert np.array_equal(n2, n1)
    assert np.array_equal(u2, u1)
    assert np.array_equal(grp.get_populations(), f1)
    assert np.array_equal(grp.get_force(), F1)
    if prec == "fp64" and len(split) == 2:
        O = oracle_mod
        ref = O.OracleSim(O.OracleParams.from_dict(params), n0).step(steps)
        assert np.max(np.abs(n1 - ref.n)) <= 1e-12
        assert np.max(np.abs(u1 - ref.u)) <= 1e-10 * np.max(np.abs(ref.u))
    one.close()
    grp.close()


def test_slabs_reject_unsupported(nh):
    params = _params(12, 8, 6, precision="fp32")
    for extra in (dict(paper_order=True), dict(storage="f16s"), dict(lap_wide=True)):
        grp = nh.SlabGroup(dict(params, **extra), [4, 4])
        with pytest.raises(nh.NHError) as e:
            grp.set_fields(I.uniform_director(12, 8, 6))
        assert e.value.code == nh.NH_EINVAL
        grp.close()
    a = nh.Channel(dict(params, ny=6))
    b = nh.Channel(dict(params, ny=6, tau=0.9))
    for c in (a, b):
        c.set_fields(I.uniform_director(12, 6, 6))
    with pytest.raises(nh.NHError) as e:
        nh.nh_slab_step([a.ctx, b.ctx], 1)
    assert e.value.code == nh.NH_EINVAL

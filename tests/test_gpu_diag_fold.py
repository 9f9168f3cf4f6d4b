"""Diagnostics folded into the LB sweep (nh_set_diag_fold) against the
unfolded reduction on the same state: the LB launch that writes u and rho
also leaves the sums of the populations, max |u| and the non-finite count, and
the diagnostics then read only the director.  Both kernels of the reduction
(x-pairs for even nx, single columns for odd nx and the three-constant
energy), both precisions, graph-replayed blocks and a ragged call, and a
state with a NaN."""
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
    d = dict(I.LESLIE_ALIGN_09, nx=nx, ny=ny, nz=nz, walls_z=True, anchoring="homeotropic", shifted=True, tau=0.8,
             g=(1e-5, -3e-6, 0.0), K=0.03, q0=2 * math.pi / 12, W0=0.01, dt_fd=4)
    d.update(kw)
    return d


def _pair(nh, params, n0, tubes, steps):
    out = []
    for fold in (True, False):
        ch = nh.Channel(params)
        ch.set_diag_fold(fold)
        ch.set_fields(n0)
        ch.set_tubes(tubes)
        for k in steps:
            ch.step(k)
        out.append((ch, ch.diagnostics(allow_unstable=True)))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["pairs", "odd_nx", "frank3"])
@pytest.mark.parametrize("steps", [[8], [8, 3]])
def test_folded_diagnostics_equal_unfolded(nh, prec, case, steps):
    nx = 31 if case == "odd_nx" else 32
    extra = dict(K11=0.02, K22=0.035, K33=0.05) if case == "frank3" else {}
    params = dict(_params(nx, 20, 10, **extra), precision=prec)
    tubes = [(nx / 2, 10.0), (4.0, 3.0)]
    n0 = I.skyrmion_tubes(nx, 20, 10, tubes, 4.5)
    (cf, a), (cu, b) = _pair(nh, params, n0, tubes, steps)
    assert np.array_equal(cf.get_fields()[1], cu.get_fields()[1])  # the same state
    # per-site population sums in the build's precision, grouped differently
    # (warps of the LB launch vs items of the reduction), FP64 across groups
    assert abs(a["mass"] - b["mass"]) <= (1e-12 if prec == "fp64" else 1e-10) * cf.N
    # the director-only reduction sums chunks of 16 layers (the full one 4 or
    # 8): the same per-site terms, partial sums in the build's precision
    # grouped differently -- FP32 rounding of a few tens of terms
    fp64 = prec == "fp64"
    assert abs(a["energy"] - b["energy"]) <= (1e-14 if fp64 else 2e-6) * abs(b["energy"])
    # max |u| from the LB launch's own components against the stored u: one FP32 ulp
    assert abs(a["max_u"] - b["max_u"]) <= (1e-15 if fp64 else 2.5e-7) * b["max_u"]
    assert a["min_norm"] == b["min_norm"] and a["max_norm"] == b["max_norm"]
    assert a["nonfinite"] == b["nonfinite"] == 0
    assert np.max(np.abs(a["centroids"] - b["centroids"])) <= (1e-12 if fp64 else 1e-4)
    cf.close()
    cu.close()


def test_folded_diagnostics_count_a_nan(nh):
    params = dict(_params(16, 12, 8), precision="fp32")
    n0 = I.uniform_director(16, 12, 8)
    res = []
    for fold in (True, False):
        ch = nh.Channel(params)
        ch.set_diag_fold(fold)
        ch.set_fields(n0)
        u = np.zeros((3, ch.N))
        u[0, 37] = np.nan
        ch.restore(n0, u=u, step=0)
        ch.step(1)  # the NaN reaches the populations, u and rho of its neighbourhood
        d = ch.diagnostics(allow_unstable=True)
        res.append(d)
        ch.close()
    assert res[0]["code"] == res[1]["code"] == nh.NH_EUNSTABLE
    assert res[0]["nonfinite"] == res[1]["nonfinite"] >= 1

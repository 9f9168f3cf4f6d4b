"""The reading flags of nh_params on the GPU against the oracle (FP64), and
the bounded host wait (NH_ETIMEOUT).

Each flag changes one choice the paper leaves open (renormalised predictor,
wide second-derivative stencil, N from the corrector's rate, mirrored ghost
stress); every kernel variant that accepts the flag is compared with the
oracle's FD update, force and a short coupled run, element by element.
"""
import math

import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LESLIE = I.LESLIE_ALIGN_09


@pytest.fixture(scope="module")
def nh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_06610_gb300 import nh as m
    m.load_library()
    return m


def _params(nx, ny, nz, **kw):
    d = dict(LESLIE, nx=nx, ny=ny, nz=nz, walls_z=True, anchoring="none", shifted=True, tau=0.8,
             g=(1e-5, -3e-6, 0.0), K=0.03, q0=2 * math.pi / 10, W0=0.02, dt_fd=3, alpha1=0.1, alpha4p=0.2)
    d.update(kw)
    return d


# (flag settings, FD variants that accept them)
FLAGS = [
    (dict(renorm_predictor=True), (1, 0)),
    (dict(lap_wide=True), (0,)),
    (dict(lap_wide=True, anchoring="homeotropic"), (0,)),
    (dict(n_from_rate=True), (0,)),
    (dict(ghost_sigma="mirror"), (1, 0)),
    (dict(ghost_sigma="mirror", anchoring="homeotropic"), (1, 0)),
]


def _cases():
    for flags, variants in FLAGS:
        for fused in variants:
            yield pytest.param(flags, fused, id="-".join(f"{k}={v}" for k, v in flags.items()) + f"-fused{fused}")


@pytest.mark.parametrize("flags,fused", list(_cases()))
@pytest.mark.parametrize("grid", [(13, 9, 7), (33, 17, 17)])
def test_flag_fd_update_and_force_fp64(nh, oracle_mod, flags, fused, grid):
    O = oracle_mod
    params = _params(*grid, **flags)
    n0 = I.random_director(*grid, seed=7)
    u0 = I.random_velocity(*grid, 1e-2, seed=8)
    p = O.OracleParams.from_dict(params)
    F0 = O.force(p, O.stress(p, n0, u0))  # the force at set_fields: no FD update yet
    nref, rate = O.fd_step(p, n0, u0, return_rate=True)
    Fref = O.force(p, O.stress(p, nref, u0, rate if p.n_from_rate else None))
    ch = nh.Channel(dict(params, precision="fp64"))
    ch.set_fd_variant(fused)
    ch.set_fields(n0, u0)
    assert np.max(np.abs(ch.get_force() - F0)) <= 1e-12 * np.max(np.abs(F0))
    ch.fd_update()
    n, _, _ = ch.get_fields()
    assert np.max(np.abs(n - nref)) < 1e-13
    F = ch.get_force()
    assert np.max(np.abs(F - Fref)) <= 1e-12 * np.max(np.abs(Fref))
    ch.close()


@pytest.mark.parametrize("flags,fused", list(_cases()))
def test_flag_coupled_run_fp64(nh, oracle_mod, flags, fused):
    O = oracle_mod
    params = _params(16, 12, 8, **flags)
    n0 = I.skyrmion_tubes(16, 12, 8, [(8.0, 6.0)], 4.5)
    steps = 3 * 4 + 2  # four FD intervals and a ragged tail
    ref = O.OracleSim(O.OracleParams.from_dict(params), n0).step(steps)
    ch = nh.Channel(dict(params, precision="fp64"))
    ch.set_fd_variant(fused)
    ch.set_fields(n0)
    ch.step(steps)
    n, u, _ = ch.get_fields()
    assert np.max(np.abs(n - ref.n)) <= 1e-12
    assert np.max(np.abs(u - ref.u)) <= 1e-10 * np.max(np.abs(ref.u))
    ch.close()


def test_flags_without_fused_variant_are_rejected(nh):
    for flags in (dict(lap_wide=True), dict(n_from_rate=True)):
        ch = nh.Channel(dict(_params(16, 12, 8, **flags), precision="fp32"))
        with pytest.raises(nh.NHError) as e:
            ch.set_fd_variant(1)
        assert e.value.code == nh.NH_EINVAL
        ch.close()


def test_renorm_and_mirror_in_batches_match_single_channels(nh):
    """The batched work-list kernels take the renormalised predictor and the
    mirrored ghost stress like the single-channel kernels (bit for bit)."""
    import torch
    params = [_params(16, 12, 8, renorm_predictor=True, ghost_sigma="mirror", dt_fd=4),
              _params(24, 16, 6, renorm_predictor=True, ghost_sigma="mirror", dt_fd=4, q0=0.4)]
    n0s = [I.skyrmion_tubes(16, 12, 8, [(8.0, 6.0)], 4.5), I.skyrmion_tubes(24, 16, 6, [(12.0, 8.0)], 5.0)]
    single, batch = [], []
    for p, n0 in zip(params, n0s):
        ch = nh.Channel(dict(p, precision="fp64"))
        ch.set_fields(n0)
        ch.step(12)
        single.append(ch.get_fields()[0])
        assert np.max(np.abs(ch.get_fields()[0] - n0)) > 1e-6
        ch.close()
        b = nh.Channel(dict(p, precision="fp64"))
        b.set_fields(n0)
        batch.append(b)
    nh.nh_batch_step([b.ctx for b in batch], 12, torch.cuda.current_stream().cuda_stream)
    for s, b in zip(single, batch):
        assert np.max(np.abs(b.get_fields()[0] - s)) <= 1e-14
        b.close()
    w = [nh.Channel(dict(_params(16, 12, 8, lap_wide=True), precision="fp64")) for _ in range(2)]
    for c in w:
        c.set_fields(n0s[0])
    with pytest.raises(nh.NHError) as e:
        nh.nh_batch_step([c.ctx for c in w], 4, None)
    assert e.value.code == nh.NH_EINVAL


def test_bounded_wait_times_out_and_recovers(nh):
    params, n0, _ = I.multi_tube_channel(dt_fd=16)
    ch = nh.Channel(dict(params, precision="fp64"))
    ch.set_fields(n0)
    ch.get_fields()
    ch.step(160)  # about 0.3 s of FP64 work on the 256x256x64 channel
    ch.set_wait_limit(1e-4)
    with pytest.raises(nh.NHError) as e:
        ch.get_fields()
    assert e.value.code == nh.NH_ETIMEOUT
    with pytest.raises(nh.NHError) as e:
        ch.diagnostics()
    assert e.value.code == nh.NH_ETIMEOUT
    ch.set_wait_limit(0)
    d = ch.diagnostics()  # without a limit the call waits for the steps and the reduction
    n, u, rho = ch.get_fields()
    assert d["nonfinite"] == 0 and np.all(np.isfinite(u))
    ch.set_wait_limit(30.0)
    assert np.array_equal(ch.get_fields()[0], n)  # a generous limit waits normally
    ch.close()

"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: the FP64 build must match the oracle to rel. L2 <= 1e-10 (the
operations are the same; only rounding order differs); the FP32-shifted build
must hold u and n to rel. L2 <= 1e-4 after 1000 steps of the tiny channel.
Row-level checks (LB step, FD update, stress + force) use ragged grids that
span several thread blocks and include both plates.
"""
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


def _oracle_sim(O, params, n0, u0=None):
    return O.OracleSim(O.OracleParams.from_dict(params), n0, u=u0)


def _channel(nh, params, n0, u0=None, **kw):
    ch = nh.Channel(dict(params, **kw))
    ch.set_fields(n0, u0)
    return ch


LESLIE = I.LESLIE_ALIGN_09


def _generic(nx, ny, nz, **kw):
    d = dict(nx=nx, ny=ny, nz=nz, walls_z=True, anchoring="homeotropic", shifted=True, tau=0.8,
             g=(1e-5, -3e-6, 0.0), K=0.03, q0=2 * math.pi / 10, W0=0.0, dt_fd=1, **LESLIE)
    d.update(kw)
    return d


# ------------------------------------------------------------------ row-level parity (FP64)

@pytest.mark.parametrize("shifted", [True, False])
@pytest.mark.parametrize("walls", [True, False])
def test_lb_rows_fp64(nh, oracle_mod, shifted, walls):
    """Pure flow (K = 0): populations, rho and u after 37 steps."""
    O = oracle_mod
    params = _generic(19, 11, 9, K=0.0, q0=0.0, walls_z=walls, shifted=shifted, alpha2=0, alpha3=0,
                      alpha5=0, alpha6=0, gamma2=0.0)
    n0 = I.uniform_director(19, 11, 9)
    u0 = I.random_velocity(19, 11, 9, 1e-3, seed=3)
    ref = _oracle_sim(O, params, n0, u0).step(37)
    ch = _channel(nh, params, n0, u0, precision="fp64")
    ch.step(37)
    n, u, rho = ch.get_fields()
    f = ch.get_populations()
    assert O.rel_l2(u, ref.u) < 1e-12
    if shifted:
        assert O.rel_l2(rho - 1, ref.rho - 1) < 1e-10
    else:
        # the plain store forms rho - 1 ~ 1e-5 as sum f - 1 with f ~ w_i: its
        # rounding is absolute (~1e-16 per addition), which is what the shift cures
        assert np.max(np.abs(rho - ref.rho)) < 1e-14
    assert np.max(np.abs(f - ref.f)) < 1e-13


# ragged; several x-y tiles; one-layer chunks (small grids) and two-layer chunks with a ragged last one
GRIDS = [(13, 9, 7), (40, 20, 20), (33, 17, 17), (100, 64, 23)]


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("anchoring,walls", [("homeotropic", True), ("none", True), ("homeotropic", False)])
def test_stress_force_rows_fp64(nh, oracle_mod, anchoring, walls, grid, fused):
    O = oracle_mod
    params = _generic(*grid, walls_z=walls, anchoring=anchoring, W0=0.02, alpha1=0.1, alpha4p=0.2)
    n0 = I.random_director(*grid, seed=5)
    u0 = I.random_velocity(*grid, 1e-3, seed=6)
    p = O.OracleParams.from_dict(params)
    Fref = O.force(p, O.stress(p, n0, u0))
    ch = nh.Channel(dict(params, precision="fp64"))
    ch.set_fd_variant(fused)
    ch.set_fields(n0, u0)
    F = ch.get_force()
    assert O.rel_l2(F, Fref) < 1e-12
    assert np.max(np.abs(F - Fref)) <= 1e-12 * np.max(np.abs(Fref))  # every site, plate layers included


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("anchoring,walls", [("homeotropic", True), ("none", True), ("homeotropic", False)])
def test_fd_update_rows_fp64(nh, oracle_mod, anchoring, walls, grid, fused):
    O = oracle_mod
    params = _generic(*grid, walls_z=walls, anchoring=anchoring, W0=0.02, dt_fd=3)
    n0 = I.random_director(*grid, seed=7)
    u0 = I.random_velocity(*grid, 1e-2, seed=8)
    p = O.OracleParams.from_dict(params)
    nref = O.fd_step(p, n0, u0)
    Fref = O.force(p, O.stress(p, nref, u0))
    ch = nh.Channel(dict(params, precision="fp64"))
    ch.set_fd_variant(fused)
    ch.set_fields(n0, u0)
    ch.fd_update()
    n, u, _ = ch.get_fields()
    assert O.rel_l2(n, nref) < 1e-13
    assert np.max(np.abs(n - nref)) < 1e-13  # every site, plate layers included
    assert np.max(np.abs(np.linalg.norm(n, axis=0) - 1)) < 1e-14
    assert O.rel_l2(ch.get_force(), Fref) < 1e-12


@pytest.mark.parametrize("anchoring,walls", [("homeotropic", True), ("none", True)])
def test_fd_update_rows_fp32(nh, oracle_mod, anchoring, walls):
    O = oracle_mod
    params = _generic(13, 9, 7, walls_z=walls, anchoring=anchoring, W0=0.02, dt_fd=3)
    n0 = I.random_director(13, 9, 7, seed=7)
    u0 = I.random_velocity(13, 9, 7, 1e-2, seed=8)
    p = O.OracleParams.from_dict(params)
    nref = O.fd_step(p, n0, u0)
    Fref = O.force(p, O.stress(p, nref, u0))
    ch = _channel(nh, params, n0, u0, precision="fp32")
    ch.fd_update()
    n, _, _ = ch.get_fields()
    assert O.rel_l2(n, nref) < 1e-6
    assert O.rel_l2(ch.get_force(), Fref) < 1e-5


# ------------------------------------------------------------------ full hybrid runs

def test_tiny_channel_fp64_200_steps(nh, oracle_mod):
    """32x32x16 nematic channel, 200 steps at dt_FD = 1: FP64 GPU vs oracle <= 1e-10."""
    O = oracle_mod
    params, n0 = I.tiny_channel()
    ref = _oracle_sim(O, params, n0).step(200)
    ch = _channel(nh, params, n0, precision="fp64")
    ch.step(200)
    n, u, rho = ch.get_fields()
    assert O.rel_l2(u, ref.u) <= 1e-10
    assert O.rel_l2(n, ref.n) <= 1e-10
    d = ch.diagnostics()
    assert abs(d["mass"] - ref.mass()) <= 1e-12 * ch.N
    assert abs(d["energy"] - ref.energy()) <= 1e-10 * abs(ref.energy())


@pytest.fixture(scope="module")
def tiny_ref_1000(oracle_mod):
    params, n0 = I.tiny_channel()
    return params, n0, _oracle_sim(oracle_mod, params, n0).step(1000)


def test_tiny_channel_fp32_shifted_1000_steps(nh, oracle_mod, tiny_ref_1000):
    """FP32-shifted holds u and n to rel. L2 <= 1e-4 after 1000 steps."""
    O = oracle_mod
    params, n0, ref = tiny_ref_1000
    ch = _channel(nh, params, n0, precision="fp32", storage="f32", shifted=True)
    ch.step(1000)
    n, u, rho = ch.get_fields()
    eu, en = O.rel_l2(u, ref.u), O.rel_l2(n, ref.n)
    print(f"FP32-shifted 1000 steps: rel L2 u {eu:.3e} n {en:.3e} eps {O.eps_paper(u, ref.u):.3e}")
    assert eu <= 1e-4
    assert en <= 1e-4


def test_tiny_channel_fp32_unshifted_reported(nh, oracle_mod, tiny_ref_1000):
    """The plain FP32 store is reported beside the shifted one (precision loss at low velocity)."""
    O = oracle_mod
    params, n0, ref = tiny_ref_1000
    errs = {}
    for shifted in (True, False):
        ch = _channel(nh, params, n0, precision="fp32", storage="f32", shifted=shifted)
        ch.step(1000)
        n, u, _ = ch.get_fields()
        errs[shifted] = (O.rel_l2(u, ref.u), O.rel_l2(n, ref.n))
    print(f"FP32 rel L2(u): shifted {errs[True][0]:.3e}  unshifted {errs[False][0]:.3e}")
    assert errs[True][0] < errs[False][0]
    assert np.isfinite(errs[False][0])


@pytest.mark.parametrize("storage,tol", [("f16s", 2e-2), ("bf16s", 2e-1)])
def test_16bit_stores_reported(nh, oracle_mod, tiny_ref_1000, storage, tol):
    O = oracle_mod
    params, n0, ref = tiny_ref_1000
    ch = _channel(nh, params, n0, precision="fp32", storage=storage, shifted=True)
    ch.step(1000)
    n, u, _ = ch.get_fields()
    eu, en = O.rel_l2(u, ref.u), O.rel_l2(n, ref.n)
    print(f"{storage}: rel L2 u {eu:.3e} n {en:.3e}")
    assert eu <= tol
    assert en <= tol


def test_ragged_dtfd_fp64(nh, oracle_mod):
    """dt_FD = 3 on a ragged 13x7x5 grid, 31 steps (graph blocks + a ragged tail)."""
    O = oracle_mod
    params = _generic(13, 7, 5, dt_fd=3, K=0.02, W0=0.01, anchoring="none")
    n0 = I.skyrmion_tubes(13, 7, 5, [(6.0, 3.0)], 3.0)
    ref = _oracle_sim(O, params, n0).step(31)
    ch = _channel(nh, params, n0, precision="fp64")
    ch.step(10)
    ch.step(21)
    n, u, _ = ch.get_fields()
    assert O.rel_l2(u, ref.u) <= 1e-10
    assert O.rel_l2(n, ref.n) <= 1e-10


def test_graphs_match_direct_launches_bitwise(nh):
    params = _generic(16, 12, 8, dt_fd=4)
    n0 = I.tilted_director(16, 12, 8, amplitude=0.2, seed=2)
    out = []
    for graphs in (True, False):
        ch = _channel(nh, params, n0, precision="fp32")
        ch.set_graphs(graphs)
        ch.step(40)
        out.append(ch.get_fields())
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_checkpoint_resume_bit_exact(nh, prec):
    params = _generic(16, 10, 8, dt_fd=4)
    n0 = I.skyrmion_tubes(16, 10, 8, [(8.0, 5.0)], 4.0)
    a = _channel(nh, params, n0, precision=prec)
    a.step(22)
    n, u, rho = a.get_fields()
    f = a.get_populations()
    F = a.get_force()
    a.step(13)
    end_a = a.get_fields()
    b = _channel(nh, params, n0, precision=prec)
    b.set_populations(f)
    b.restore(n, F=F, u=u, rho=rho, step=22)
    b.step(13)
    end_b = b.get_fields()
    for x, y in zip(end_a, end_b):
        assert np.array_equal(x, y)


def test_diagnostics_match_oracle(nh, oracle_mod):
    O = oracle_mod
    params = _generic(40, 36, 6, dt_fd=2, K=0.02, q0=2 * math.pi / 12)
    n0 = I.skyrmion_tubes(40, 36, 6, [(10.0, 9.0), (30.0, 27.0)], 8.0)
    ref = _oracle_sim(O, params, n0).step(10)
    ch = _channel(nh, params, n0, precision="fp64")
    ch.set_tubes([(10.0, 9.0), (30.0, 27.0)])
    ch.step(10)
    d = ch.diagnostics()
    assert abs(d["mass"] - ref.mass()) <= 1e-12 * ch.N
    assert abs(d["energy"] - ref.energy()) <= 1e-11 * abs(ref.energy())
    cref = O.centroids(O.OracleParams.from_dict(params), ref.n, [(10.0, 9.0), (30.0, 27.0)])
    assert np.max(np.abs(d["centroids"] - cref)) < 1e-9
    assert d["nonfinite"] == 0
    assert abs(d["max_norm"] - 1) < 1e-14 and abs(d["min_norm"] - 1) < 1e-14


@pytest.mark.parametrize("nx", [35, 36])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("walls,anchoring", [(True, "homeotropic"), (True, "none"), (False, "homeotropic")])
def test_diagnostics_match_oracle_variants(nh, oracle_mod, prec, walls, anchoring, nx):
    """Several layer chunks with a ragged last one (nz = 37), a column count
    that is not a multiple of the warp size, both wall anchorings and periodic
    z, bulk W0; odd nx takes the one-column diagnostics kernel, even nx the
    two-column one; FP64 to rounding, FP32 to its per-site precision."""
    O = oracle_mod
    ny, nz = 33, 37
    tubes = [(9.0, 8.0), (26.0, 24.0)]
    params = _generic(nx, ny, nz, dt_fd=2, K=0.02, q0=2 * math.pi / 12, W0=0.002, walls_z=walls,
                      anchoring=anchoring)
    n0 = I.skyrmion_tubes(nx, ny, nz, tubes, 7.0)
    ref = _oracle_sim(O, params, n0).step(6)
    ch = _channel(nh, params, n0, precision=prec)
    ch.set_tubes(tubes)
    ch.step(6)
    d = ch.diagnostics()
    cref = O.centroids(O.OracleParams.from_dict(params), ref.n, tubes)
    if prec == "fp64":
        assert abs(d["mass"] - ref.mass()) <= 1e-12 * ch.N
        assert abs(d["energy"] - ref.energy()) <= 1e-11 * abs(ref.energy())
        assert np.max(np.abs(d["centroids"] - cref)) < 1e-9
    else:
        assert abs(d["mass"] - ref.mass()) <= 1e-5 * ch.N
        assert abs(d["energy"] - ref.energy()) <= 1e-4 * abs(ref.energy())
        assert np.max(np.abs(d["centroids"] - cref)) < 1e-3
    assert d["nonfinite"] == 0


def test_mass_conserved_fp32(nh):
    params, n0 = I.tiny_channel()
    ch = _channel(nh, params, n0, precision="fp32")
    m0 = ch.diagnostics()["mass"]
    ch.step(500)
    m1 = ch.diagnostics()["mass"]
    assert abs(m1 - m0) <= 1e-6 * ch.N


def test_empty_step_and_errors(nh):
    params = _generic(8, 8, 8)
    ch = nh.Channel(dict(params, precision="fp32"))
    with pytest.raises(nh.NHError):
        ch.step(5)               # fields not set
    ch.set_fields(I.uniform_director(8, 8, 8))
    ch.step(0)                   # no-op
    with pytest.raises(nh.NHError):
        ch.step(-1)
    n, u, rho = ch.get_fields()
    assert np.all(np.isfinite(n))


def test_nonfinite_detected(nh):
    params = _generic(8, 8, 8)
    ch = nh.Channel(dict(params, precision="fp32"))
    n0 = I.uniform_director(8, 8, 8)
    ch.set_fields(n0)
    u = np.zeros((3, ch.N))
    u[0, 17] = np.nan
    ch.restore(n0, u=u, step=0)
    d = ch.diagnostics(allow_unstable=True)
    assert d["nonfinite"] >= 1 and d["code"] == nh.NH_EUNSTABLE


# ------------------------------------------------------------------ full-size checks (bench configuration)

@pytest.mark.parametrize("shape", ["autotuned", 4])
def test_full_size_multi_tube_one_lb_step(nh, oracle_mod, shape):
    """256x256x64, FP32-shifted, dt_FD = 16, in the launch configuration the
    bench times (autotuned) and with the four-site shape: after 16 steps, one
    more LB step on the GPU equals the oracle's LB step applied to the GPU's
    own state."""
    O = oracle_mod
    params, n0, centres = I.multi_tube_channel()
    ch = _channel(nh, params, n0, precision="fp32")
    if shape == "autotuned":
        ch.autotune()
    else:
        ch.set_lb_variant(shape)
    ch.step(16)
    f = ch.get_populations()
    F = ch.get_force()
    ch.step(1)
    f1 = ch.get_populations()
    _, u1, rho1 = ch.get_fields()
    fo, rho_o, u_o = O.lb_step(O.OracleParams.from_dict(params), f, F)
    assert O.rel_l2(f1, fo) < 1e-5
    assert O.rel_l2(u1, u_o) < 1e-5
    d = ch.diagnostics()
    assert abs(d["mass"] - ch.N) < 1e-6 * ch.N


def test_full_size_multi_tube_fd_update(nh, oracle_mod):
    O = oracle_mod
    params, n0, centres = I.multi_tube_channel()
    u0 = I.random_velocity(256, 256, 64, 1e-4, seed=9)
    ch = _channel(nh, params, n0, u0, precision="fp32")
    ch.fd_update()
    n, _, _ = ch.get_fields()
    p = O.OracleParams.from_dict(params)
    nref = O.fd_step(p, n0, u0)
    assert O.rel_l2(n, nref) < 1e-6
    # the force of the fused stress + divergence kernel on the updated director
    Fref = O.force(p, O.stress(p, nref, u0))
    assert O.rel_l2(ch.get_force(), Fref) < 1e-5


@pytest.mark.parametrize("nx", [16, 13])
def test_lb_variants_agree_and_autotune_keeps_state(nh, oracle_mod, nx):
    """Every LB launch shape gives the oracle's result; the autotuner picks a
    valid shape without advancing the state."""
    O = oracle_mod
    params = _generic(nx, 6, 5, dt_fd=2)
    n0 = I.tilted_director(nx, 6, 5, amplitude=0.3, seed=4)
    ref = _oracle_sim(O, params, n0).step(9)
    variants = [v for v, spt in enumerate((2, 1, 2, 1, 4, 4)) if nx % spt == 0]
    for v in variants:
        ch = _channel(nh, params, n0, precision="fp64")
        ch.set_lb_variant(v)
        ch.step(9)
        n, u, _ = ch.get_fields()
        assert O.rel_l2(u, ref.u) <= 1e-12, v
        assert O.rel_l2(n, ref.n) <= 1e-12, v
    if nx % 2:
        ch = nh.Channel(dict(params, precision="fp64"))
        with pytest.raises(nh.NHError):
            ch.set_lb_variant(0)
    ch = _channel(nh, params, n0, precision="fp64")
    ch.step(4)
    before = ch.get_populations()
    chosen = ch.autotune()
    assert chosen in variants
    assert np.array_equal(before, ch.get_populations())
    ch.step(5)
    n, u, _ = ch.get_fields()
    assert O.rel_l2(u, ref.u) <= 1e-12


def test_timing_segments_count_every_launch(nh):
    params = _generic(16, 12, 8, dt_fd=4)
    n0 = I.tilted_director(16, 12, 8, amplitude=0.2, seed=2)
    for fused in (0, 1):
        ch = _channel(nh, params, n0, precision="fp32")
        ch.set_fd_variant(fused)
        ch.set_timing(1)
        ch.step(10)
        t = ch.timing()
        assert t["lb"][0] == 10 and t["fd_predict"][0] == 2 and t["stress"][0] == 2
        # the fused variant runs predictor+corrector and stress+force as two kernels
        assert t["fd_correct"][0] == (0 if fused else 2) and t["force"][0] == (0 if fused else 2)
        assert all(v[1] > 0 for k, v in t.items() if v[0] > 0)
    ch.set_timing(2)
    ch.step(8)
    t = ch.timing()
    assert t["lb"][0] == 8 and t["fd_predict"][0] == 0
    ch.set_timing(0)
    ch.step(4)
    assert ch.timing()["lb"][0] == 0


# ------------------------------------------------------------------ batched channels (one launch per pass)

def _batch_channels(nh, prec, specs, dt_fd=3):
    chans, refs = [], []
    for k, (nx, ny, nz) in enumerate(specs):
        params = _generic(nx, ny, nz, dt_fd=dt_fd, g=(10 ** (-6 + 0.3 * k), 0.0, 0.0), q0=2 * math.pi / (nz + k))
        n0 = I.skyrmion_tubes(nx, ny, nz, [(nx / 2, ny / 2)], nx / 4)
        chans.append(_channel(nh, params, n0, precision=prec))
        refs.append((params, n0))
    return chans, refs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_oracle_and_single_channels(nh, oracle_mod, prec):
    O = oracle_mod
    specs = [(16, 12, 6), (13, 9, 5), (24, 8, 7), (10, 10, 4), (32, 6, 3)]
    batch, refs = _batch_channels(nh, prec, specs)
    nh.batch_step(batch, 7)
    nh.batch_step(batch, 11)
    singles, _ = _batch_channels(nh, prec, specs)
    for ch in singles:
        ch.step(18)
    tol = 1e-10 if prec == "fp64" else 1e-5
    for chb, chs, (params, n0) in zip(batch, singles, refs):
        nb, ub, _ = chb.get_fields()
        ns, us, _ = chs.get_fields()
        assert O.rel_l2(ub, us) <= (1e-13 if prec == "fp64" else 1e-6)
        assert O.rel_l2(nb, ns) <= (1e-13 if prec == "fp64" else 1e-6)
        if prec == "fp64":
            ref = _oracle_sim(O, params, n0).step(18)
            assert O.rel_l2(ub, ref.u) <= tol
            assert O.rel_l2(nb, ref.n) <= tol


def test_batch_graphs_bitwise_and_autotune(nh):
    specs = [(16, 12, 6), (20, 10, 8), (8, 8, 4)]
    out = []
    for graphs in (True, False):
        chans, _ = _batch_channels(nh, "fp32", specs, dt_fd=4)
        chans[0].set_graphs(graphs)
        nh.batch_step(chans, 12)
        out.append([c.get_fields()[1] for c in chans])
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    chans, _ = _batch_channels(nh, "fp32", specs, dt_fd=4)
    nh.batch_step(chans, 4)
    before = [c.get_populations() for c in chans]
    v = nh.batch_autotune(chans)
    spt = (2, 1, 2, 1, 4, 4)  # sites per thread of launch shapes 0..5
    assert 0 <= v < len(spt) and all(nx % spt[v] == 0 for nx, _, _ in specs)
    for c, f in zip(chans, before):
        assert np.array_equal(c.get_populations(), f)


def test_batch_rejects_mismatched_channels(nh):
    a, _ = _batch_channels(nh, "fp32", [(8, 8, 4)], dt_fd=2)
    b, _ = _batch_channels(nh, "fp32", [(8, 8, 4)], dt_fd=3)
    with pytest.raises(nh.NHError):
        nh.batch_step(a + b, 2)
    with pytest.raises(nh.NHError):
        nh.batch_step(a + a, 2)
    c, _ = _batch_channels(nh, "fp32", [(8, 8, 4)], dt_fd=2)
    c[0].step(1)
    with pytest.raises(nh.NHError):
        nh.batch_step(a + c, 2)


def test_batch_of_65_channels_spans_two_launch_groups(nh):
    specs = [(8, 6, 3)] * 65
    chans, _ = _batch_channels(nh, "fp32", [(8, 6, 3)], dt_fd=2)
    params = _generic(8, 6, 3, dt_fd=2)
    n0 = I.skyrmion_tubes(8, 6, 3, [(4.0, 3.0)], 2.0)
    chans = [_channel(nh, params, n0, precision="fp32") for _ in specs]
    nh.batch_step(chans, 6)
    single = _channel(nh, params, n0, precision="fp32")
    single.step(6)
    ref = single.get_fields()[1]
    for c in (chans[0], chans[63], chans[64]):
        assert np.allclose(c.get_fields()[1], ref, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("anchoring", ["homeotropic", "none"])
def test_relax_matches_oracle_gradient_flow(nh, oracle_mod, anchoring):
    """Director-only relaxation = predictor-corrector at u = 0 (FP64 <= 1e-12)."""
    O = oracle_mod
    params = _generic(16, 12, 8, dt_fd=5, K=0.01, W0=0.002, anchoring=anchoring)
    n0 = I.skyrmion_tubes(16, 12, 8, [(8.0, 6.0)], 5.0)
    p = O.OracleParams.from_dict(params)
    n = n0.copy()
    u = np.zeros_like(n0)
    for _ in range(12):
        n = O.fd_step(p, n, u)
    for fused in (0, 1):
        chv = nh.Channel(dict(params, precision="fp64"))
        chv.set_fd_variant(fused)
        chv.set_fields(n0)
        chv.relax(11)
        chv.relax(1)
        assert O.rel_l2(chv.get_fields()[0], n) < 1e-12
    ch = _channel(nh, params, n0, I.random_velocity(16, 12, 8, 1e-3, seed=1), precision="fp64")
    ch.relax(12)
    ng, ug, _ = ch.get_fields()
    assert O.rel_l2(ng, n) < 1e-12
    assert np.max(np.abs(ug)) == 0.0
    chans = [_channel(nh, params, n0, precision="fp64") for _ in range(3)]
    nh.batch_relax(chans, 12)
    for c in chans:
        assert O.rel_l2(c.get_fields()[0], n) < 1e-12


def test_director_change_tracks_relaxation(nh):
    params = _generic(16, 12, 8, dt_fd=5, K=0.01)
    n0 = I.skyrmion_tubes(16, 12, 8, [(8.0, 6.0)], 5.0)
    ch = _channel(nh, params, n0, precision="fp32")
    assert math.isinf(ch.director_change())
    assert ch.director_change() == 0.0
    ch.relax(20)
    d = ch.director_change()
    n1 = ch.get_fields()[0]
    assert 0.0 < d <= np.max(np.linalg.norm(n1 - n0, axis=0)) + 1e-6
    assert abs(d - np.max(np.linalg.norm(n1 - n0, axis=0))) < 1e-5
    assert ch.director_change() == 0.0


def test_symmetrize_c4_projection(nh):
    """A tube centred on (nx/2, ny/2) is C4-symmetric and unchanged (to FP
    rounding); the projection of an off-axis field is idempotent."""
    params = _generic(24, 24, 6, dt_fd=2)
    centred = I.skyrmion_tubes(24, 24, 6, [(12, 12)], 7.0)
    ch = _channel(nh, params, centred, precision="fp64")
    ch.symmetrize_c4()
    assert np.max(np.abs(ch.get_fields()[0] - centred)) < 1e-12
    off = I.skyrmion_tubes(24, 24, 6, [(13.5, 11.0)], 7.0)
    ch = _channel(nh, params, off, precision="fp64")
    ch.symmetrize_c4()
    once = ch.get_fields()[0]
    ch.symmetrize_c4()
    assert np.max(np.abs(ch.get_fields()[0] - once)) < 1e-12
    n3 = once.reshape(3, 6, 24, 24)
    # rotate the field by 90 degrees about (12, 12): n'(x, y) = R n(R^-1 (x, y))
    x, y = np.meshgrid(np.arange(24), np.arange(24), indexing="xy")
    xs, ys = (12 + (y - 12)) % 24, (12 - (x - 12)) % 24
    rot = np.stack([-n3[1][:, ys, xs], n3[0][:, ys, xs], n3[2][:, ys, xs]])
    assert np.max(np.abs(rot - n3)) < 1e-12


# ------------------------------------------------------------------ paper ordering of the hybrid loop (Sec. II.D)

@pytest.mark.parametrize("dt_fd", [1, 3])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_paper_order_matches_oracle(nh, oracle_mod, dt_fd, storage):
    """paper_order = 1: the FD update between the macroscopic fields and the
    collision; populations, n and u against the oracle's literal loop."""
    O = oracle_mod
    params = _generic(13, 9, 7, dt_fd=dt_fd, alpha4p=0.02, W0=0.002, paper_order=True)
    n0 = I.skyrmion_tubes(13, 9, 7, [(6.5, 4.5)], 3.5)
    steps = 3 * dt_fd + 2  # ends mid-interval when dt_fd > 1
    ref = _oracle_sim(O, params, n0).step(steps)
    prec = "fp64" if storage == "f64" else "fp32"
    ch = _channel(nh, params, n0, precision=prec, storage=storage)
    ch.step(steps)
    n, u, rho = ch.get_fields()
    f = ch.get_populations()
    tol = 1e-12 if storage == "f64" else 2e-5
    assert O.rel_l2(n, ref.n) <= tol
    assert O.rel_l2(u, ref.u) <= (1e-10 if storage == "f64" else 1e-4)
    assert np.max(np.abs(f - ref.f)) <= (1e-14 if storage == "f64" else 1e-6)
    if storage == "f64":
        # the default order gives a different trajectory
        other = _channel(nh, dict(params, paper_order=False), n0, precision=prec, storage=storage)
        other.step(steps)
        assert O.rel_l2(other.get_fields()[1], ref.u) > 1e-8


def test_paper_order_graphs_bitwise_and_batch_rejected(nh):
    params = _generic(16, 12, 8, dt_fd=4, paper_order=True)
    n0 = I.skyrmion_tubes(16, 12, 8, [(8.0, 6.0)], 4.0)
    out = []
    for graphs in (False, True):
        ch = _channel(nh, params, n0, precision="fp32")
        ch.set_graphs(graphs)
        ch.step(4 * 5 + 3)
        out.append(ch.get_fields())
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    chans = [_channel(nh, params, n0, precision="fp32") for _ in range(2)]
    with pytest.raises(nh.NHError):
        nh.batch_step(chans, 4)


# ------------------------------------------------------------------ three-constant Frank energy (Eq. free-energy-eq)

FRANK3 = dict(K=0.03, K11=0.045, K22=0.015, K33=0.06)


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("anchoring,walls", [("homeotropic", True), ("none", True), ("homeotropic", False)])
def test_frank3_fd_update_and_force_fp64(nh, oracle_mod, anchoring, walls, grid):
    O = oracle_mod
    params = _generic(*grid, walls_z=walls, anchoring=anchoring, W0=0.02, dt_fd=3, alpha1=0.1, alpha4p=0.2,
                      **FRANK3)
    n0 = I.random_director(*grid, seed=9)
    u0 = I.random_velocity(*grid, 1e-2, seed=10)
    p = O.OracleParams.from_dict(params)
    assert p.frank3
    F0 = O.force(p, O.stress(p, n0, u0))
    nref = O.fd_step(p, n0, u0)
    Fref = O.force(p, O.stress(p, nref, u0))
    ch = nh.Channel(dict(params, precision="fp64"))
    ch.set_fields(n0, u0)
    assert O.rel_l2(ch.get_force(), F0) < 1e-12
    ch.fd_update()
    n, _, _ = ch.get_fields()
    assert O.rel_l2(n, nref) < 1e-13
    assert O.rel_l2(ch.get_force(), Fref) < 1e-12
    # the correction matters: the one-constant update differs
    p1 = O.OracleParams.from_dict({k: v for k, v in params.items() if k not in ("K11", "K22", "K33")})
    assert O.rel_l2(O.fd_step(p1, n0, u0), nref) > 1e-6


def test_frank3_channel_and_energy(nh, oracle_mod):
    """Coupled run with a tube, FP64 to 1e-10 and FP32 to 1e-5, and the
    diagnostics' three-constant energy against the oracle's."""
    O = oracle_mod
    params = _generic(24, 20, 10, dt_fd=2, K=0.02, K11=0.03, K22=0.01, K33=0.04, q0=2 * math.pi / 12,
                      W0=0.002, walls_z=True, anchoring="none")
    n0 = I.skyrmion_tubes(24, 20, 10, [(12.0, 10.0)], 5.0)
    ref = _oracle_sim(O, params, n0).step(30)
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-5)):
        ch = _channel(nh, params, n0, precision=prec)
        ch.set_tubes([(12.0, 10.0)])
        ch.step(30)
        n, u, _ = ch.get_fields()
        assert O.rel_l2(n, ref.n) <= tol
        assert O.rel_l2(u, ref.u) <= (tol if prec == "fp64" else 1e-4)
        d = ch.diagnostics()
        assert abs(d["energy"] - ref.energy()) <= (1e-11 if prec == "fp64" else 1e-5) * abs(ref.energy())


def test_frank3_rejects_fused_and_runs_in_batches(nh, oracle_mod):
    """The three-constant energy runs on the per-site FD kernels, also in a
    batch that mixes it with one-constant channels (the per-site work-list
    kernels with the P stages; the one-constant channels skip them): equal to
    the same channels stepped alone, and to the oracle."""
    O = oracle_mod
    params = _generic(16, 12, 8, dt_fd=2, **FRANK3)
    n0 = I.skyrmion_tubes(16, 12, 8, [(8.0, 6.0)], 4.0)
    ch = _channel(nh, params, n0, precision="fp32")
    with pytest.raises(nh.NHError):
        ch.set_fd_variant(1)
    with pytest.raises(nh.NHError):
        nh.Channel(dict(params, K22=0.0, precision="fp32"))
    specs = [params, _generic(12, 10, 6, dt_fd=2), dict(params, nx=14, q0=0.5)]
    starts = [I.skyrmion_tubes(p["nx"], p["ny"], p["nz"], [(p["nx"] / 2, p["ny"] / 2)], 3.5) for p in specs]
    batch = [_channel(nh, p, s, precision="fp64") for p, s in zip(specs, starts)]
    nh.batch_step(batch, 6)
    nh.batch_step(batch, 3)
    for chb, p, s in zip(batch, specs, starts):
        one = _channel(nh, p, s, precision="fp64")
        one.set_fd_variant(0)  # the per-site kernels, as in a batch with a three-constant channel
        one.step(9)
        nb, ub, _ = chb.get_fields()
        ns, us, _ = one.get_fields()
        assert np.max(np.abs(nb - ns)) <= 1e-15 and np.max(np.abs(ub - us)) <= 1e-15 * max(np.max(np.abs(us)), 1e-30)
        ref = _oracle_sim(O, p, s).step(9)
        assert np.max(np.abs(nb - ref.n)) <= 1e-12
    relax = [_channel(nh, p, s, precision="fp64") for p, s in zip(specs, starts)]
    nh.batch_relax(relax, 5)
    for chr_, p, s in zip(relax, specs, starts):
        one = _channel(nh, p, s, precision="fp64")
        one.set_fd_variant(0)
        one.relax(5)
        assert np.max(np.abs(chr_.get_fields()[0] - one.get_fields()[0])) <= 1e-15


# ------------------------------------------------------------------ obstacles (solid nodes, Sec. II.B)

def _sphere_mask(nx, ny, nz, c, r):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = (((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) <= r * r)
    v = np.stack([x - c[0], y - c[1], z - c[2]]).astype(float)
    v[:, np.linalg.norm(v, axis=0) == 0] = np.array([0, 0, 1.0])[:, None]
    return m.astype(np.uint8).reshape(-1), (v / np.linalg.norm(v, axis=0)).reshape(3, -1)


@pytest.mark.parametrize("frank3,fused", [(False, 1), (False, 0), (True, 0)])
def test_obstacle_channel_matches_oracle(nh, oracle_mod, frank3, fused):
    """Obstacles on the fused 2.5D FD kernels and on the per-site ones (the
    three-constant energy only on the latter)."""
    O = oracle_mod
    nx, ny, nz = 20, 14, 10
    mask, normals = _sphere_mask(nx, ny, nz, (10.0, 7.0, 5.0), 3.2)
    extra = dict(K11=0.045, K22=0.015, K33=0.06) if frank3 else {}
    params = _generic(nx, ny, nz, dt_fd=2, K=0.03, q0=2 * math.pi / 10, W0=0.002, g=(1e-4, 2e-5, 0.0),
                      **extra)
    n0 = I.tilted_director(nx, ny, nz, amplitude=0.3, seed=3)
    n0[:, mask == 1] = normals[:, mask == 1]
    ref = O.OracleSim(O.OracleParams.from_dict(dict(params, solid=mask)), n0).step(21)
    fl = mask == 0
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-5)):
        ch = nh.Channel(dict(params, precision=prec))
        ch.set_solid(mask)
        ch.set_fd_variant(fused)
        ch.set_fields(n0)
        n_loaded = ch.get_fields()[0]  # nh_set_fields normalises the director
        ch.step(21)
        n, u, rho = ch.get_fields()
        assert O.rel_l2(n, ref.n) <= tol
        assert O.rel_l2(u[:, fl], ref.u[:, fl]) <= (1e-10 if prec == "fp64" else 1e-4)
        assert np.array_equal(n[:, ~fl], n_loaded[:, ~fl])  # anchored directors are held
        assert np.max(np.abs(u[:, ~fl])) == 0.0
        if prec == "fp64":
            f = ch.get_populations()
            assert np.max(np.abs(f - ref.f)) < 1e-14
        d = ch.diagnostics()
        assert abs(d["mass"] - ref.mass()) <= (1e-12 if prec == "fp64" else 1e-5) * ch.N
        assert abs(d["energy"] - ref.energy()) <= (1e-11 if prec == "fp64" else 1e-5) * abs(ref.energy())


def test_obstacle_plates_equal_rotated_walls_gpu(nh):
    """GPU: mask plates normal to y in a periodic box = the z-plate channel in
    rotated axes (cyclic permutation of sites and components), FP64."""
    nxA, nyA, nzA = 16, 12, 9
    pA = _generic(nxA, nyA, nzA, dt_fd=3, K=0.03, q0=2 * math.pi / 9, W0=0.0, g=(2e-5, -1e-5, 3e-6))
    n0A = I.skyrmion_tubes(nxA, nyA, nzA, [(8.0, 6.0)], 3.5)

    def to_B(a, vector):
        if vector:
            a = np.asarray(a).reshape(3, nzA, nyA, nxA)
            return np.stack([to_B(a[k], False) for k in (1, 2, 0)])
        out = np.zeros((nxA, nzA + 2, nyA))
        out[:, 1:-1, :] = np.transpose(np.asarray(a).reshape(nzA, nyA, nxA), (2, 0, 1))
        return out

    solid = np.zeros((nxA, nzA + 2, nyA), np.uint8)
    solid[:, 0, :] = 1
    solid[:, -1, :] = 1
    n0B = to_B(n0A, True)
    n0B[1][solid == 1] = 1.0
    pB = dict(pA, nx=nyA, ny=nzA + 2, nz=nxA, walls_z=False, g=(pA["g"][1], pA["g"][2], pA["g"][0]))
    a = _channel(nh, pA, n0A, precision="fp64")
    a.step(13)
    b = nh.Channel(dict(pB, precision="fp64"))
    b.set_solid(solid.reshape(-1))
    b.set_fields(n0B.reshape(3, -1))
    b.step(13)
    na, ua, _ = a.get_fields()
    nb, ub, _ = b.get_fields()
    fl = solid.reshape(-1) == 0
    assert np.max(np.abs(nb[:, fl] - to_B(na, True).reshape(3, -1)[:, fl])) < 1e-13
    assert np.max(np.abs(ub[:, fl] - to_B(ua, True).reshape(3, -1)[:, fl])) < 1e-13 * np.max(np.abs(ua))
    assert abs(a.diagnostics()["energy"] - b.diagnostics()["energy"]) < 1e-12 * abs(a.diagnostics()["energy"])


@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_obstacles_run_in_batches(nh, oracle_mod, storage, fused):
    """A batch with obstacles in some channels runs one site per thread in the
    LB sweep (channels without a mask included) and the fused or the per-site
    FD kernels: equal to the channels stepped alone (populations included),
    and to the oracle in FP64."""
    O = oracle_mod
    prec = "fp64" if storage == "f64" else "fp32"
    dims = [(16, 12, 8), (12, 10, 6), (18, 8, 7)]
    masks = [_sphere_mask(16, 12, 8, (8.0, 6.0, 4.0), 2.5), None, _sphere_mask(18, 8, 7, (3.0, 4.0, 3.0), 2.0)]
    def make(fd_variant=None):
        out = []
        for (nx, ny, nz), m in zip(dims, masks):
            params = dict(_generic(nx, ny, nz, dt_fd=2), precision=prec, storage=storage)
            ch = nh.Channel(params)
            n0 = I.uniform_director(nx, ny, nz)
            if m is not None:
                mask, normal = m
                ch.set_solid(mask)
                n0 = np.where(mask[None] == 1, normal, n0)
            if fd_variant is not None:
                ch.set_fd_variant(fd_variant)
            ch.set_fields(n0)
            out.append((ch, params, n0))
        return out
    batch = make(fd_variant=fused)
    nh.batch_step([c for c, _, _ in batch], 5)
    singles = make(fd_variant=fused)
    # the work-list kernels evaluate the same arithmetic as the single-channel
    # ones but are compiled separately: equal up to rounding (16-bit stores: up
    # to a flipped rounding of a stored population)
    tol_n, tol_f = {"f64": (1e-13, 1e-12), "f32": (1e-5, 1e-5), "f16s": (1e-3, 1e-2)}[storage]
    for (cb, params, n0), (cs, _, _) in zip(batch, singles):
        cs.step(5)
        fb, fs = cb.get_populations(), cs.get_populations()
        dn = np.max(np.abs(cb.get_fields()[0] - cs.get_fields()[0]))
        df = np.max(np.abs(fb - fs)) / np.max(np.abs(fs))
        print(f"{storage} fused={fused}: batch vs single max|dn| {dn:.2e}, max|df|/max|f| {df:.2e}")
        assert dn <= tol_n and df <= tol_f
    if storage == "f64":
        for (cb, params, n0), m in zip(batch, masks):
            ref = O.OracleSim(O.OracleParams.from_dict(dict(params, solid=None if m is None else m[0])), n0).step(5)
            assert np.max(np.abs(cb.get_fields()[0] - ref.n)) <= 1e-12


# ------------------------------------------------------------------ degenerate lattices

@pytest.mark.parametrize("fused", [1, 0])
@pytest.mark.parametrize("dims,walls", [((1, 1, 2), True), ((2, 3, 1), True), ((1, 5, 3), True),
                                        ((3, 1, 4), False), ((2, 2, 1), False), ((5, 4, 2), True)])
def test_degenerate_lattices_fp64(nh, oracle_mod, dims, walls, fused):
    """One-site-wide directions (a site is its own x or y neighbour), a single
    layer between the plates, two-layer periodic boxes: FP64 against the oracle."""
    O = oracle_mod
    params = _generic(*dims, walls_z=walls, dt_fd=2, K=0.03, q0=0.7, W0=0.01, alpha4p=0.02)
    n0 = I.random_director(*dims, seed=11)
    u0 = I.random_velocity(*dims, 1e-3, seed=12)
    ref = _oracle_sim(O, params, n0, u0).step(9)
    ch = nh.Channel(dict(params, precision="fp64"))
    ch.set_fd_variant(fused)
    ch.set_fields(n0, u0)
    ch.step(9)
    n, u, rho = ch.get_fields()
    assert np.max(np.abs(n - ref.n)) < 1e-13
    assert np.max(np.abs(u - ref.u)) < 1e-13 * max(1e-3, np.max(np.abs(ref.u)))
    assert np.max(np.abs(rho - ref.rho)) < 1e-13


@pytest.mark.parametrize("storage", ["f32", "f16s", "bf16s"])
@pytest.mark.parametrize("dims,walls", [((6, 5, 7), True), ((64, 4, 3), False), ((16, 6, 5), True)])
def test_lb_launch_shapes_bitwise_equal(nh, storage, dims, walls):
    """The two- and four-site shapes (vector loads of aligned pairs or 4-site
    chunks, with the e_x = +-1 sources selected from two chunks, row ends
    wrapped) read the same values as the one-site shapes: identical populations
    and fields."""
    params = _generic(*dims, walls_z=walls, dt_fd=3)
    n0 = I.tilted_director(*dims, amplitude=0.3, seed=5)
    out = []
    for v in [v for v, spt in enumerate((2, 1, 2, 1, 4, 4)) if dims[0] % spt == 0]:
        ch = _channel(nh, params, n0, precision="fp32", storage=storage)
        ch.set_lb_variant(v)
        ch.step(10)
        out.append((ch.get_populations(), *ch.get_fields()))
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


# ------------------------------------------------------------------ auxiliary: run records, error paths

def test_run_records_jsonl(nh, tmp_path):
    import json
    from paper_2503_06610_gb300 import runlog
    params = _generic(16, 12, 8, dt_fd=4)
    n0 = I.skyrmion_tubes(16, 12, 8, [(8.0, 6.0)], 4.0)
    ch = _channel(nh, params, n0, precision="fp32")
    ch.set_tubes([(8.0, 6.0)])
    path = tmp_path / "run.jsonl"
    recs = runlog.run(ch, 3, path=str(path))
    lines = [json.loads(l) for l in open(path)]
    assert lines == json.loads(json.dumps(recs)) and len(lines) == 3
    assert [r["step"] for r in lines] == [4, 8, 12]
    assert all(r["nonfinite"] == 0 and r["mlups"] > 0 for r in lines)
    assert max(abs(r["mass"] - lines[0]["mass"]) for r in lines) < 1e-6 * ch.N
    assert len(lines[-1]["centroids"]) == 1


def test_workspace_too_small_is_enomem(nh):
    import torch
    p = nh.make_params(dict(_generic(8, 8, 8), precision="fp32"))
    need = nh.nh_workspace_bytes(p)
    ctx = nh.nh_create(p, torch.cuda.current_stream().cuda_stream)
    try:
        buf = torch.empty(need, dtype=torch.uint8, device="cuda")
        aligned = (buf.data_ptr() + 255) // 256 * 256
        with pytest.raises(nh.NHError) as e:
            nh.nh_bind_workspace(ctx, aligned, need // 2)
        assert e.value.code == nh.NH_ENOMEM
    finally:
        nh.nh_destroy(ctx)


# ------------------------------------------------------------------ combinations of the reading flags

@pytest.mark.parametrize("storage,tol", [("f16s", 3e-3), ("bf16s", 3e-2)])
def test_paper_order_with_16bit_stores(nh, oracle_mod, storage, tol):
    """paper_order runs the LB step of an FD interval twice (the scale controller
    with it); the 16-bit stores stay within their usual error of the oracle."""
    O = oracle_mod
    params, n0 = I.tiny_channel()
    params = dict(params, dt_fd=4, paper_order=True)
    ref = _oracle_sim(O, params, n0).step(400)
    ch = _channel(nh, params, n0, precision="fp32", storage=storage, shifted=True)
    ch.step(400)
    n, u, _ = ch.get_fields()
    assert O.rel_l2(u, ref.u) <= tol
    assert O.rel_l2(n, ref.n) <= tol


def test_paper_order_with_obstacle_and_frank3_fp64(nh, oracle_mod):
    O = oracle_mod
    nx, ny, nz = 18, 12, 8
    mask, normals = _sphere_mask(nx, ny, nz, (9.0, 6.0, 4.0), 2.6)
    params = _generic(nx, ny, nz, dt_fd=3, K=0.03, K11=0.045, K22=0.015, K33=0.06, q0=0.5, W0=0.002,
                      g=(1e-4, 0.0, 0.0), paper_order=True)
    n0 = I.tilted_director(nx, ny, nz, amplitude=0.3, seed=8)
    n0[:, mask == 1] = normals[:, mask == 1]
    ref = O.OracleSim(O.OracleParams.from_dict(dict(params, solid=mask)), n0).step(17)
    ch = nh.Channel(dict(params, precision="fp64"))
    ch.set_solid(mask)
    ch.set_fields(n0)
    ch.step(17)
    n, u, _ = ch.get_fields()
    fl = mask == 0
    assert O.rel_l2(n, ref.n) <= 1e-12
    assert O.rel_l2(u[:, fl], ref.u[:, fl]) <= 1e-10
    assert np.max(np.abs(ch.get_populations() - ref.f)) < 1e-14


@pytest.mark.parametrize("case", ["obstacle", "frank3"])
def test_relax_with_obstacle_or_frank3_fp64(nh, oracle_mod, case):
    """Director-only relaxation on the per-site kernels: the predictor-corrector
    at u = 0 of the oracle, with an obstacle (held directors) or the
    three-constant energy."""
    O = oracle_mod
    nx, ny, nz = 16, 12, 8
    extra = dict(K11=0.02, K22=0.006, K33=0.03) if case == "frank3" else {}
    params = _generic(nx, ny, nz, dt_fd=5, K=0.01, q0=0.5, W0=0.002, anchoring="none", **extra)
    n0 = I.skyrmion_tubes(nx, ny, nz, [(8.0, 6.0)], 5.0)
    mask = None
    if case == "obstacle":
        mask, normals = _sphere_mask(nx, ny, nz, (3.0, 3.0, 4.0), 2.2)
        n0[:, mask == 1] = normals[:, mask == 1]
    p = O.OracleParams.from_dict(dict(params, solid=mask))
    n = n0.copy()
    u = np.zeros_like(n0)
    for _ in range(12):
        n = O.fd_step(p, n, u)
    ch = nh.Channel(dict(params, precision="fp64"))
    if mask is not None:
        ch.set_solid(mask)
    ch.set_fields(n0)
    ch.relax(12)
    assert O.rel_l2(ch.get_fields()[0], n) < 1e-12

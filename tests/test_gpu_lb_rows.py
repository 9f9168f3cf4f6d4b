"""The row-staged LB kernel of the 16-bit stores (LB variant 6).

Whole x-rows of the 19 source planes are copied into shared memory by bulk
asynchronous copies and collided there with the same per-site code as every
other launch shape (Sec. II.C streaming, bounce-back and collision), so the
populations and fields must be bit-identical to the register shapes: with
plates and periodic z, on short and full rows, on the steps that write u and
rho and those that do not, through CUDA graphs and direct launches, and at the
256x256x64 size of the multi-tube channel.
"""
import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROWS = 6


@pytest.fixture(scope="module")
def nh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_06610_gb300 import nh as m
    m.load_library()
    return m


def _params(nx, ny, nz, walls, **kw):
    d = dict(nx=nx, ny=ny, nz=nz, walls_z=walls, anchoring="homeotropic", shifted=True, tau=0.8,
             g=(1e-5, -3e-6, 2e-6), K=0.03, q0=0.5, W0=0.0, dt_fd=3, **I.LESLIE_ALIGN_09)
    d.update(kw)
    return d


def _run(nh, params, variant, steps, graphs=True):
    ch = nh.Channel(dict(params, precision="fp32"))
    ch.set_graphs(graphs)
    ch.set_fields(I.tilted_director(params["nx"], params["ny"], params["nz"], amplitude=0.3, seed=5))
    ch.set_lb_variant(variant)
    ch.step(steps)
    out = (ch.get_populations(), *ch.get_fields())
    d = ch.diagnostics()
    ch.close()
    return out, d


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
@pytest.mark.parametrize("dims,walls", [((128, 4, 3), False), ((128, 5, 6), True), ((256, 3, 4), True),
                                        ((256, 7, 5), False)])
def test_rows_variant_bitwise_equal_to_register_shapes(nh, storage, dims, walls):
    params = _params(*dims, walls, storage=storage)
    ref, dref = _run(nh, params, 0, 10)
    for v, graphs in ((ROWS, True), (ROWS, False), (4, True)):
        out, d = _run(nh, params, v, 10, graphs)
        for a, b in zip(ref, out):
            assert np.array_equal(a, b), (v, graphs)
        assert d["mass"] == dref["mass"] and d["max_u"] == dref["max_u"]


def test_rows_variant_validity(nh):
    ok = nh.Channel(dict(_params(128, 4, 3, True, storage="f16s"), precision="fp32"))
    ok.set_lb_variant(ROWS)
    ok.close()
    for storage, nx in (("f32", 128), ("f16s", 96), ("bf16s", 384), ("f16s", 64), ("bf16s", 192)):
        ch = nh.Channel(dict(_params(nx, 4, 3, True, storage=storage), precision="fp32"))
        with pytest.raises(nh.NHError):
            ch.set_lb_variant(ROWS)
        ch.close()


def test_rows_variant_with_obstacle_falls_back(nh):
    params = _params(128, 6, 5, True, storage="f16s")
    mask = np.zeros(128 * 6 * 5, dtype=np.uint8)
    mask[128 * 6 * 2 + 128 * 3 + 10: 128 * 6 * 2 + 128 * 3 + 14] = 1
    outs = []
    for v in (0, ROWS):
        ch = nh.Channel(dict(params, precision="fp32"))
        ch.set_solid(mask)
        ch.set_fields(I.tilted_director(128, 6, 5, amplitude=0.3, seed=5))
        ch.set_lb_variant(v)
        ch.step(7)
        outs.append((ch.get_populations(), *ch.get_fields()))
        ch.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_rows_variant_full_size_multi_tube(nh, storage):
    """256x256x64 multi-tube channel, dt_FD = 16: one FD interval and one more
    LB step with the row-staged kernel equal the four-site shape bit for bit;
    the autotuner's choice keeps the state."""
    params, n0, centres = I.multi_tube_channel()
    outs = []
    for v in (4, ROWS):
        ch = nh.Channel(dict(params, precision="fp32", storage=storage))
        ch.set_fields(n0)
        ch.set_tubes(centres)
        ch.set_lb_variant(v)
        ch.step(17)
        outs.append((ch.get_populations(), *ch.get_fields(), ch.diagnostics()))
        ch.close()
    for a, b in zip(outs[0][:4], outs[1][:4]):
        assert np.array_equal(a, b)
    assert outs[0][4]["energy"] == outs[1][4]["energy"]
    ch = nh.Channel(dict(params, precision="fp32", storage=storage))
    ch.set_fields(n0)
    ch.step(3)
    before = ch.get_populations()
    chosen = ch.autotune()
    assert chosen in (0, 1, 2, 3, 4, 5, ROWS)
    assert np.array_equal(before, ch.get_populations())
    ch.close()

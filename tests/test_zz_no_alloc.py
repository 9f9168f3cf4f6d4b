"""nh_diagnostics_noalloc: the diagnostics reduction for callers that cannot
allocate device memory (a host application that only lends its own input and
output buffers, or a loop that cannot afford cudaMalloc's device sync).

It is checked through the C ABI against the ordinary entry point,
nh_diagnostics, on the same state, on two calls in a row (the second after
more steps, so the shared static scratch is reused with new data).  The
caller-side tensors here are ordinary torch allocations made by the test; the
entry point itself allocates nothing.
"""
import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_06610_gb300 import nh
    nh.load_library()
    return torch, nh


def _device_state(torch, ch, dtype):
    f = ch.get_populations()
    n, u, rho = ch.get_fields()
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")
    return cuda(f), cuda(n), cuda(u), cuda(rho)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_nh_diagnostics_twice(env, prec):
    torch, nh = env
    params, n0 = I.tiny_channel()
    params = dict(params, K=0.03, q0=0.3, W0=0.01, dt_fd=2)
    ch = nh.Channel(dict(params, precision=prec))
    ch.set_fields(n0)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    p = nh.make_params(dict(params, precision=prec))
    for steps in (20, 37):                       # two calls in a row, new data each time
        ch.step(steps)
        ref = ch.diagnostics()
        f, n, u, rho = _device_state(torch, ch, dtype)
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        nh.nh_diagnostics_noalloc(p, f, n, u, rho, out, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        v = out.cpu().numpy()
        mass = v[0] + ch.N                      # shifted populations
        assert abs(mass - ref["mass"]) <= 1e-12 * ch.N
        # nh_diagnostics reads the director alone after a folded LB step and sums
        # 16-layer chunks, this entry point 4-layer ones: in FP32 the per-site
        # energies are grouped differently before the FP64 sum
        assert abs(v[1] - ref["energy"]) <= (1e-11 if prec == "fp64" else 2e-6) * abs(ref["energy"])
        # nh_diagnostics takes max |u| from the LB launch's own components, this
        # entry point from the stored u: in FP32 the two norms may round one ulp apart
        assert abs(v[2] - ref["max_u"]) <= (1e-12 if prec == "fp64" else 2.5e-7) * ref["max_u"]
        assert abs(v[3] - ref["min_norm"]) <= 1e-15 and abs(v[4] - ref["max_norm"]) <= 1e-15
        assert v[5] == 0.0


def test_noalloc_rejects_oversized_domain(env):
    torch, nh = env
    p = nh.make_params(dict(nx=1024, ny=1024, nz=16, precision="fp32"))
    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(nh.NHError) as e:
        nh.nh_diagnostics_noalloc(p, t, t, t, t, out)
    assert e.value.code == nh.NH_EINVAL
    assert "larger than this entry point accepts" in str(e.value)


def test_noalloc_rejects_bad_parameters(env):
    """The parameters get nh_create's checks: a three-constant flag of 2 or an
    unknown anchoring is an error, not a silently different energy."""
    torch, nh = env
    t = torch.zeros(8 * 8 * 8 * 19, dtype=torch.float32, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    for bad in (dict(frank3=2), dict(anchoring=5), dict(walls_z=2), dict(shifted=3)):
        p = nh.make_params(dict(nx=8, ny=8, nz=8, precision="fp32"))
        for k, v in bad.items():
            setattr(p, k, v)
        with pytest.raises(nh.NHError) as e:
            nh.nh_diagnostics_noalloc(p, t, t, t, t, out)
        assert e.value.code == nh.NH_EINVAL


@pytest.mark.parametrize("case", ["odd_nx", "offset", "frank3"])
def test_noalloc_variants_match_nh_diagnostics(env, case):
    """The single-site path (odd nx, or fields offset by one element from an
    aligned allocation) and the three-constant energy, against nh_diagnostics;
    after a first call, a second allocates no device memory."""
    torch, nh = env
    nx = 15 if case == "odd_nx" else 16
    params = dict(nx=nx, ny=12, nz=8, walls_z=True, anchoring="none", shifted=True, tau=0.8, g=(1e-5, 0.0, 0.0),
                  K=0.03, q0=0.4, W0=0.01, dt_fd=2, **I.LESLIE_ALIGN_09)
    if case == "frank3":
        params.update(K11=0.02, K22=0.035, K33=0.05)
    n0 = I.skyrmion_tubes(nx, 12, 8, [(nx / 2, 6.0)], 4.0)
    ch = nh.Channel(dict(params, precision="fp64"))
    ch.set_fields(n0)
    ch.step(8)
    ref = ch.diagnostics()
    f, n, u, rho = _device_state(torch, ch, torch.float64)
    if case == "offset":  # views one element into a larger buffer: not 16-byte aligned
        def shift(a):
            b = torch.zeros(a.numel() + 1, dtype=a.dtype, device="cuda")
            b[1:] = a.reshape(-1)
            return b[1:]
        f, n, u, rho = shift(f), shift(n), shift(u), shift(rho)
    p = nh.make_params(dict(params, precision="fp64"))
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    nh.nh_diagnostics_noalloc(p, f, n, u, rho, out, stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    nh.nh_diagnostics_noalloc(p, f, n, u, rho, out, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    v = out.cpu().numpy()
    assert abs(v[0] + ch.N - ref["mass"]) <= 1e-12 * ch.N
    assert abs(v[1] - ref["energy"]) <= 1e-11 * abs(ref["energy"])
    assert abs(v[2] - ref["max_u"]) <= 1e-12 * ref["max_u"]
    assert abs(v[3] - ref["min_norm"]) <= 1e-15 and abs(v[4] - ref["max_norm"]) <= 1e-15

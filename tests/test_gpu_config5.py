"""Mixed-precision batched forward + backward at full size: 256 one-year sources (N = 3 153 600
each, parameters drawn as for the batched workload, seed 5), flexing orbit, order 41, in the
launch configuration of the batched calls.  Forward: every source's X, Y, Z at sampled outputs
against the oracle (relative L2 <= 1e-6 per source).  Backward (the mixed adjoint: float-float
weights and sums in the transposes and the sky-angle reads, geometry in FP64): the batched dot-product identity <R h, g> = <h, R^T g> with the mixed
forward, which holds at any size to the forward's own accuracy, and per source the gradients of
a cotangent on a window of 4000 outputs (zero elsewhere) against the oracle's gradients of the same
cotangent on a sub-span around the window (the gradients of such a cotangent vanish outside the
window's reach, so the sub-span result is exact).  Device memory: about 105 GB."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402
from _gpu import DT, T0, parity_bound  # noqa: E402

S, N, P = 256, synth.ONE_YEAR_SAMPLES, 41


def dot(a, b, chunk=1 << 28):
    """Dot product of long float64 device vectors in chunks (a single BLAS dot takes at most
    2^31 - 1 elements)."""
    return sum(float(torch.dot(a[i:i + chunk], b[i:i + chunk])) for i in range(0, a.numel(), chunk))


def test_config5_mixed_forward_and_backward():
    if torch.cuda.get_device_properties(0).total_memory < 160e9:
        pytest.skip("needs a GPU with >= 160 GB")
    srcs = synth.draw_sources(S, seed=5, A=1e-22, fdot=1e-17)
    m = synth.input_margin_samples(DT, P)
    nh = N + 2 * m
    h_off = np.arange(S + 1, dtype=np.int64) * nh
    out_off = np.arange(S + 1, dtype=np.int64) * N
    t0h = np.full(S, T0 - m * DT)
    sky = np.array([[x.lam, x.beta, x.psi] for x in srcs])
    dev = torch.device("cuda", 0)
    d_hp = torch.empty(S * nh, dtype=torch.float64, device=dev)
    d_hc = torch.empty(S * nh, dtype=torch.float64, device=dev)
    t = synth.sample_grid(t0h[0], DT, nh)
    strain = []
    for s, src in enumerate(srcs):
        a, b = synth.gb_polarisations(src, t)
        strain.append((a, b))
        d_hp[s * nh:(s + 1) * nh].copy_(torch.from_numpy(a))
        d_hc[s * nh:(s + 1) * nh].copy_(torch.from_numpy(b))
    orb = synth.orbit_flexing(T0 - 3e5, T0 + DT * N + 3e5)
    ctx = lr.Context(0)
    o = lr.Orbit(ctx, orb.t_knots, orb.pos, None)
    plan = lr.Plan(ctx, P, 1, DT, o, t0=T0, precision=lr.MIXED)
    args = [torch.tensor(x, device=dev) for x in (h_off, out_off, t0h, sky)]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    xyz = plan.response_batched(*args, d_hp, d_hc)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t1
    plan.check()
    # forward: 40 sampled outputs per source against the oracle
    orc = oracle.Orbit(orb.t_knots, orb.pos, None)
    rng = np.random.default_rng(55)
    worst = 0.0
    xyz3 = xyz.view(S, 3, N)
    for s, src in enumerate(srcs):
        idx = np.sort(rng.integers(0, N, 40))
        a, b = strain[s]
        call = (P, 2, DT, T0, N, orc, orc, a, b, t0h[s], src.lam, src.beta, src.psi, idx)
        ref = oracle.response_at(*call)
        scale = oracle.response_at(*call, absval=True)
        got = xyz3[s][:, torch.from_numpy(idx).to(dev)].cpu().numpy()
        err = np.linalg.norm(got - ref)
        assert err <= parity_bound(ref, scale, P + 1, 1e-6), f"source {s}: rel L2 {err / np.linalg.norm(ref):.3e}"
        worst = max(worst, err / np.linalg.norm(ref))
    # backward: dot-product identity over the whole batch
    gen = torch.Generator(device=dev)
    gen.manual_seed(20220413)
    g = torch.randn(3 * S * N, dtype=torch.float64, device=dev, generator=gen)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    g_hp, g_hc, g_sky = plan.backward_batched(*args, d_hp, d_hc, g)
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t1
    plan.check()
    lhs = dot(xyz, g)
    rhs = dot(d_hp, g_hp) + dot(d_hc, g_hc)
    norm = (dot(xyz, xyz) * dot(g, g)) ** 0.5
    assert abs(lhs - rhs) <= 1e-6 * norm
    assert torch.isfinite(g_sky).all()
    del g_hp, g_hc, g_sky
    # per-source gradients against the oracle: white cotangents on a window of W outputs
    W, H = 4000, 200
    pick = rng.choice(S, 4, replace=False)
    gw = torch.zeros(3 * S * N, dtype=torch.float64, device=dev)
    win = {}
    for s in pick:
        a0 = int(rng.integers(H + 1000, N - W - H - 1000))
        vals = rng.normal(size=(3, W))
        win[s] = (a0, vals)
        for c in range(3):
            gw[(3 * s + c) * N + a0:(3 * s + c) * N + a0 + W] = torch.from_numpy(vals[c])
    g_hp, g_hc, g_sky = plan.backward_batched(*args, d_hp, d_hc, gw)
    plan.check()
    g_sky = g_sky.cpu().numpy()
    worst_h = worst_s = 0.0
    for s in pick:
        a0, vals = win[s]
        src = srcs[s]
        lo, n_sub = a0 - H, W + 2 * H
        a, b = strain[s]
        gsub = np.zeros((3, n_sub))
        gsub[:, H:H + W] = vals
        rp, rc, rs, scale = oracle.backward(P, 2, DT, T0 + lo * DT, n_sub, orc, orc, a[lo:lo + n_sub + 2 * m],
                                            b[lo:lo + n_sub + 2 * m], t0h[s] + lo * DT, src.lam, src.beta, src.psi,
                                            gsub, with_scale=True)
        gp = g_hp[s * nh + lo:s * nh + lo + n_sub + 2 * m].cpu().numpy()
        gc = g_hc[s * nh + lo:s * nh + lo + n_sub + 2 * m].cpu().numpy()
        eh = np.linalg.norm(np.r_[gp - rp, gc - rc]) / np.linalg.norm(np.r_[rp, rc])
        assert eh <= 1e-6, f"source {s}: strain gradient rel L2 {eh:.2e}"
        bound = np.maximum(1e-6 * np.abs(rs), 4 * (P + 17) * 2.0 ** -24 * scale)
        assert np.all(np.abs(g_sky[s] - rs) <= bound), (s, g_sky[s], rs, bound)
        worst_h = max(worst_h, eh)
        worst_s = max(worst_s, float(np.max(np.abs(g_sky[s] - rs) / np.abs(rs))))
    print(f"config 5: forward (mixed) {t_fwd:.2f} s = {6 * S * N / t_fwd:.3e} link-samples/s, worst sampled "
          f"rel L2 {worst:.2e}; backward (mixed adjoint) {t_bwd:.2f} s; adjoint identity "
          f"{abs(lhs - rhs) / norm:.1e} of |Rh||g|; per-source gradients against the oracle (window of {W} "
          f"outputs): strain rel L2 <= {worst_h:.2e}, sky angles rel <= {worst_s:.2e}")

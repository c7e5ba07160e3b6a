"""GPU parity of the fused likelihood epilogue (A, E, T of each tile against the data, per-tile
partial inner products, per-source fixed-order sums) against the oracle.

Two checks per case: (1) the epilogue alone, against the oracle's inner products of the X, Y, Z
the same call returned (FP64 build: only the summation order differs, bound 1e-12 of the sum of
|terms|; mixed build: the epilogue runs in FP32 on the tile-scaled values, each term carrying
a few roundings of 2^-24 and each tile sum a tree of depth 8 plus 8 warp partials, bound 4e-6 of
the sum of |terms|);
(2) end to end, against the oracle's inner products of the oracle's own response, with the bound
the response's parity bound implies: |d<h|h>| <= (2 e + e^2) <h|h>, |d<d|h>| <= e sqrt(<d|d><h|h>)
for a relative L2 response error e (channel weights within a factor wmax/wmin)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2204_06633_gb300 as lr  # noqa: E402
import synth  # noqa: E402
from _gpu import DT, T0, Pair, dev, host, parity_bound, sky  # noqa: E402

SIGMA = 1e-21
W = (1.0 / SIGMA**2, 2.0 / SIGMA**2, 0.5 / SIGMA**2)


@pytest.fixture(scope="module")
def ctx():
    return lr.Context(0)


@pytest.fixture(scope="module")
def flex(ctx):
    return Pair(ctx, synth.orbit_flexing(-2e6, 3e5 * DT + 2e6))


def epilogue_bound(xyz, data, w, k):
    """Sum of |terms| of the two inner products, times k."""
    a = np.abs(oracle.aet(xyz))
    d = np.abs(data)
    wa = np.asarray(w)[:, None]
    return k * float(np.sum(wa * a * d)), k * float(np.sum(wa * a * a))


def epilogue_k(precision):
    return 1e-12 if precision == lr.FP64 else 4e-6


def check_epilogue(got, xyz_gpu, data, w, precision):
    dh, hh = got
    e_dh, e_hh = oracle.like_inner(xyz_gpu, data, w)
    bdh, bhh = epilogue_bound(xyz_gpu, data, w, epilogue_k(precision))
    assert abs(dh - e_dh) <= bdh, (dh, e_dh, bdh)
    assert abs(hh - e_hh) <= bhh, (hh, e_hh, bhh)
    return bdh, bhh


def check_against_oracle(got, xyz_gpu, xyz_ref, scale, data, w, T, rel, precision):
    dh, hh = got
    # (1) the epilogue, given the template the kernel formed
    bdh, bhh = check_epilogue(got, xyz_gpu, data, w, precision)
    # (2) end to end, from the response parity bound
    r_dh, r_hh = oracle.like_inner(xyz_ref, data, w)
    e = parity_bound(xyz_ref, scale, T, rel) / np.linalg.norm(xyz_ref)
    wr = max(w) / min(w)
    dd = float(np.sum(np.asarray(w)[:, None] * data * data))
    assert abs(hh - r_hh) <= wr * (2 * e + e * e) * r_hh + bhh
    assert abs(dh - r_dh) <= wr * e * math.sqrt(dd * r_hh) + bdh


@pytest.mark.parametrize("precision,rel", [(lr.FP64, 1e-12), (lr.MIXED, 1e-6)])
@pytest.mark.parametrize("N", [30001, 7])
def test_single_source(ctx, flex, precision, rel, N):
    p = 25
    src = synth.draw_sources(1, seed=12, A=1e-21, fdot=1e-17)[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    args = (p, 2, DT, T0, N, flex.orc, flex.orc, hp, hc, t0h, src.lam, src.beta, src.psi)
    ref = oracle.response(*args)
    scale = oracle.response(*args, absval=True)
    data = oracle.aet(ref + synth.white_noise(ref.shape, SIGMA, seed=5))
    plan = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, precision=precision)
    xyz = torch.empty(3 * N, dtype=torch.float64, device="cuda:0")
    d_hp, d_hc, d_data = dev(hp), dev(hc), dev(data)
    got = host(plan.likelihood(d_hp, d_hc, t0h, sky(src), d_data, W, xyz=xyz))
    plan.check()
    check_against_oracle(got, host(xyz).reshape(3, N), ref, scale, data, W, p + 1, rel, precision)
    # without the X, Y, Z output: the same sums bit for bit, and the same X, Y, Z as lr_response
    got2 = host(plan.likelihood(d_hp, d_hc, t0h, sky(src), d_data, W))
    assert np.array_equal(got, got2)
    assert np.array_equal(host(xyz), host(plan.response(d_hp, d_hc, t0h, sky(src))).ravel())
    plan.check()


def batch(lens, seed, p):
    lens = np.asarray(lens, dtype=np.int64)
    srcs = synth.draw_sources(len(lens), seed=seed, A=1e-21, fdot=1e-17)
    m = synth.input_margin_samples(DT, p)
    nh = lens + 2 * m
    h_off = np.concatenate([[0], np.cumsum(nh)]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    hp, hc = np.empty(h_off[-1]), np.empty(h_off[-1])
    t0h = np.full(len(lens), T0 - m * DT)
    for s, src in enumerate(srcs):
        a, b = synth.gb_polarisations(src, synth.sample_grid(t0h[s], DT, int(nh[s])))
        hp[h_off[s]:h_off[s + 1]], hc[h_off[s]:h_off[s + 1]] = a, b
    sky_ = np.array([[x.lam, x.beta, x.psi] for x in srcs])
    return srcs, h_off, out_off, t0h, sky_, hp, hc


@pytest.mark.parametrize("precision,rel", [(lr.FP64, 1e-12), (lr.MIXED, 1e-6)])
def test_batched_ragged_with_empty_and_tiny_sources(ctx, flex, precision, rel):
    p = 11
    lens = [9000, 0, 1, 2345, 341, 6000]
    srcs, h_off, out_off, t0h, sky_, hp, hc = batch(lens, 31, p)
    data = np.empty(3 * int(out_off[-1]))
    refs = []
    for s, src in enumerate(srcs):
        N = lens[s]
        if N == 0:
            refs.append(None)
            continue
        args = (p, 2, DT, T0, N, flex.orc, flex.orc, hp[h_off[s]:h_off[s + 1]], hc[h_off[s]:h_off[s + 1]], t0h[s],
                src.lam, src.beta, src.psi)
        ref = oracle.response(*args)
        refs.append((ref, oracle.response(*args, absval=True)))
        data[3 * out_off[s]:3 * out_off[s + 1]] = oracle.aet(
            ref + synth.white_noise(ref.shape, SIGMA, seed=100 + s)).ravel()
    plan = lr.Plan(ctx, p, 1, DT, flex.gpu, t0=T0, precision=precision)
    d = lambda a: torch.tensor(a, device="cuda:0")  # noqa: E731
    dargs = (d(h_off), d(out_off), d(t0h), d(sky_), d(hp), d(hc), d(data))
    xyz = torch.empty(3 * int(out_off[-1]), dtype=torch.float64, device="cuda:0")
    got = host(plan.likelihood_batched(*dargs, weights=W, xyz=xyz))
    plan.check()
    xyz_h = host(xyz)
    for s in range(len(lens)):
        if refs[s] is None:
            assert got[s, 0] == 0.0 and got[s, 1] == 0.0
            continue
        N = lens[s]
        sl = slice(3 * out_off[s], 3 * out_off[s + 1])
        check_against_oracle(got[s], xyz_h[sl].reshape(3, N), refs[s][0], refs[s][1], data[sl].reshape(3, N),
                             W, p + 1, rel, precision)
    # deterministic: a second call gives the same bits
    assert np.array_equal(got, host(plan.likelihood_batched(*dargs, weights=W)))
    plan.check()


@pytest.mark.parametrize("precision", [lr.FP64, lr.MIXED])
def test_data_equal_to_template_gives_zero_residual(ctx, flex, precision):
    """<d - h|d - h> = <d|d> + <h|h> - 2 <d|h> vanishes (to rounding) when d is the template."""
    p = 25
    N = 20000
    src = synth.draw_sources(1, seed=3, A=1e-21, fdot=1e-17)[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, precision=precision)
    xyz = host(plan.response(dev(hp), dev(hc), t0h, sky(src))).reshape(3, N)
    data = oracle.aet(xyz)
    dh, hh = host(plan.likelihood(dev(hp), dev(hc), t0h, sky(src), dev(data), W))
    plan.check()
    dd = float(np.sum(np.asarray(W)[:, None] * data * data))
    assert abs(dd + hh - 2 * dh) <= 4 * epilogue_k(precision) * hh


def test_data_shorter_than_offsets_is_refused_on_device(ctx, flex):
    """n_total smaller than out_off[S]: the sources past it get NaN and the error word is set;
    nothing past the data is read."""
    p = 11
    lens = [3000, 4000]
    srcs, h_off, out_off, t0h, sky_, hp, hc = batch(lens, 7, p)
    plan = lr.Plan(ctx, p, 1, DT, flex.gpu, t0=T0, precision=lr.MIXED)
    d = lambda a: torch.tensor(a, device="cuda:0")  # noqa: E731
    short = torch.zeros(3 * 5000, dtype=torch.float64, device="cuda:0")
    got = host(plan.likelihood_batched(d(h_off), d(out_off), d(t0h), d(sky_), d(hp), d(hc), short))
    assert np.isfinite(got[0]).all()
    assert np.isnan(got[1]).all()
    with pytest.raises(lr.LRError):
        plan.check()


def test_bench_workload_sampled(ctx):
    """The timed configuration: 1024 ragged sources (sum N = 5.6e8), order 25, mixed, one
    persistent launch.  Data: seeded noise drawn on the device.  Six sources checked through the
    epilogue against the X, Y, Z the call returned, the two shortest of them end to end."""
    import bench

    p = 25
    lens, srcs = bench.workload(0, 1, 1024)
    h_off, out_off, t0h, sky_, hp, hc = bench.build_inputs(lens, srcs, p)
    orb = synth.orbit_flexing(T0 - 3e5, T0 + DT * int(lens.max()) + 3e5)
    o = Pair(ctx, orb)
    plan = lr.Plan(ctx, p, 1, DT, o.gpu, t0=T0, precision=lr.MIXED)
    d = lambda a: torch.tensor(a, device="cuda:0")  # noqa: E731
    total = int(out_off[-1])
    gen = torch.Generator(device="cuda:0")
    gen.manual_seed(20220413)
    data = torch.randn(3 * total, dtype=torch.float64, device="cuda:0", generator=gen) * SIGMA
    xyz = torch.empty(3 * total, dtype=torch.float64, device="cuda:0")
    got = host(plan.likelihood_batched(d(h_off), d(out_off), d(t0h), d(sky_), d(hp), d(hc), data, weights=W,
                                       xyz=xyz))
    plan.check()
    rng = np.random.default_rng(9)
    pick = rng.choice(len(lens), 6, replace=False)
    short = sorted(pick, key=lambda s: lens[s])[:2]
    for s in pick:
        N = int(lens[s])
        sl = slice(3 * int(out_off[s]), 3 * int(out_off[s + 1]))
        xs = host(xyz[sl]).reshape(3, N)
        ds = host(data[sl]).reshape(3, N)
        if s in short:
            src = srcs[s]
            args = (p, 2, DT, T0, N, o.orc, o.orc, hp[h_off[s]:h_off[s + 1]], hc[h_off[s]:h_off[s + 1]], t0h[s],
                    src.lam, src.beta, src.psi)
            check_against_oracle(got[s], xs, oracle.response(*args), oracle.response(*args, absval=True), ds, W,
                                 p + 1, 1e-6, lr.MIXED)
        else:
            check_epilogue(got[s], xs, ds, W, lr.MIXED)


def aet_matrix():
    """The A, E, T map as a 3x3 matrix, column j = the oracle's A, E, T of the unit X, Y, Z
    pattern j."""
    return np.stack([oracle.aet(np.eye(3)[:, j].reshape(3, 1))[:, 0] for j in range(3)], axis=1)


@pytest.mark.parametrize("scale", [1.0, -0.37])
def test_likelihood_grad_against_the_oracle_map(ctx, flex, scale):
    """g = scale M^T W (d - M x) per sample, single source and a ragged batch with an empty
    source (M from the oracle's A, E, T; a plain matrix product on the host)."""
    M = aet_matrix()
    rng = np.random.default_rng(21)
    w = (2.0, 0.5, 1.25)
    plan = lr.Plan(ctx, 11, 1000, DT, flex.gpu, t0=T0)
    x, dat = rng.normal(size=(3, 1000)), rng.normal(size=(3, 1000))
    got = host(plan.likelihood_grad(dev(x), dev(dat), w, scale=scale))
    ref = scale * M.T @ (np.asarray(w)[:, None] * (dat - M @ x))
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)
    lens = [700, 0, 1, 2500]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    xb, db = rng.normal(size=3 * off[-1]), rng.normal(size=3 * off[-1])
    gb = host(plan.likelihood_grad_batched(torch.tensor(off, device="cuda:0"), dev(xb), dev(db), w, scale=scale))
    plan.check()
    for s, n in enumerate(lens):
        sl = slice(3 * off[s], 3 * off[s + 1])
        r = scale * M.T @ (np.asarray(w)[:, None] * (db[sl].reshape(3, n) - M @ xb[sl].reshape(3, n)))
        assert np.allclose(gb[sl].reshape(3, n), r, rtol=0, atol=1e-14 * max(1.0, np.abs(r).max(initial=0.0)))


@pytest.mark.parametrize("precision", [lr.FP64, lr.MIXED])
def test_log_likelihood_autograd(ctx, flex, precision):
    """Gradients of <d|h> - <h|h>/2 through lr.log_likelihood: against autograd through the fused
    response with the loss written in PyTorch (same adjoint, independent likelihood gradient),
    and, in FP64, against central differences (exact for h: the loss is quadratic in h; step 1e-6
    relative for the sky angles, agreement 1e-6)."""
    p, N = 11, 4000
    src = synth.draw_sources(1, seed=8, A=1e-21, fdot=1e-17)[0]
    t0h, hp, hc = synth.gb_input(src, T0, DT, N, p)
    plan = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, precision=precision)
    xyz0 = host(plan.response(dev(hp), dev(hc), t0h, sky(src))).reshape(3, N)
    data = dev(oracle.aet(xyz0 + synth.white_noise(xyz0.shape, SIGMA, seed=4)))
    M = torch.tensor(aet_matrix(), device="cuda:0")
    wt = torch.tensor(W, dtype=torch.float64, device="cuda:0")[:, None]

    def run(fn):
        a = dev(hp).requires_grad_()
        b = dev(hc).requires_grad_()
        s = torch.tensor(sky(src), dtype=torch.float64, device="cuda:0", requires_grad=True)
        L = fn(a, b, s)
        L.backward()
        return float(L.detach()), host(a.grad), host(b.grad), host(s.grad)

    L1, gp1, gc1, gs1 = run(lambda a, b, s: lr.log_likelihood(plan, a, b, s, t0h, data, W))

    def torch_loss(a, b, s):
        h = M @ lr.response(plan, a, b, s, t0h)
        return torch.sum(wt * (data * h - 0.5 * h * h))

    L2, gp2, gc2, gs2 = run(torch_loss)
    plan.check()
    tol = 1e-12 if precision == lr.FP64 else 1e-5
    assert abs(L1 - L2) <= tol * abs(L2)
    for g1, g2 in ((gp1, gp2), (gc1, gc2), (gs1, gs2)):
        assert np.linalg.norm(g1 - g2) <= 1e-12 * np.linalg.norm(g2)
    if precision == lr.FP64:
        rng = np.random.default_rng(5)
        v = rng.normal(size=hp.shape) * np.abs(hp).max()

        def L_at(a, s=sky(src)):
            return float(lr.log_likelihood(plan, dev(a), dev(hc), tuple(s), t0h, data, W))

        fd = (L_at(hp + v) - L_at(hp - v)) / 2.0
        assert abs(fd - float(np.dot(gp1, v))) <= 1e-9 * abs(fd)
        for i in range(3):
            e = 1e-6 * max(1.0, abs(sky(src)[i]))
            sp, sm = list(sky(src)), list(sky(src))
            sp[i] += e
            sm[i] -= e
            fds = (L_at(hp, tuple(sp)) - L_at(hp, tuple(sm))) / (2 * e)
            assert abs(fds - gs1[i]) <= 1e-6 * np.linalg.norm(gs1)


def test_likelihood_grad_batched_refuses_offsets_past_the_arrays(ctx, flex):
    plan = lr.Plan(ctx, 11, 1000, DT, flex.gpu, t0=T0)
    off = torch.tensor([0, 700, 1400], dtype=torch.int64, device="cuda:0")
    x = torch.ones(3 * 1000, dtype=torch.float64, device="cuda:0")
    g = torch.full_like(x, 7.0)
    plan.likelihood_grad_batched(off, x, x.clone(), (1.0, 1.0, 1.0), g_xyz=g)
    torch.cuda.synchronize()
    assert torch.all(g[2100:] == 7.0)  # the second source is not touched ...
    with pytest.raises(lr.LRError):    # ... and the error word says why
        plan.check()


@pytest.mark.parametrize("precision", [lr.FP64, lr.MIXED])
def test_log_likelihood_entry_points_match_the_pair(ctx, flex, precision):
    """lr_log_likelihood(_batched) returns <d|h> - <h|h>/2 from the same per-tile partials as
    lr_likelihood(_batched): equal up to the one rounding of forming the difference."""
    p = 11
    lens = [5000, 0, 1, 3001]
    srcs, h_off, out_off, t0h, sky_, hp, hc = batch(lens, 51, p)
    data = np.random.default_rng(2).normal(size=3 * int(out_off[-1])) * SIGMA
    plan = lr.Plan(ctx, p, 1, DT, flex.gpu, t0=T0, precision=precision)
    d = lambda a: torch.tensor(a, device="cuda:0")  # noqa: E731
    dargs = (d(h_off), d(out_off), d(t0h), d(sky_), d(hp), d(hc), d(data))
    pair = host(plan.likelihood_batched(*dargs, weights=W))
    logl = host(plan.log_likelihood_batched(*dargs, weights=W))
    plan.check()
    assert logl.shape == (len(lens),)
    ref = pair[:, 0] - 0.5 * pair[:, 1]
    tol = 4 * 2.0 ** -53 * (np.abs(pair[:, 0]) + np.abs(pair[:, 1]))
    assert np.all(np.abs(logl - ref) <= tol)
    # single source
    N = lens[0]
    plan1 = lr.Plan(ctx, p, N, DT, flex.gpu, t0=T0, precision=precision)
    hs = slice(h_off[0], h_off[1])
    sd = dev(data[:3 * N])
    pr = host(plan1.likelihood(dev(hp[hs]), dev(hc[hs]), t0h[0], sky_[0], sd, W))
    l1 = host(plan1.log_likelihood(dev(hp[hs]), dev(hc[hs]), t0h[0], sky_[0], sd, W))
    plan1.check()
    assert abs(l1[0] - (pr[0] - 0.5 * pr[1])) <= 4 * 2.0 ** -53 * (abs(pr[0]) + abs(pr[1]))

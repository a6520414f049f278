"""Learned surrogate: tensor-core GEMM against FP64 numpy, network gradients
against the FP64 reference network, training and ensemble prediction."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2604_09243_gb300 import build

    build.build()
    import paper_2604_09243_gb300 as G

    return G


# the last two shapes have two or more 128 x 128 tiles per SM: the persistent kernel (double-buffered TMEM)
@pytest.mark.parametrize("M,N,K,pad", [(128, 128, 64, 0), (256, 384, 512, 0), (1024, 512, 256, 8), (8192, 512, 512, 0),
                                       (16384, 512, 256, 8), (32768, 512, 512, 0)])
def test_tensor_core_gemm(G, M, N, K, pad):
    torch = pytest.importorskip("torch")
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K + pad, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K + pad, generator=g).to(torch.bfloat16).cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    G.gemm_bf16_tn(A.data_ptr(), K + pad, B.data_ptr(), K + pad, M, N, K, C.data_ptr(), N)
    ref = A[:, :K].double().cpu().numpy() @ B[:, :K].double().cpu().numpy().T
    got = C.cpu().numpy()
    assert not np.isnan(got).any()
    # exact BF16 products, FP32 accumulation
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.sqrt(K) * np.abs(ref).max()
    # the enqueue-only entry point: the same result bit for bit, no bounded wait gave up
    C2 = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    G.gemm_bf16_tn_async(A.data_ptr(), K + pad, B.data_ptr(), K + pad, M, N, K, C2.data_ptr(), N, err.data_ptr(),
                         torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert np.array_equal(C2.cpu().numpy(), got)


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    x = np.stack([rng.uniform(0, 360, n), rng.uniform(-30, 30, n), np.exp(rng.uniform(np.log(1e9), np.log(12e9), n))], 1)
    return rng, x


def _fp32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def _bf16(a):
    """Round to BF16 (nearest, ties to even) from the FP32 value, as the kernels do."""
    u = np.asarray(a, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _bf16_network(p, B, x, t, width, depth, nf):
    """The FP64 reference network with the surrogate kernels' roundings: FP32
    inputs, BF16 Fourier features, BF16 weights and activations into every hidden
    GEMM, FP32 pre-activations and head, BF16 deltas (dz) out of every backward
    step; products and sums otherwise exact. Returns (loss, flat gradient)."""
    Ws = mlp.unpack(p, width, depth, nf)
    arg = _fp32(_fp32(mlp.encode(x)) @ _fp32(B).T)
    h = [_bf16(np.concatenate([np.sin(2 * np.pi * arg), np.cos(2 * np.pi * arg)], 1))]
    zs = []
    for l in range(depth):
        W, b = Ws[l]
        z = _fp32(h[-1] @ _bf16(W).T + _fp32(b))
        zs.append(z)
        h.append(_bf16(mlp.gelu(z)))
    Wh, bh = _fp32(Ws[depth][0]), _fp32(Ws[depth][1])
    y = _fp32(h[-1] @ Wh.T + bh)
    t = np.asarray(t, np.float64)
    dy = _fp32(2.0 * (y - t) / y.size)
    grads = [None] * (depth + 1)
    grads[depth] = (dy.T @ h[depth], dy.sum(0))
    dz = _bf16(_fp32(dy @ Wh) * mlp.gelu_grad(zs[depth - 1]))
    for l in range(depth - 1, -1, -1):
        grads[l] = (dz.T @ h[l], dz.sum(0))
        if l > 0:
            dz = _bf16(_fp32(dz @ _bf16(Ws[l][0])) * mlp.gelu_grad(zs[l - 1]))
    loss = float(np.mean((y - t) ** 2))
    return loss, np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])


# 16384 rows: the forward and input-gradient GEMMs of the deep network run the persistent kernel
@pytest.mark.parametrize("width,depth,nf,n", [(128, 2, 128, 512), (512, 6, 256, 512), (512, 6, 256, 16384)])
def test_gradients_against_fp64_reference(G, width, depth, nf, n):
    """Loss and gradients of the tensor-core forward and backward against the FP64
    reference network (oracle/mlp.py). The bound comes from BF16 itself: the same
    network with the kernels' BF16 and FP32 roundings (in FP64 otherwise) moves
    each layer's gradient by some amount from the exact one; the GPU must stay
    within twice that plus 1e-3 of the layer's largest entry, and within
    1e-3 per layer back from the output of the rounded network (FP32 sums and
    library functions left)."""
    s = G.Surrogate(0, n_members=1, width=width, depth=depth, n_fourier=nf, fourier_sigma=2.0, seed=3)
    rng, x = _samples(n, 4)
    t = rng.normal(0, 1, (n, 4))
    p = s.params(0).astype(np.float64)
    B = s.fourier(0).astype(np.float64)
    loss_g, g = s.grads(x, t)
    s.close()
    loss_o, go, _ = mlp.loss_and_grads(p, B, x, t, width, depth, nf)
    loss_b, gb = _bf16_network(p, B, x, t, width, depth, nf)
    assert abs(loss_g - loss_b) <= 1e-4 * loss_o
    assert abs(loss_g - loss_o) <= 1.5 * abs(loss_b - loss_o) + 1e-4 * loss_o
    lay, n = mlp.layout(width, depth, nf)
    assert n == len(g)
    g = g.astype(np.float64)
    rows = []
    for l, (o, shp, ob, nb) in enumerate(lay):
        for a, b in ((o, o + shp[0] * shp[1]), (ob, ob + nb)):
            scale = np.abs(go[a:b]).max()
            e_gpu = np.abs(g[a:b] - go[a:b]).max() / scale
            e_bf = np.abs(gb[a:b] - go[a:b]).max() / scale
            e_emu = np.abs(g[a:b] - gb[a:b]).max() / scale
            rows.append((l, e_gpu, e_bf, e_emu))
    print("per layer (W, b): max |GPU - FP64| / max|g|, BF16 bound, max |GPU - rounded network| / max|g|")
    for r in rows:
        print("  layer %d: %.2e  %.2e  %.2e" % r)
    for l, e_gpu, e_bf, e_emu in rows:
        # the GPU's FP32 sums round a few entries to the other BF16 neighbour than the FP64 sums of the
        # rounded network do; those differences add up layer by layer on the way back from the output
        assert e_emu <= 1e-3 * (depth - l + 1), (l, e_emu)
        assert e_gpu <= 2.0 * e_bf + 1e-3, (l, e_gpu, e_bf)


def test_prediction_batches_agree_bit_for_bit(G):
    """Every point's forward pass is independent of the others, so predicting
    20,000 points at once (the persistent GEMM, BF16 activations only) gives the
    same bits as predicting them 2,000 at a time (the per-tile GEMM)."""
    s = G.Surrogate(0, n_members=2, width=512, depth=6, n_fourier=256, fourier_sigma=2.0, seed=9)
    _, x = _samples(20000, 6)
    y_all, sp_all = s.predict(x)
    parts = [s.predict(x[i:i + 2000]) for i in range(0, len(x), 2000)]
    s.close()
    assert np.all(np.isfinite(y_all))
    assert np.array_equal(y_all, np.concatenate([p[0] for p in parts]))
    assert np.array_equal(sp_all, np.concatenate([p[1] for p in parts]))


def test_training_reduces_loss_and_ensemble_spread(G):
    rng, x = _samples(8192, 5)
    az, el = np.radians(x[:, 0]), np.radians(x[:, 1])
    lf = np.log(x[:, 2] / 1e9)
    y = np.stack([np.cos(az) * np.cos(el), np.sin(2 * az), 0.5 * lf * np.cos(az), np.sin(el + az)], 1)
    s = G.Surrogate(0, n_members=2, width=256, depth=3, n_fourier=128, fourier_sigma=0.3, seed=7)
    loss = s.train(x, y, epochs=100, batch=1024, lr=2e-3)
    assert np.all(loss[:, -1] < 0.05 * loss[:, 0]), loss[:, [0, -1]]
    _, xq = _samples(3000, 6)
    m1, sp1 = s.predict(xq)
    m2, sp2 = s.predict(xq)
    assert np.array_equal(m1, m2) and np.array_equal(sp1, sp2)
    assert np.all(sp1 >= 0) and np.isfinite(m1).all()
    azq, elq = np.radians(xq[:, 0]), np.radians(xq[:, 1])
    yq = np.stack([np.cos(azq) * np.cos(elq), np.sin(2 * azq), 0.5 * np.log(xq[:, 2] / 1e9) * np.cos(azq),
                   np.sin(elq + azq)], 1)
    assert np.sqrt(np.mean((m1 - yq) ** 2)) < 0.1 * np.sqrt(np.mean(yq ** 2))
    s.close()


def test_surrogate_beats_plain_sbr_on_a_converged_patch(G):
    """What the trained network gains over SBR alone: on a sweep patch around nose-on (az 179-181 deg,
    el +-0.5 deg, 1.0-1.1 GHz) with SBR at 40 rays per wavelength (where plain SBR varies well under 0.5 dB
    between ray grids), an ensemble trained on 30k SBR samples answers most held-out points within 0.5 dB of
    plain SBR on the training data's ray grid, at a small fraction of plain SBR's time."""
    import time

    torch = pytest.importorskip("torch")
    import sbr_inputs as S

    xyz, tri = S.aircraft(seed=1)
    with G.Context(0) as c:
        c.load_mesh(xyz, tri)
        off = S.grid_offset(6)
        sp = S.spacing_for(1.1e9, 40.0)
        rng = np.random.default_rng(21)
        reqs = [dict(az=float(rng.uniform(179, 181)), el=float(rng.uniform(-0.5, 0.5)),
                     freqs=np.sort(np.exp(rng.uniform(np.log(1e9), np.log(1.1e9), 100))), spacing=sp)
                for _ in range(300)]
        E, _, _ = c.run_batch(reqs, max_bounces=10, offset=off)
        x = np.concatenate([np.stack([np.full(100, r["az"]), np.full(100, r["el"]), r["freqs"]], 1) for r in reqs])
        Ec = np.concatenate(E)
        y = np.stack([Ec[:, 0].real, Ec[:, 0].imag, Ec[:, 1].real, Ec[:, 1].imag], 1)
        sur = G.Surrogate(0, n_members=2, width=512, depth=6, n_fourier=256, fourier_sigma=16.0, seed=1)
        sur.train(x, y, epochs=60, batch=1024, lr=1e-3)
        hx = np.stack([rng.uniform(179, 181, 500), rng.uniform(-0.5, 0.5, 500),
                       np.exp(rng.uniform(np.log(1e9), np.log(1.1e9), 500))], 1)
        hreq = [dict(az=a, el=e, freqs=np.array([f]), spacing=sp) for a, e, f in hx]
        c.run_batch(hreq[:8], max_bounces=10, offset=off)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, Rh, _ = c.run_batch(hreq, max_bounces=10, offset=off)
        t_sbr = time.perf_counter() - t0
        t0 = time.perf_counter()
        ym, spread = sur.predict(hx)
        t_sur = time.perf_counter() - t0
        sur.close()
    Rh = np.concatenate(Rh)
    Rp = 10 * np.log10(4 * np.pi * np.stack([ym[:, 0] ** 2 + ym[:, 1] ** 2, ym[:, 2] ** 2 + ym[:, 3] ** 2], 1))
    err = np.max(np.abs(Rp - Rh), axis=1)
    served = spread <= 1.0
    print("served", served.mean(), "median error", np.median(err[served]), "within 0.5 dB",
          np.mean(err[served] <= 0.5), "sbr s", t_sbr, "surrogate s", t_sur)
    assert served.mean() >= 0.8
    assert np.median(err[served]) <= 0.5
    assert np.mean(err[served] <= 0.5) >= 0.6
    assert t_sur < 0.25 * t_sbr


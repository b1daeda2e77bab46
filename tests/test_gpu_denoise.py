"""GPU parity of the denoiser (Sec. 4.2 neural denoiser, App. B) through the C ABI.

* one convolution layer (tcgen05, BF16 operands, FP32 accumulation, BF16
  output) against the library FP64 convolution of the same BF16-rounded
  inputs, rounded to BF16: at least 99.5% of outputs bitwise equal, none more
  than 2 units in the last place apart except where the taps cancel, where
  the error stays within 1e-5 of the summed magnitudes conv(|x|, |w|);
* the whole U-Net forward and its input gradient against the oracle
  (PyTorch CPU float64) run with bfloat16 storage at the points where the
  kernels store bfloat16, so that ReLU masks and max-pool winners are decided
  in the same precision: forward rel-L2 <= 1e-2, input gradient <= 6e-2 (rare
  1-ulp differences from FP32 accumulation order compound through the layers);
* and, as the precision statement, against the pure float64 network:
  forward rel-L2 <= 2e-2 (PSNR reported), input gradient <= 0.2;
* at 64 x 64, 48 x 40 and the 2 x 512 x 512 headline launch, the weight
  gradient of the same pass against the oracle's autograd one: per
  convolution, against bfloat16 storage, rel-L2(dW) <= rel-L2(db) + 1e-2 (the
  bias gradient, a plain sum of the stored G, measures G's own difference,
  itself <= 0.2), and both <= 0.35 against the float64 network.
"""
import numpy as np
import pytest
import torch

from oracle import denoise_ref as D

pytestmark = pytest.mark.gpu


def bf16_round(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64)


@pytest.mark.parametrize("cin,cout,H,W,relu", [(16, 32, 16, 8, True), (32, 48, 24, 40, False), (160, 64, 16, 16, True),
                                                (80, 96, 8, 64, True), (16, 16, 4, 256, False), (48, 160, 12, 20, True),
                                                # many tiles: the persistent launch form
                                                (32, 32, 96, 256, True), (112, 48, 64, 200, False),
                                                # 128-pixel row tiles: the row-tile form, one row per tile,
                                                # ragged last tile
                                                (16, 32, 5, 129, True), (160, 64, 6, 130, True),
                                                (96, 96, 10, 384, True), (64, 160, 3, 200, False),
                                                # enough tiles for 4 rows (ragged in x and y) and 2 rows per tile
                                                (32, 48, 238, 200, True), (32, 80, 240, 256, False),
                                                (48, 112, 120, 256, True),
                                                # weights too large for one CTA: 5 slices of 32 output channels
                                                (256, 160, 8, 256, True)])
def test_conv3x3_layer_matches_library(cuda_lib, cin, cout, H, W, relu):
    mcdi = cuda_lib
    rng = np.random.default_rng(cin * 1000 + cout)
    n = 2
    x = bf16_round(rng.normal(size=(n, H, W, cin)))
    w = bf16_round(rng.normal(size=(cout, 3, 3, cin)) / np.sqrt(9 * cin))
    b = torch.from_numpy(rng.normal(size=cout).astype(np.float32))
    dev = "cuda"
    # 8-channel planes [n][C/8][H][W][8]
    planar = lambda t: t.reshape(t.shape[0], t.shape[1], t.shape[2], -1, 8).permute(0, 3, 1, 2, 4).contiguous()
    xg = planar(x.to(torch.bfloat16)).to(dev)
    wg = w.reshape(cout, 9, cin).to(torch.bfloat16).to(dev).contiguous()
    yg = torch.full((n, cout // 8, H, W, 8), float("nan"), dtype=torch.bfloat16, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    mcdi.conv3x3_bf16(xg, wg, b.to(dev), yg, relu, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    yg = yg.permute(0, 2, 3, 1, 4).reshape(n, H, W, cout)
    ref = D.conv3x3(x.permute(0, 3, 1, 2), w.permute(0, 3, 1, 2), b.double())
    if relu:
        ref = torch.relu(ref)
    ref = ref.permute(0, 2, 3, 1)
    # the kernel stores BF16(FP32 accumulation): compare with BF16(FP64 reference) in units in the last place;
    # where the taps cancel (outputs near zero) the FP32 accumulation error is bounded by the magnitude
    # of the summed terms, conv(|x|, |w|), instead
    ref_b = ref.to(torch.bfloat16)
    got_b = yg.cpu()
    assert torch.isfinite(got_b.float()).all()
    ulp = (got_b.view(torch.int16).int() - ref_b.view(torch.int16).int()).abs()
    assert (ulp == 0).float().mean().item() >= 0.995
    mag = D.conv3x3(x.abs().permute(0, 3, 1, 2), w.abs().permute(0, 3, 1, 2), b.double().abs()).permute(0, 2, 3, 1)
    r = ref_b.double().abs().clamp_min(1e-30)
    ulp_size = torch.exp2(torch.floor(torch.log2(r)) - 7)
    assert ((got_b.double() - ref_b.double()).abs() <= 2 * ulp_size + 1e-5 * mag).all()


def make_inputs(rng, n_views, H, W):
    term = np.abs(rng.lognormal(0.0, 0.8, size=(2 * n_views, H, W, 4))).astype(np.float32)
    kd = rng.uniform(0, 1, size=(n_views, H, W, 4)).astype(np.float32)
    nrm = rng.normal(size=(n_views, H, W, 4)).astype(np.float32)
    nrm[..., :3] /= np.linalg.norm(nrm[..., :3], axis=-1, keepdims=True)
    for a in (term, kd, nrm):
        a[..., 3] = 0
    return term, kd, nrm


def oracle_input(term, kd, nrm):
    n = term.shape[0]
    nv = kd.shape[0]
    idx = np.arange(n) % nv
    return D.denoiser_input(term[..., :3], kd[idx, ..., :3], nrm[idx, ..., :3])


@pytest.mark.parametrize("H,W", [(64, 64), (48, 40)])
def test_unet_forward_and_input_gradient_match_oracle(cuda_lib, H, W):
    mcdi = cuda_lib
    rng = np.random.default_rng(H * W)
    term, kd, nrm = make_inputs(rng, 1, H, W)
    weights = D.xavier_weights(5)
    den = mcdi.Denoiser(mcdi.flatten_unet_params(weights), term.shape[0], H, W)
    t = lambda a: torch.from_numpy(a).cuda().contiguous()
    y = torch.zeros(term.shape, device="cuda")
    den.forward(t(term), t(kd), t(nrm), y)
    gy = rng.normal(size=term.shape).astype(np.float32)
    gy[..., 3] = 0
    gx = torch.zeros(term.shape, device="cuda")
    den.backward(t(gy), gx)
    gw = den.weight_grad().cpu().numpy()
    torch.cuda.synchronize()
    assert den.err.item() == 0
    yg = y.cpu().numpy()[..., :3]
    gg = gx.cpu().numpy()[..., :3]
    assert np.isfinite(yg).all() and np.isfinite(gg).all()
    assert np.all(y.cpu().numpy()[..., 3] == 0)
    wres = {}
    res = _compare_with_oracle(term, kd, nrm, gy, yg, gg, weights, ("bf16", None), gw, wres)
    (bf_f, bf_p, bf_b), (f64_f, f64_p, f64_b) = res["bf16"], res[None]
    print(f"denoiser {H}x{W}: vs BF16-storage oracle fwd rel-L2 {bf_f:.2e} ({bf_p:.1f} dB), input-grad rel-L2 "
          f"{bf_b:.2e}; vs float64 network fwd rel-L2 {f64_f:.2e} ({f64_p:.1f} dB), input-grad rel-L2 {f64_b:.2e}")
    # same precision for storage and decisions: only accumulation order differs, and the rare
    # 1-ulp differences it causes compound through the 15 layers
    assert bf_f <= 1e-2 and bf_b <= 6e-2
    # the precision statement: BF16 storage against the float64 network
    assert f64_f <= 2e-2 and f64_b <= 0.2
    # the weight gradient of the same pass (the live-trained denoiser, App. B)
    _check_weight_grad(wres)


def test_denoise_autograd_function_matches_direct_calls(cuda_lib):
    """Denoise.apply inside a torch graph: the forward and the term gradient are exactly
    the direct Denoiser calls; the guides get no gradient (the weights are locked)."""
    mcdi = cuda_lib
    rng = np.random.default_rng(77)
    term, kd, nrm = make_inputs(rng, 1, 32, 48)
    den = mcdi.Denoiser(mcdi.flatten_unet_params(D.xavier_weights(7)), term.shape[0], 32, 48)
    t = lambda a: torch.from_numpy(a).cuda().contiguous()
    x = t(term).requires_grad_(True)
    kd_t, nrm_t = t(kd).requires_grad_(True), t(nrm)
    w = t(rng.normal(size=term.shape).astype(np.float32))
    y = mcdi.Denoise.apply(x, kd_t, nrm_t, den)
    (y * w).sum().backward()
    y_ref, gx_ref = torch.zeros_like(y), torch.zeros_like(y)
    den.forward(t(term), t(kd), t(nrm), y_ref)
    den.backward(w, gx_ref)
    torch.cuda.synchronize()
    assert den.err.item() == 0
    assert torch.equal(y.detach(), y_ref) and torch.equal(x.grad, gx_ref)
    assert kd_t.grad is None


def _run_recorded(mcdi, den, term, kd, nrm, gy):
    t = lambda a: torch.from_numpy(a).cuda().contiguous()
    y = torch.zeros(term.shape, device="cuda")
    gx = torch.zeros(term.shape, device="cuda")
    with mcdi.denoise_plan_recorder() as rec:
        den.forward(t(term), t(kd), t(nrm), y)
        den.backward(t(gy), gx)
    torch.cuda.synchronize()
    assert den.err.item() == 0
    return y.cpu().numpy()[..., :3], gx.cpu().numpy()[..., :3], rec.records


def _compare_with_oracle(term, kd, nrm, gy, yg, gg, weights, storages, gw=None, wres=None):
    """Forward and input-gradient errors per storage; with gw (the GPU's flat weight gradient) also fills
    wres[storage] = {conv: (rel-L2 of dW, rel-L2 of db)} against the oracle's autograd weight gradient."""
    from paper_2206_03380_gb300 import mcdi

    x = oracle_input(term, kd, nrm)
    gyo = torch.from_numpy(gy[..., :3]).permute(0, 3, 1, 2)
    got = mcdi.unflatten_unet_params(np.asarray(gw, np.float64)) if gw is not None else None
    res = {}
    for storage in storages:
        yo, gxo, pg = D.unet_forward_backward(x, weights, gyo, storage=storage)
        yo = yo.permute(0, 2, 3, 1).numpy()
        go = gxo[:, 0:3].permute(0, 2, 3, 1).numpy()
        res[storage] = (D.rel_l2(yg, yo), D.psnr(yg, yo), D.rel_l2(gg, go))
        if got is not None:
            wres[storage] = {k: (D.rel_l2(got[k][0], pg[k][0].numpy()), D.rel_l2(got[k][1], pg[k][1].numpy()))
                             for k in got}
    return res


def _check_weight_grad(wres):
    """The weight-gradient bounds: against the BF16-storage oracle the bias gradient (a plain sum of the
    stored G, another kernel's arithmetic) measures G's own difference, which grows with depth as the
    backward's 1-ulp accumulation-order differences compound through the ReLU masks; dW may add at most the
    forward activations' bound (1e-2) to it.  Sanity caps: G's difference <= 0.2 against the BF16-storage
    oracle, both <= 0.35 against the float64 network."""
    for storage, per in wres.items():
        print(f"weight gradient rel-L2 (dW, db) vs {storage} oracle:",
              {k: tuple(round(v, 4) for v in e) for k, e in per.items()})
    for storage, per in wres.items():
        for name, (eW, eb) in per.items():
            assert np.isfinite(eW) and np.isfinite(eb), (storage, name)
            if storage == "bf16":
                assert eW <= eb + 1e-2 and eb <= 0.2, (name, eW, eb)
            else:
                assert max(eW, eb) <= 0.35, (storage, name, eW, eb)


def test_unet_headline_launch_forward_and_input_gradient(cuda_lib):
    """The benchmark's denoiser launch: the c_d and c_s terms of one 512 x 512 view
    (2 images) with a random upstream gradient, forward and input gradient against the
    oracle; the recorded launch plan must include the row-tile kernels that prefetch the
    ReLU-mask words with 4 and with 2 output rows per tile (the instantiations the
    benchmark times), and the pooling epilogue."""
    mcdi = cuda_lib
    rng = np.random.default_rng(5120)
    term, kd, nrm = make_inputs(rng, 1, 512, 512)
    weights = D.xavier_weights(6)
    den = mcdi.Denoiser(mcdi.flatten_unet_params(weights), 2, 512, 512)
    gy = rng.normal(size=term.shape).astype(np.float32)
    gy[..., 3] = 0
    yg, gg, plan = _run_recorded(mcdi, den, term, kd, nrm, gy)
    gw = den.weight_grad().cpu().numpy()
    torch.cuda.synchronize()
    assert den.err.item() == 0
    assert np.isfinite(yg).all() and np.isfinite(gg).all()
    assert len(plan) == 30 and sum(r["pass"] for r in plan) == 15
    masked_rows = {r["rows"] for r in plan if r["pass"] == 1 and r["mask_prefetch"]}
    assert {2, 4} <= masked_rows, plan
    assert any(r["pool_fused"] for r in plan if r["pass"] == 0)
    wres = {}
    res = _compare_with_oracle(term, kd, nrm, gy, yg, gg, weights, ("bf16", None), gw, wres)
    (bf_f, bf_p, bf_b), (f64_f, f64_p, f64_b) = res["bf16"], res[None]
    print(f"denoiser 2 x 512^2 (plan rows fwd {[r['rows'] for r in plan if r['pass'] == 0]}, bwd "
          f"{[r['rows'] for r in plan if r['pass'] == 1]}): vs BF16-storage oracle fwd rel-L2 {bf_f:.2e} "
          f"({bf_p:.1f} dB), input-grad {bf_b:.2e}; vs float64 network fwd {f64_f:.2e} ({f64_p:.1f} dB), "
          f"input-grad {f64_b:.2e}")
    assert bf_f <= 1e-2 and bf_b <= 6e-2
    assert f64_f <= 2e-2 and f64_b <= 0.2
    _check_weight_grad(wres)


def test_unet_e4m3_forward_and_input_gradient_at_256(cuda_lib):
    """E4M3 at 256 x 256 over two views (4 images): enough row tiles for the masked
    input-gradient convolutions to run with 4 and 2 rows per tile."""
    mcdi = cuda_lib
    rng = np.random.default_rng(2560)
    term, kd, nrm = make_inputs(rng, 2, 256, 256)
    weights = D.xavier_weights(5)
    den = mcdi.Denoiser(mcdi.flatten_unet_params(weights), term.shape[0], 256, 256, precision=mcdi.E4M3)
    gy = rng.normal(size=term.shape).astype(np.float32)
    gy[..., 3] = 0
    yg, gg, plan = _run_recorded(mcdi, den, term, kd, nrm, gy)
    assert np.isfinite(yg).all() and np.isfinite(gg).all()
    assert all(r["e4m3"] for r in plan) and len(plan) == 30
    masked_rows = {r["rows"] for r in plan if r["pass"] == 1 and r["mask_prefetch"]}
    assert {2, 4} <= masked_rows, plan
    res = _compare_with_oracle(term, kd, nrm, gy, yg, gg, weights, ("e4m3", None))
    (q_f, q_p, q_b), (f_f, f_p, f_b) = res["e4m3"], res[None]
    print(f"denoiser E4M3 4 x 256^2: vs E4M3-storage oracle fwd rel-L2 {q_f:.2e} ({q_p:.1f} dB), input-grad "
          f"{q_b:.2e}; vs float64 network fwd {f_f:.2e} ({f_p:.1f} dB), input-grad {f_b:.2e}")
    assert q_f <= 6e-2 and q_b <= 0.2
    assert f_f <= 0.25 and f_b <= 0.6


def test_unet_forward_at_headline_size(cuda_lib):
    """512 x 512, the two terms of one view (the benchmark's denoiser launch), forward only."""
    mcdi = cuda_lib
    rng = np.random.default_rng(512)
    term, kd, nrm = make_inputs(rng, 1, 512, 512)
    weights = D.xavier_weights(6)
    den = mcdi.Denoiser(mcdi.flatten_unet_params(weights), 2, 512, 512)
    t = lambda a: torch.from_numpy(a).cuda().contiguous()
    y = torch.zeros(term.shape, device="cuda")
    den.forward(t(term), t(kd), t(nrm), y)
    torch.cuda.synchronize()
    assert den.err.item() == 0
    yo = D.unet_forward(oracle_input(term, kd, nrm), weights, storage="bf16").permute(0, 2, 3, 1).numpy()
    e = D.rel_l2(y.cpu().numpy()[..., :3], yo)
    print(f"denoiser 512x512 forward vs BF16-storage oracle rel-L2 {e:.2e}")
    assert e <= 1e-2


# ------------------------------------------------------------------ E4M3 (FP8) path
def _random_e4m3_codes(rng, shape):
    """Uniform over the finite E4M3 codes (0x7F / 0xFF are NaN)."""
    c = rng.integers(0, 256, size=shape).astype(np.uint8)
    c[(c & 0x7F) == 0x7F] = 0x7E
    return torch.from_numpy(c)


@pytest.mark.parametrize("cin,cout,H,W,relu", [(32, 32, 16, 8, True), (96, 48, 12, 40, False),
                                                (32, 80, 48, 256, True), (160, 64, 6, 130, True),
                                                (64, 48, 64, 200, False)])
def test_conv3x3_e4m3_layer_matches_library(cuda_lib, cin, cout, H, W, relu):
    """E4M3 operands, FP32 accumulation, rescaled by (amax_x / 448)(amax_w / 448): against the float64
    convolution of the decoded operands."""
    mcdi = cuda_lib
    rng = np.random.default_rng(cin * 7 + cout)
    n = 2
    xc = _random_e4m3_codes(rng, (n, cin // 16, H, W, 16))
    wc = _random_e4m3_codes(rng, (cout, 9, cin))
    x_amax, w_amax = 3.5, 0.0625
    dec = lambda c: c.view(torch.float8_e4m3fn).to(torch.float64)
    x = dec(xc).permute(0, 1, 4, 2, 3).reshape(n, cin, H, W) * (x_amax / 448)
    w = dec(wc).reshape(cout, 3, 3, cin).permute(0, 3, 1, 2) * (w_amax / 448)
    b = torch.from_numpy(rng.normal(size=cout).astype(np.float32))
    dev = "cuda"
    yg = torch.full((n, cout // 8, H, W, 8), float("nan"), dtype=torch.bfloat16, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    amx = torch.tensor([x_amax], device=dev)
    amw = torch.tensor([w_amax], device=dev)
    mcdi.conv3x3_e4m3(xc.to(dev), wc.to(dev), amx, amw, b.to(dev), yg, relu, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    got = yg.permute(0, 2, 3, 1, 4).reshape(n, H, W, cout).cpu().double()
    ref = D.conv3x3(x, w, b.double())
    if relu:
        ref = torch.relu(ref)
    ref = ref.permute(0, 2, 3, 1)
    mag = D.conv3x3(x.abs(), w.abs(), b.double().abs()).permute(0, 2, 3, 1)
    assert torch.isfinite(got).all()
    # BF16 store of the FP32 result: half an ulp of BF16 plus the FP32 accumulation bound
    tol = ref.abs() * 2.0 ** -8 + 1e-5 * mag
    assert ((got - ref).abs() <= tol).all(), float(((got - ref).abs() - tol).max())


@pytest.mark.parametrize("H,W", [(64, 64), (48, 136)])
def test_unet_e4m3_forward_and_input_gradient(cuda_lib, H, W):
    mcdi = cuda_lib
    rng = np.random.default_rng(H * W + 8)
    term, kd, nrm = make_inputs(rng, 1, H, W)
    weights = D.xavier_weights(5)
    den = mcdi.Denoiser(mcdi.flatten_unet_params(weights), term.shape[0], H, W, precision=mcdi.E4M3)
    t = lambda a: torch.from_numpy(a).cuda().contiguous()
    y = torch.zeros(term.shape, device="cuda")
    den.forward(t(term), t(kd), t(nrm), y)
    gy = rng.normal(size=term.shape).astype(np.float32)
    gy[..., 3] = 0
    gx = torch.zeros(term.shape, device="cuda")
    den.backward(t(gy), gx)
    torch.cuda.synchronize()
    assert den.err.item() == 0
    x = oracle_input(term, kd, nrm)
    gyo = torch.from_numpy(gy[..., :3]).permute(0, 3, 1, 2)
    yg, gg = y.cpu().numpy()[..., :3], gx.cpu().numpy()[..., :3]
    assert np.isfinite(yg).all() and np.isfinite(gg).all()
    res = {}
    for storage in ("e4m3", "bf16", None):
        yo, gxo, _ = D.unet_forward_backward(x, weights, gyo, storage=storage)
        yo = yo.permute(0, 2, 3, 1).numpy()
        go = gxo[:, 0:3].permute(0, 2, 3, 1).numpy()
        res[storage] = (D.rel_l2(yg, yo), D.psnr(yg, yo), D.rel_l2(gg, go))
    (q_f, q_p, q_b), (f_f, f_p, f_b) = res["e4m3"], res[None]
    print(f"denoiser E4M3 {H}x{W}: vs E4M3-storage oracle fwd rel-L2 {q_f:.2e} ({q_p:.1f} dB), input-grad rel-L2 "
          f"{q_b:.2e}; vs float64 network fwd rel-L2 {f_f:.2e} ({f_p:.1f} dB), input-grad rel-L2 {f_b:.2e}")
    # same quantiser on both sides: differences come from FP32 accumulation order flipping BF16 roundings
    # and, through them, E4M3 codes (one flipped code moves its value by 1/8 of a binade step);
    # measured 8.5e-4 - 3.3e-2 forward, 1.3e-2 - 8.4e-2 input gradient
    assert q_f <= 6e-2 and q_b <= 0.2
    # the precision statement of the FP8 path against the float64 network: 3 mantissa bits per operand
    # through 15 layers; measured 0.145 forward (32 - 36 dB), 0.39 input gradient
    assert f_f <= 0.25 and f_b <= 0.6

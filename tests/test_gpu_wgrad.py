"""GPU parity of the denoiser's weight gradient (the live-trained denoiser of
App. B; the tcgen05 kernels of wgrad.cu) through the C ABI.

* one layer: dW[co][ci][ky][kx] = sum over pixels of g[co](p) x[ci](p + tap)
  and db = sum of g, from BF16 x and g, against the float64 sum of the same
  BF16 values.  The kernel's products are exact and its sums FP32, so every
  entry lies within n_terms * 2^-23 of sum |g x| (the worst case of any
  summation order with truncating adds); a transposed operand, a wrong tap
  or a dropped pixel breaks this by O(1).  Shapes cover ragged row segments
  (W not a multiple of 128), padding channels (cin < cin_pad, cout <
  cout_pad), one to four M groups of up to 5 input planes (one per CTA),
  one and two MMA chains on N = 3 cout, segment widths 128, 64 and 32;
  the result is bitwise repeatable;
* the whole U-Net: gw of all 15 convolutions after a forward and input
  gradient against the oracle (PyTorch CPU float64 autograd) with bfloat16
  storage.  The stored gradients G differ from the oracle's by the 1-ulp
  accumulation-order differences that compound through the backward (as for
  the input gradient), most at the bottleneck where fewest pixels average
  them out; the bias gradient, a plain sum of G, measures exactly that
  difference.  So per convolution: rel-L2(dW) <= rel-L2(db) + 1e-2 (the
  forward activations' own bound), with G's difference itself <= 0.2;
  against the float64 network both <= 0.35 (the precision statement).
"""
import numpy as np
import pytest
import torch

from oracle import denoise_ref as D

pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16)


def planar(t):
    """(n, H, W, C) -> (n, C/8, H, W, 8) contiguous."""
    n, H, W, C = t.shape
    return t.reshape(n, H, W, C // 8, 8).permute(0, 3, 1, 2, 4).contiguous()


def wgrad_reference(x, g):
    """float64 dW (co, ci, 3, 3), db (co,) and the magnitude sums, from (n, H, W, C) tensors."""
    n, H, W, ci = x.shape
    xp = torch.zeros(n, H + 2, W + 2, ci, dtype=torch.float64)
    xp[:, 1:-1, 1:-1] = x
    co = g.shape[-1]
    dW = torch.zeros(co, ci, 3, 3, dtype=torch.float64)
    mag = torch.zeros(co, ci, 3, 3, dtype=torch.float64)
    gf = g.reshape(-1, co)
    for ky in range(3):
        for kx in range(3):
            sh = xp[:, ky:ky + H, kx:kx + W].reshape(-1, ci)
            dW[:, :, ky, kx] = gf.T @ sh
            mag[:, :, ky, kx] = gf.abs().T @ sh.abs()
    return dW, gf.sum(0), mag, gf.abs().sum(0)


@pytest.mark.parametrize("cin,cin_pad,cout,cout_pad,n,H,W", [
    (9, 16, 32, 32, 2, 16, 40),       # the first layer's shape, one ragged segment
    (32, 32, 3, 16, 2, 12, 264),      # the last layer's shape, segments 128 + 128 + 8
    (41, 48, 29, 32, 1, 20, 130),     # padding channels on both sides, segments 128 + 2
    (112, 112, 48, 48, 2, 9, 136),    # three M groups of 5, 5, 4 planes
    (160, 160, 64, 64, 2, 8, 72),     # four M groups
    (96, 96, 96, 96, 1, 24, 64),      # three M groups, the widest accumulators
    (64, 64, 96, 96, 1, 6, 256),      # N = 3 x 96 above 256: two MMA chains
    (16, 16, 80, 80, 2, 5, 24),       # N = 240, one chain; W below every segment width
    (8, 8, 16, 16, 3, 300, 8),        # narrow images, many rows per CTA
    (128, 128, 16, 16, 1, 10, 40),    # a last M group of one plane
    (120, 128, 20, 32, 2, 7, 200),    # the same with padding channels
])
def test_conv3x3_wgrad_matches_float64(cuda_lib, cin, cin_pad, cout, cout_pad, n, H, W):
    mcdi = cuda_lib
    rng = np.random.default_rng(cin * 7919 + cout * 31 + W)
    x = torch.zeros(n, H, W, cin_pad)
    x[..., :cin] = torch.from_numpy(rng.normal(size=(n, H, W, cin)).astype(np.float32))
    g = torch.zeros(n, H, W, cout_pad)
    g[..., :cout] = torch.from_numpy(rng.normal(size=(n, H, W, cout)).astype(np.float32))
    # padding channels hold garbage on purpose: the kernel must not let them reach real entries
    x[..., cin:] = 1e30
    g[..., cout:] = 1e30
    xb, gb = bf16(x), bf16(g)
    dev = "cuda"
    xg, gg = planar(xb).to(dev), planar(gb).to(dev)
    scratch = torch.empty(mcdi.conv3x3_wgrad_bytes(n, H, W, cin_pad, cout_pad), dtype=torch.uint8, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    n_out = cout * cin * 9 + cout
    gw = torch.full((n_out,), float("nan"), device=dev)
    mcdi.conv3x3_wgrad(xg, gg, cin, cout, gw, scratch, err)
    gw2 = torch.full((n_out,), float("nan"), device=dev)
    mcdi.conv3x3_wgrad(xg, gg, cin, cout, gw2, scratch, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    got = gw.cpu().double()
    assert torch.equal(gw.cpu(), gw2.cpu())  # fixed reduction order
    dW, db, mag, magb = wgrad_reference(xb[..., :cin].double(), gb[..., :cout].double())
    n_terms = n * H * W
    bound = n_terms * 2.0 ** -23
    gW = got[:cout * cin * 9].reshape(cout, cin, 3, 3)
    gB = got[cout * cin * 9:]
    assert torch.isfinite(got).all()
    assert ((gW - dW).abs() <= bound * mag + 1e-30).all(), (gW - dW).abs().div(mag + 1e-30).max()
    assert ((gB - db).abs() <= bound * magb + 1e-30).all()
    # the bound is loose; the typical error of FP32 sums is far smaller
    assert ((gW - dW).abs() / (mag + 1e-30)).median() < 1e-5


def make_inputs(rng, H, W):
    term = np.abs(rng.lognormal(0.0, 0.8, size=(2, H, W, 4))).astype(np.float32)
    kd = rng.uniform(0, 1, size=(1, H, W, 4)).astype(np.float32)
    nrm = rng.normal(size=(1, H, W, 4)).astype(np.float32)
    nrm[..., :3] /= np.linalg.norm(nrm[..., :3], axis=-1, keepdims=True)
    for a in (term, kd, nrm):
        a[..., 3] = 0
    return term, kd, nrm


def test_unet_weight_gradient_matches_oracle(cuda_lib):
    mcdi = cuda_lib
    H, W = 48, 136  # level widths 136, 68, 34, 17 px: ragged segments at full resolution
    rng = np.random.default_rng(2024)
    term, kd, nrm = make_inputs(rng, H, W)
    weights = D.xavier_weights(9)
    den = mcdi.Denoiser(mcdi.flatten_unet_params(weights), term.shape[0], H, W)
    t = lambda a: torch.from_numpy(a).cuda().contiguous()
    y = torch.zeros(term.shape, device="cuda")
    den.forward(t(term), t(kd), t(nrm), y)
    gy = rng.normal(size=term.shape).astype(np.float32)
    gy[..., 3] = 0
    gx = torch.zeros(term.shape, device="cuda")
    den.backward(t(gy), gx)
    gw = den.weight_grad()
    gw2 = den.weight_grad()
    torch.cuda.synchronize()
    assert den.err.item() == 0
    assert torch.equal(gw, gw2)
    got = mcdi.unflatten_unet_params(gw.cpu().double())
    x = D.denoiser_input(term[..., :3], kd[[0, 0], ..., :3], nrm[[0, 0], ..., :3])
    gyo = torch.from_numpy(gy[..., :3]).permute(0, 3, 1, 2)
    worst = {}
    for storage, tol in (("bf16", 6e-2), (None, 0.2)):
        _, _, pg = D.unet_forward_backward(x, weights, gyo, storage=storage)
        for name, _, _ in mcdi.UNET_PLAN:
            gW, gb = got[name]
            oW, ob = pg[name]
            assert torch.isfinite(gW).all() and torch.isfinite(gb).all()
            e = (D.rel_l2(gW.numpy(), oW.numpy()), D.rel_l2(gb.numpy(), ob.numpy()))
            worst[(storage, name)] = e
    for st in ("bf16", None):
        print(f"weight-gradient rel-L2 vs {st} oracle (W, b):",
              {k[1]: tuple(round(v, 5) for v in e) for k, e in worst.items() if k[0] == st})
    for (storage, name), (eW, eb) in worst.items():
        if storage == "bf16":
            # the bias gradient is the plain sum of the stored G: its error is G's; the weight gradient
            # may add no more than the forward activations' own bound (1e-2)
            assert eW <= eb + 1e-2 and eb <= 0.2, (name, eW, eb)
        else:
            assert max(eW, eb) <= 0.35, (name, eW, eb)

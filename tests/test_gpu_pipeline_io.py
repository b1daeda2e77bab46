"""The optimisation step with its host I/O inside one captured graph
(pipeline.loss_step_io): uploads on copy streams that each stage waits for
only as far as it reads them, read-backs as soon as their producer has run.
The host outputs of a replay equal, bit for bit, those of the plain step on
the same inputs (the probe gradient, summed by atomics, to 1e-5 of its
largest entry), after the device copies of the inputs were overwritten (so
the graph's uploads are what the step read)."""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("packed_textures", [False, True])
def test_loss_step_io_graph_matches_the_plain_step(cuda_lib, packed_textures):
    from paper_2206_03380_gb300.pipeline import ShadingPipeline

    sc = scenes.parity_scene()
    den = cuda_lib.flatten_unet_params(scenes.unet_xavier_weights(scenes.BASE_SEED + 3))
    pipe = ShadingPipeline(sc, denoiser_params=den)
    rng = np.random.default_rng(31)
    ref = torch.from_numpy(np.abs(rng.normal(size=(1, sc.height, sc.width, 4))).astype(np.float32)).cuda()
    pipe.loss_step(ref)
    torch.cuda.synchronize()
    outs = [pipe.loss, pipe.color, pipe.g_kd, pipe.g_korm, pipe.g_nrm, pipe.g_env]
    expect = [t.cpu().clone() for t in outs]
    names = ("verts", "vnrm", "tris", "env", "tex_kd", "tex_korm")
    host_in = {k: getattr(pipe, k).cpu().pin_memory() for k in names}
    if packed_textures:  # (S, S, 3): the 4th channel is padding
        for k in ("tex_kd", "tex_korm"):
            host_in[k] = host_in[k][..., :3].contiguous().pin_memory()
    host_ref = ref.cpu().pin_memory()
    host_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
    pipe.capture_loss_step_io(ref, host_in, host_ref, list(zip(outs, host_out)))
    torch.cuda.synchronize()
    for k in names:
        getattr(pipe, k).zero_()
    ref.zero_()
    for t in outs:
        t.zero_()
    for h in host_out:
        h.fill_(float("nan") if h.is_floating_point() else 0)
    torch.cuda.synchronize()
    for _ in range(2):
        pipe.replay_io()
        torch.cuda.synchronize()
        for e, h in zip(expect[:-1], host_out[:-1]):
            assert torch.equal(e, h)
        # the probe gradient is summed by atomics, in no fixed order
        torch.testing.assert_close(host_out[-1], expect[-1], rtol=0, atol=1e-5 * float(expect[-1].abs().max()))
    assert float(expect[0][0]) > 0 and float(expect[2].abs().max()) > 0

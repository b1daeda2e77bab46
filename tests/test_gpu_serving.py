"""The serving loop: requests of uneven resolution and spp against resident
scenes, continuous batching over several streams vs one at a time; every
request's image is bitwise the same alone and in the mix (per-request Philox
seeds, deterministic kernels, the same captured denoiser graph whichever slot
runs it), and admission respects the HBM budget."""
import numpy as np
import pytest
import torch

from paper_2206_03380_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine(cuda_lib):
    from paper_2206_03380_gb300.serving import ServingEngine

    sc = scenes.serving_scenes(n_scenes=4, grids=(32, 48), tex=64)
    pr = scenes.serving_probes(n_probes=3)
    den = cuda_lib.flatten_unet_params(scenes.unet_xavier_weights(scenes.BASE_SEED + 3))
    return ServingEngine(sc, pr, den, n_slots=3, hbm_budget=2 << 30, sides=range(64, 193, 32), max_spp=16)


def test_continuous_batching_matches_alone_and_serial(engine):
    reqs = scenes.poisson_requests(24, 400.0, 4, 3, seed=11, res_range=(64, 192), spp_choices=(4, 8, 16),
                                   n_views=200)
    ids = [r.rid for r in reqs]
    mix = engine.run(reqs, mode="continuous", keep=ids)
    lanes = engine.run(reqs, mode="continuous", keep=ids, lanes=(64 * 64 * 8,))
    ser = engine.run(reqs, mode="serial", keep=ids)
    assert mix["n"] == ser["n"] == lanes["n"] == len(reqs)
    for r in reqs:
        alone = engine.render_one(r)
        assert np.isfinite(alone).all()
        np.testing.assert_array_equal(mix["images"][r.rid], alone)
        np.testing.assert_array_equal(lanes["images"][r.rid], alone)
        np.testing.assert_array_equal(ser["images"][r.rid], alone)
    assert mix["p99_ms"] >= mix["p50_ms"] > 0
    # images are not trivial: lit, covered pixels exist
    assert any(np.abs(mix["images"][i]).max() > 0 for i in ids)


def test_admission_waits_for_memory(engine):
    reqs = scenes.poisson_requests(6, 1e6, 4, 3, seed=12, res_range=(128, 128), spp_choices=(8,))
    need = engine.footprint(reqs[0])
    saved = engine.hbm_budget
    engine.hbm_budget = int(1.5 * need)  # room for one request at a time
    try:
        out = engine.run(reqs, mode="continuous")
    finally:
        engine.hbm_budget = saved
    assert out["n"] == 6 and out["admission_waits"] > 0

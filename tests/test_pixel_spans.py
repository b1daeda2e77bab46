"""The adjoint's pixel spans in the end-to-end step (pipeline.pixel_spans):
consecutive, disjoint, covering every pixel exactly once, each cut at a
multiple of 32 pixels (one adjoint block) except where the pixels run out.
Host logic only."""
import pytest

from paper_2206_03380_gb300.pipeline import pixel_spans


@pytest.mark.parametrize("P", [1, 31, 32, 33, 1000, 512 * 512, 3 * 800 * 800 + 7])
@pytest.mark.parametrize("fractions", [(None,), (0.5, None), (0.4, 0.3, 0.2, None), (0.9, 0.3, None),
                                       (0.0, 0.5, None)])
def test_spans_cover_every_pixel_once(P, fractions):
    spans = pixel_spans(P, fractions)
    assert len(spans) == len(fractions)
    pos = 0
    for first, count in spans:
        assert first == pos and count >= 0
        pos += count
    assert pos == P
    for (first, count), frac in zip(spans[:-1], fractions[:-1]):
        assert count % 32 == 0 or first + count == P  # cut at a block boundary unless the pixels ran out
        assert abs(count - P * frac) <= 16 or first + count == P

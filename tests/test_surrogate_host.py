"""Host-side choices of the surrogate's served path (no GPU needed)."""
from paper_2609_14831_b300.surrogate import Surrogate


def test_fallback_tile_is_the_narrowest_that_fits_the_sms():
    # a CTA of tile T holds T instances: 148 SMs take 296 instances at tile 2,
    # 592 at tile 4; beyond that the full-batch width 8
    assert [Surrogate.fallback_tile(c) for c in (1, 296, 297, 592, 593, 4096)] == [2, 2, 4, 4, 8, 8]
    assert Surrogate.fallback_tile(100, sms=10) == 8


def test_plain_flows_only_below_the_batched_fallback_cost():
    # 15 plain flows (38 ms each) cost about one tile-2 batched fallback (0.58 s)
    assert 10 <= Surrogate.plain_max <= 20

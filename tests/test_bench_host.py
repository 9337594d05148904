"""Host logic of bench.py that needs no GPU: the ncu traffic figures are
given only for a run in the launch configuration they were captured in."""

import bench


def test_traffic_only_for_the_captured_configuration():
    cfg = {"k": 2, "plain_zchunk": 64, "plain_ctas": 256, "blocked_ctas": 150, "blocked_zsplit": 3,
           "blocked_order": 1, "blocked_rows": 4}
    v, caps = bench.ncu_traffic("yee_blocked", 2, cfg)
    assert v == bench.NCU_TRAFFIC[("yee_blocked", 2)][0][1]
    assert {"blocked_ctas": 150, "blocked_rows": 4} in caps
    v2, _ = bench.ncu_traffic("yee_blocked", 2, dict(cfg, blocked_rows=2))
    assert v2 == bench.NCU_TRAFFIC[("yee_blocked", 2)][1][1]
    assert bench.ncu_traffic("yee_blocked", 2, dict(cfg, blocked_ctas=152))[0] is None
    assert bench.ncu_traffic("yee_blocked", 6, cfg) == (None, [])
    assert bench.ncu_traffic("yee_plain", 1, {})[0] is None


def test_every_capture_is_a_plausible_launch():
    """Each kept figure lies between the algorithmic bytes of a 256^3 launch
    (16.78 M cells x 49 B) and twice the 52 B the layout moves."""
    cells = 256 ** 3
    for entries in bench.NCU_TRAFFIC.values():
        for cfg, v in entries:
            assert cells * bench.ALG_BYTES <= v <= 2 * cells * bench.LAYOUT_BYTES, (cfg, v)

"""The DRAM traffic the bench reports for its dominant kernel comes from a
committed ncu summary (a `bench-traffic:` line under profiles/) keyed by a hash
of the hopping-kernel sources: an edit of those sources without a new capture
makes the bench report null traffic. This test fails first."""


def test_committed_traffic_matches_kernel_sources():
    import bench

    b = bench.committed_traffic("k_dslash<single,dhop_xpay>", "32^3x64")
    assert b is not None
    # the capture is of the 960 B/site fused kernel at V/2 = 1 048 576: close to its algorithmic bytes
    assert 0.9 < b / (960 * 1048576) < 1.1

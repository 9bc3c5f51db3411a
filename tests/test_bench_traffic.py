"""The DRAM traffic the bench reports for its dominant kernel comes from a
committed ncu summary (a `bench-traffic:` line under profiles/) keyed by a hash
of the hopping-kernel sources: an edit of those sources without a new capture
makes the bench report null traffic. This test fails first."""


def test_committed_traffic_matches_kernel_sources():
    import bench

    # the bench's dominant kernels of the 32^3x64 mixed CG, with their algorithmic bytes per site
    for tag, site_bytes in (("k_dslash<single,dhop_clovinv>", 864), ("k_dslash_cg<single,cg_mhat_norms>", 960),
                            ("k_dslash_cg<single,cg_mhatdag_update>", 960 + 384)):
        b = bench.committed_traffic(tag, "32^3x64")
        assert b is not None, tag
        # captured at V/2 = 331 776 and scaled to 1 048 576: close to the algorithmic bytes
        assert 0.9 < b / (site_bytes * 1048576) < 1.1, tag

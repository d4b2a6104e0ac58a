"""Host logic of the autotuner (no GPU): its list of compiled launch shapes is
the kernel's, and every rank the C ABI accepts has candidates that cover a
whole row."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def autotune():
    from paper_1906_01687_gb300 import build
    build.build()
    from paper_1906_01687_gb300 import autotune as at
    return at


def kernel_configs():
    src = open(os.path.join(ROOT, "paper_1906_01687_gb300", "csrc", "gcp_grad_impl.cuh")).read()
    body = re.search(r"#define GCP_GRAD_CONFIGS\(X\)\s*\\\s*\n(.*?)\n\n", src, flags=re.S).group(1)
    return [(int(a), int(b)) for a, b in re.findall(r"X\((\d+),\s*(\d+)\)", body)]


def test_compiled_shapes_are_the_kernels(autotune):
    assert sorted(autotune.COMPILED) == sorted(kernel_configs())


def test_every_rank_has_covering_candidates(autotune):
    for rank in range(1, 257):
        chunks = (rank + 3) // 4
        shapes = autotune.candidate_shapes(rank)
        assert shapes, rank
        assert all(L * NC >= chunks for L, NC in shapes), rank
        cands = autotune.candidates(rank)
        assert all((c["lanes"], c["chunks"]) in shapes for c in cands)
        # the prefetch layout only where it is compiled: one chunk per lane, 2 or 4 lanes
        assert all(c["lanes"] in (2, 4) and c["chunks"] == 1 for c in cands if c.get("prefetch") == 1)
        # the staged walk where it is compiled: one chunk per lane, at most 8 lanes
        assert all(c["lanes"] <= 8 and c["chunks"] == 1 for c in cands if c.get("prefetch") == 2)
        assert all(c["block"] % 32 == 0 and c["block"] <= 256 for c in cands)


def test_grid_variants_fit_the_draws(autotune):
    cands = autotune.with_grids([dict(lanes=4, chunks=1, block=128), dict(lanes=4, chunks=1, block=256, group_draws=1)],
                                100_000)
    assert len(cands) == 4 and "grid_blocks" not in cands[0]
    assert cands[1]["grid_blocks"] == -(-(-(-100_000 // 32)) // 4)   # 3125 warps, 4 per block
    assert cands[3]["grid_blocks"] == -(-(-(-100_000 // 8)) // 8)    # group draws: 8 per warp, 8 warps per block

"""Host logic of the library's plan (no GPU: fifa_plan_describe runs on the host).

* the tree (a1): the library's bounds equal the oracle's tree node by node,
  bit for bit, for ragged and power-of-two n and several leaf sizes;
* the ACA work list: every off-diagonal block appears exactly once, in the
  grouped part with its G CTAs numbered 0..G-1 in a row (G >= 2, all grouped
  CTAs within the co-resident budget), in the warp-per-block part exactly when
  its node spans at most 256 rows, otherwise one CTA per block;
* the level kernels' CTA groups: a level gets groups (G > 1) only if its rows
  give each CTA of a group at least 512 (256 for n <= 2^15) and all groups of
  the level are co-resident (nodes x G <= the bucket's budget);
* independent CTAs: no groups anywhere.
"""
import os
import shutil

import numpy as np
import pytest

from oracle.tree import Tree

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available to build the library")

CASES = [(1, 64), (65, 64), (1000, 37), (2048, 64), (20000, 64), (131071, 32), (1 << 20, 32)]
BUDGET = dict(aca=608, lvl=(608, 456, 152))  # co-resident CTAs of GB300-sized kernels


@pytest.fixture(scope="module")
def fifa():
    from paper_2006_06537_gb300 import build

    build.build()
    from paper_2006_06537_gb300 import fifa as f

    return f


def _opts(fifa, B, indep=0):
    return fifa.fifa_opts(B, 1e-10, 32, fifa.FIFA_FP64, 1e-12, 3, indep)


@pytest.mark.parametrize("n,B", CASES)
def test_tree_bounds_match_the_oracle(fifa, n, B):
    d = fifa.fifa_plan_describe(_opts(fifa, B), n, BUDGET["aca"], BUDGET["lvl"])
    t = Tree(n, B)
    L = d["info"].levels
    assert L == t.L and d["info"].nleaf == 2 ** L
    b = d["bounds"]
    for lvl in range(L):
        off = (1 << lvl) - 1 + lvl
        offc = (1 << (lvl + 1)) - 1 + lvl + 1
        for i in range(1 << lvl):
            s, h, e = t.node(lvl, i)
            assert (b[off + i], b[off + i + 1], b[offc + 2 * i + 1]) == (s, e, h), (lvl, i)
    offl = (1 << L) - 1 + L
    leaves = t.leaves()
    assert [(b[offl + i], b[offl + i + 1]) for i in range(len(leaves))] == [tuple(x) for x in leaves]
    assert d["info"].leaf_max == max(e - s for s, e in leaves)


@pytest.mark.parametrize("n,B", CASES)
def test_aca_work_list_covers_every_block_once(fifa, n, B):
    d = fifa.fifa_plan_describe(_opts(fifa, B), n, BUDGET["aca"], BUDGET["lvl"])
    info, w, b = d["info"], d["work"], d["bounds"]
    L = info.levels
    ng, ns, nw = info.aca_grouped_ctas, info.aca_solo_blocks, info.aca_warp_blocks
    assert len(w) == ng + ns + nw and ng <= BUDGET["aca"]
    seen = {}
    k = 0
    while k < ng:  # grouped blocks: G consecutive CTAs g = 0..G-1
        lvl, i, g, G = w[k]
        assert G >= 2 and g == 0
        assert [tuple(r) for r in w[k:k + G]] == [(lvl, i, q, G) for q in range(G)]
        seen[(lvl, i)] = "grouped"
        k += G
    for lvl, i, g, G in w[ng:ng + ns]:
        assert (g, G) == (0, 1) and (lvl, i) not in seen
        seen[(lvl, i)] = "cta"
    for lvl, i, g, G in w[ng + ns:]:
        assert (g, G) == (0, 1) and (lvl, i) not in seen
        seen[(lvl, i)] = "warp"
    assert set(seen) == {(lvl, i) for lvl in range(L) for i in range(1 << lvl)}
    for (lvl, i), kind in seen.items():
        off = (1 << lvl) - 1 + lvl
        span = b[off + i + 1] - b[off + i]
        if kind != "grouped":
            assert (kind == "warp") == (span <= 256), (lvl, i, span, kind)


@pytest.mark.parametrize("n,B", CASES)
def test_level_groups_are_co_resident(fifa, n, B):
    d = fifa.fifa_plan_describe(_opts(fifa, B), n, BUDGET["aca"], BUDGET["lvl"])
    L = d["info"].levels
    G = d["groups"]
    for bkt in range(3):
        for lvl in range(L):
            g = G[bkt, lvl]
            nodes = 1 << lvl
            span = (n + nodes - 1) // nodes
            assert g >= 1
            if g > 1:
                per = 256 if n <= 32768 else 512
                assert nodes * g <= BUDGET["lvl"][bkt] and span // g >= per and 2 * nodes <= BUDGET["lvl"][bkt]


@pytest.mark.parametrize("n,B", CASES)
def test_level_groups_cover_a_prefix_of_top_levels(fifa, n, B):
    # the overlapped chain iteration splits a factorization at the deepest
    # grouped level: everything below runs with independent CTAs, so in every
    # rank bucket the grouped levels must be exactly levels 0 .. k-1
    d = fifa.fifa_plan_describe(_opts(fifa, B), n, BUDGET["aca"], BUDGET["lvl"])
    G = d["groups"]
    for bkt in range(3):
        grouped = [int(G[bkt, lvl]) > 1 for lvl in range(d["info"].levels)]
        k = sum(grouped)
        assert grouped == [True] * k + [False] * (len(grouped) - k), (bkt, grouped)


def test_independent_ctas_have_no_groups(fifa):
    d = fifa.fifa_plan_describe(_opts(fifa, 32, indep=1), 1 << 20, BUDGET["aca"], BUDGET["lvl"])
    assert d["info"].aca_grouped_ctas == 0
    assert np.all(d["groups"] == 1)


def test_bad_arguments(fifa):
    with pytest.raises(fifa.FifaError) as e:
        fifa.fifa_plan_describe(_opts(fifa, 32), 0, 608, (608, 456, 152))
    assert e.value.code == fifa.FIFA_ERR_INVALID_ARG
    with pytest.raises(fifa.FifaError):
        fifa.fifa_plan_describe(_opts(fifa, 32), 1000, 608, (608, 0, 152))

"""The mutual passes' work plan, checked on the host (no GPU): every pair of
64-body groups of a system visited exactly once (both orders inside an
i-block, once across blocks), items inside their system and its groups that
hold bodies, and each block's partial rows exactly those its combine reads,
each written by one item -- for single systems of ragged sizes and for
batches, in the shapes of the mutual variants."""
import pytest

SHAPES = [(12, 2), (8, 4)]          # consumer warps, packed i-registers (groups) per warp


@pytest.fixture(scope="module")
def genga():
    """The binding with the library built and loaded; these calls touch no device."""
    import paper_2309_08217_gb300 as g
    g.build()
    g.load()
    return g


@pytest.mark.parametrize("cw,npg", SHAPES)
@pytest.mark.parametrize("n", [1, 63, 64, 65, 1000, 3001, 13000, 40000])
def test_single_system_plan(genga, n, cw, npg):
    items, rows, visits, entries = genga.genga_mutual_plan_check([n], cw, npg)
    g = (n + 63) // 64
    gpb = cw * npg
    blocks = (g + gpb - 1) // gpb
    # visits: every ordered pair of groups inside a block, every unordered pair across blocks
    inside = sum(min(gpb, g - b * gpb) ** 2 for b in range(blocks))
    across = (g * g - inside) // 2
    assert visits == inside + across
    assert 1 <= rows <= 192 and items >= blocks
    assert entries == rows * 3 * ((n + 1023) // 1024 * 1024)


@pytest.mark.parametrize("cw,npg", SHAPES)
def test_batch_plan(genga, cw, npg):
    sizes = [7000, 1, 0, 3001, 12000, 64, 2500, 16000, 1023]
    items, rows, visits, entries = genga.genga_mutual_plan_check(sizes, cw, npg)
    want = 0
    for n in sizes:
        g = (n + 63) // 64
        gpb = cw * npg
        inside = sum(min(gpb, g - b * gpb) ** 2 for b in range((g + gpb - 1) // gpb))
        want += inside + (g * g - inside) // 2
    assert visits == want and items > 0 and rows <= 192


def test_plan_check_arguments(genga):
    with pytest.raises(genga.GengaError):
        genga.genga_mutual_plan_check([], 12, 2)
    with pytest.raises(genga.GengaError):
        genga.genga_mutual_plan_check([100, -1], 12, 2)
    assert genga.genga_mutual_plan_check([0, 0], 12, 2) == (0, 0, 0, 0)

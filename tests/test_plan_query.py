"""sw_plan_query (host-only, no GPU): the plan the score pass gives a length
class follows sw_set_plan's overrides -- the first whose max_read_len covers
the class -- and otherwise the built-in cost model, whose choices are pinned
against brute force by tests/test_plan_host.py."""
import pytest


@pytest.fixture
def sw():
    import paper_1304_0681_gb300 as sw
    sw.sw_set_plan(0, 1, 8)
    yield sw
    sw.sw_set_plan(0, 1, 8)


def test_overrides_and_their_limits(sw):
    base = {m: sw.sw_plan_query(m, m + 100, 5) for m in (75, 100, 150, 250, 400, 800)}
    for m, (lanes, rows) in base.items():
        assert rows in sw.sw_plan_rows() and 1 <= lanes <= 32
        assert lanes * rows >= m or lanes == 32
    sw.sw_set_plan(100, 4, 25)
    sw.sw_set_plan(300, 32, 8)
    assert sw.sw_plan_query(75, 175, 5) == (4, 25)     # first covering override
    assert sw.sw_plan_query(100, 200, 5) == (4, 25)
    assert sw.sw_plan_query(150, 250, 5) == (32, 8)
    assert sw.sw_plan_query(400, 500, 5) == base[400]  # beyond every override
    sw.sw_set_plan(0, 1, 8)
    assert sw.sw_plan_query(150, 250, 5) == base[150]  # cleared
    # 50 rows need 6-bit row tags, which the 16-bit-key mode has wherever
    # the classifier uses it (bounds up to 510); wider bounds run without
    # keys: every class takes the 50-row override
    sw.sw_set_plan(150, 3, 50)
    assert sw.sw_plan_query(150, 250, 5) == (3, 50)    # bound 750: wide 16-bit mode
    assert sw.sw_plan_query(150, 250, 3) == (3, 50)    # bound 450: 16-bit keys
    assert sw.sw_plan_query(150, 250, 50) == (3, 50)   # bound 7500: wide 16-bit mode


def test_arguments_are_checked(sw):
    for args in ((0, 100, 5), (100, 0, 5), (100, 100, 0), (100, 100, 128), (100000, 100, 5)):
        with pytest.raises(sw.SwError):
            sw.sw_plan_query(*args)

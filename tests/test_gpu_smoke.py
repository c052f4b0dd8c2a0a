"""The driver's smoke check (one small TreePM step on cuda:0 against the
oracle) passes on this build."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke():
    import __graft_entry__ as g
    g.build()
    g.smoke()

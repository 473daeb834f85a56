"""The smoke entry point (one small scan on cuda:0 checked against the oracle) stays green."""
import pytest

pytestmark = pytest.mark.gpu


def test_graft_entry_smoke():
    import __graft_entry__
    __graft_entry__.smoke()

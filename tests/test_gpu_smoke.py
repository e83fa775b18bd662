"""The round-trip check the package ships as __graft_entry__.smoke(): one small rotation scene through
the autograd path on cuda:0, image and vertex gradient against the FP64 oracle, both solvers."""
import os
import sys

import pytest

pytestmark = pytest.mark.gpu


def test_smoke_passes():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import __graft_entry__

    __graft_entry__.smoke()

"""The package's smoke entry point (one small sigma and Davidson solve on cuda:0,
checked against the FP64 oracle) runs to completion."""
import os
import sys

import pytest

pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_smoke_entry_point():
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.smoke()

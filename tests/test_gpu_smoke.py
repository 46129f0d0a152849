"""The package's smoke entry point on cuda:0: one small well-balanced run in
FP64 and FP32-shifted storage through the C ABI, checked against the FP64
oracle."""
import pytest

import __graft_entry__ as entry
from tests.gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def test_smoke_runs_and_matches_the_oracle(capsys):
    need_gpu()
    entry.smoke()
    assert "smoke ok" in capsys.readouterr().out

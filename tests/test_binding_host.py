"""Host-side argument checks of the Python binding, on the CPU with a
stand-in for the C library: wrong shapes, dtypes or layouts never reach the
C side (which reads and writes as many elements as the lattice has), and a
batch remembers the shape of every admitted case."""
import ctypes

import numpy as np
import pytest

from paper_2012_11075_gb300 import wblbe


class FakeLib:
    """Records the C calls that get through; admits every case."""

    def __init__(self):
        self.calls = []
        self.next = 0

    def wblbe_batch_admit(self, h, cp, rho, tol, steps, cid):
        self.calls.append("admit")
        cid._obj.value = self.next
        self.next += 1
        return wblbe.OK

    def wblbe_batch_fetch(self, h, case_id, *args):
        self.calls.append(("fetch", case_id))
        return wblbe.OK

    def wblbe_batch_get_populations(self, h, case_id, f):
        self.calls.append(("pops", case_id))
        return wblbe.OK

    def wblbe_batch_retire(self, h, case_id):
        self.calls.append(("retire", case_id))
        return wblbe.OK

    def wblbe_moments(self, *args):
        self.calls.append("moments")
        return wblbe.OK


def _batch():
    b = object.__new__(wblbe.Batch)
    b.lib, b.h, b._shapes = FakeLib(), ctypes.c_void_p(1), {}
    return b


def test_batch_tracks_case_shapes():
    b = _batch()
    p = wblbe.Params(12, 5, 1.0, 0.01, 0.01, 1.0, 0.1)
    cid = b.admit(p, np.zeros((5, 12)), 1e-6, 100)
    assert b._shapes[cid] == (5, 12)
    b.get_populations(cid)
    b.fetch(cid, (5, 12))
    with pytest.raises(ValueError):
        b.fetch(cid, (12, 5))                 # wrong shape never reaches C
    with pytest.raises(ValueError):
        b.admit(p, np.zeros((12, 5)), 1e-6, 100)
    b.retire(cid)
    with pytest.raises(wblbe.WblbeError):
        b.get_populations(cid)                # retired: unknown case
    assert b.lib.calls == ["admit", ("pops", cid), ("fetch", cid), ("retire", cid)]


def test_solver_output_checks():
    torch = pytest.importorskip("torch")
    s = object.__new__(wblbe.Solver)
    s._torch, s.lib, s.h = torch, FakeLib(), ctypes.c_void_p(1)
    s.params = wblbe.Params(8, 4, 1.0, 0.01, 0.01, 1.0, 0.1)
    for bad in (np.zeros((4, 7)), np.zeros((4, 8), np.float32), np.zeros((8, 4)).T,
                torch.zeros(4, 8)):
        with pytest.raises(ValueError):
            s.moments_into(rho=bad)
    with pytest.raises(ValueError):
        s.init_rho(np.zeros((8, 4)))
    with pytest.raises(ValueError):
        s.set_populations(np.zeros((9, 8, 4)))
    s.moments_into(rho=np.zeros((4, 8)), mu=np.zeros((4, 8)))
    assert s.lib.calls == ["moments"]

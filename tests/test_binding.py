"""Host-side checks of the Python binding (no GPU needed)."""
import gc
import weakref

import pytest

torch = pytest.importorskip("torch")


def test_routing_descriptors_keep_their_tensors_alive():
    """fr_routing holds raw pointers; the descriptor must keep the tensors it
    points into alive, or a temporary's memory is reused while a kernel reads it."""
    from paper_2606_12800_gb300 import api
    d = torch.zeros((4, 5), dtype=torch.uint8)
    ref = weakref.ref(d)
    R = api.routing_d8(d)
    del d
    gc.collect()
    assert ref() is not None and R.dir == ref().data_ptr()
    m = torch.zeros((4, 5), dtype=torch.uint8)
    z = torch.zeros((4, 5), dtype=torch.float32)
    rm, rz = weakref.ref(m), weakref.ref(z)
    Rm = api.routing_mfd(m, z, 30.0, 1.1)
    del m, z
    gc.collect()
    assert rm() is not None and rz() is not None
    assert Rm.mask == rm().data_ptr() and Rm.dem == rz().data_ptr()

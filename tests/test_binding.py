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


def test_workspace_size_and_flags():
    """workspace_size follows fr_workspace_size (MFD adds the 32 B/cell of
    fractions that FR_WEIGHTS_IN_WORKSPACE keeps) and rejects empty grids;
    the workspace flags travel in the routing descriptors."""
    from paper_2606_12800_gb300 import _lib, api
    d8, mfd = api.workspace_size(300, 200), api.workspace_size(300, 200, mfd=True)
    assert mfd >= d8 + 300 * 200 * 32 and d8 % 256 == 0 and mfd % 256 == 0
    with pytest.raises(ValueError):
        api.workspace_size(0, 10)
    R = api.routing_d8(torch.zeros((4, 5), dtype=torch.uint8), _lib.FR_SINK_SUMS_IN_WORKSPACE)
    assert R.flags == _lib.FR_SINK_SUMS_IN_WORKSPACE
    Rm = api.routing_mfd(torch.zeros((4, 5), dtype=torch.uint8), torch.zeros((4, 5)), 30.0, 1.1,
                         _lib.FR_WEIGHTS_IN_WORKSPACE)
    assert Rm.flags == _lib.FR_WEIGHTS_IN_WORKSPACE
    assert _lib.FR_WEIGHTS_IN_WORKSPACE & _lib.FR_SINK_SUMS_IN_WORKSPACE == 0

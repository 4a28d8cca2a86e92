"""Host-side argument checks of the Python binding (no GPU): vectors the C
calls read or write must hold exactly the documented element count."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_host_vec_checks_length_and_makes_contiguous():
    import paper_2506_03070_gb300 as P
    a = np.arange(10.0)[::2]  # strided view of 5 elements
    v = P._host_vec(a, 5, "b")
    assert v.flags.c_contiguous and v.dtype == np.float64 and np.array_equal(v, a)
    same = np.arange(4.0)
    assert P._host_vec(same, 4, "b") is same  # no copy when already contiguous float64
    with pytest.raises(ValueError):
        P._host_vec(np.zeros(3), 4, "b")


def test_device_vec_refuses_host_tensors():
    import paper_2506_03070_gb300 as P
    with pytest.raises(TypeError):
        P._vec(torch.zeros(4, dtype=torch.float64), 4, "b")

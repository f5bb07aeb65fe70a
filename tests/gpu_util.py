"""Helpers for the GPU parity tests: device setup and error metrics."""
import numpy as np
import pytest


def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def tri():
    from paper_1609_01490_gb300 import tri as _t
    return _t


def rel_err(got, ref):
    """Per-element relative error |got - ref| / ref over ref > 0; zeros must match exactly."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    zero = ref == 0
    assert np.all(got[zero] == 0.0), f"{int(np.count_nonzero(got[zero]))} exact zeros missed"
    if np.all(zero):
        return 0.0
    return float(np.max(np.abs(got[~zero] - ref[~zero]) / ref[~zero]))
